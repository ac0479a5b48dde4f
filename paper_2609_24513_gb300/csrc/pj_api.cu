// C-ABI entry points: contexts, dataset loading (quantisation check, closed-
// manifold check and unique edges, per-mesh boxes, lexicographic vertex
// order), exports and counters.
//
// Loading follows the paper's preprocessing/loading split (Sec. 4.2): each
// dataset becomes flat triangles with a triangle-to-object map (here: per-mesh
// offset ranges) and a per-object unique-edge set (Sec. 3.1 Step I: interior
// edges of a closed manifold are shared by exactly two triangles, so each is
// kept once, owned by one of its triangles).
#include <cub/cub.cuh>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "pj_internal.cuh"

namespace pj {

thread_local Exec *t_exec = nullptr;

// a serving thread keeps its own message; API calls set the context's
pj_status fail(Ctx *c, pj_status code, const std::string &msg) {
  if (t_exec) {
    t_exec->err = msg;
  } else if (c) {
    std::lock_guard<std::mutex> lk(c->err_mu);
    c->err = msg;
  }
  return code;
}

void clear_err(Ctx *c) {
  std::lock_guard<std::mutex> lk(c->err_mu);
  c->err.clear();
}

pj_status cuda_fail(Ctx *c, cudaError_t e, const char *what) {
  std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" +
                  cudaGetErrorString(e) + ") in " + what;
  return fail(c, e == cudaErrorMemoryAllocation ? PJ_ERR_NO_MEMORY : PJ_ERR_CUDA, m);
}

pj_status exec_init(Ctx *ctx, Exec *e) {
  cudaError_t r = cudaMalloc(&e->d_err, sizeof(int) * 4);
  if (r == cudaSuccess) r = cudaMemset(e->d_err, 0, sizeof(int) * 4);
  if (r == cudaSuccess) r = cudaMallocHost(&e->h_pinned, 4096);
  for (auto &ev : e->ev)
    if (r == cudaSuccess) r = cudaEventCreate(&ev);
  if (r != cudaSuccess) return cuda_fail(ctx, r, "exec_init");
  return PJ_OK;
}

void exec_free(Exec *e) {
  if (e->stream) {
    for (auto &kv : e->ws)
      if (kv.second.ptr) cudaFreeAsync(kv.second.ptr, e->stream);
    cudaStreamSynchronize(e->stream);
  } else {
    for (auto &kv : e->ws) cudaFree(kv.second.ptr);
  }
  e->ws.clear();
  cudaFree(e->d_err);
  cudaFreeHost(e->h_pinned);
  for (auto &ev : e->ev)
    if (ev) cudaEventDestroy(ev);
  e->d_err = nullptr;
  e->h_pinned = nullptr;
  for (auto &ev : e->ev) ev = nullptr;
}

void *ws_get(Ctx *ctx, const char *name, size_t bytes, pj_status *st) {
  *st = PJ_OK;
  Exec *ex = cur_exec(ctx);
  Workspace &w = ex->ws[name];
  if (bytes == 0) bytes = 16;
  if (w.cap >= bytes) return w.ptr;
  const size_t old_cap = w.cap;
  w.zeroed = false;  // a new block, even at the same address, holds anything
  size_t want = bytes + bytes / 4;
  cudaError_t e;
  if (ex->stream) {
    // a serving slot: the old block is released and the new one taken in
    // the slot's stream order, so a growth does not wait for the batches of
    // the other slots (cudaFree would wait for the whole device); it grows
    // at least twofold, so that it grows a few times at most
    want = std::max(want, 2 * old_cap);
    if (w.ptr) cudaFreeAsync(w.ptr, ex->stream);
    w.ptr = nullptr;
    w.cap = 0;
    e = cudaMallocAsync(&w.ptr, want, ex->stream);
  } else {
    if (w.ptr) cudaFree(w.ptr);
    w.ptr = nullptr;
    w.cap = 0;
    e = cudaMalloc(&w.ptr, want);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    w.ptr = nullptr;
    *st = cuda_fail(ctx, e, name);
    return nullptr;
  }
  w.cap = want;
  // workspaces back captured graphs: a new address invalidates them (only
  // the context's own scratch is ever captured)
  if (ex == &ctx->main) {
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
  }
  return w.ptr;
}

void *ws_get_zeroed(Ctx *ctx, const char *name, size_t bytes, cudaStream_t s, pj_status *st) {
  Workspace &w = cur_exec(ctx)->ws[name];
  const void *before = w.ptr;
  void *p = ws_get(ctx, name, bytes, st);
  if (!p) return nullptr;
  if (p != before || !w.zeroed) {
    cudaError_t e = cudaMemsetAsync(p, 0, w.cap, s);
    if (e != cudaSuccess) {
      *st = cuda_fail(ctx, e, name);
      return nullptr;
    }
    w.zeroed = true;
  }
  return p;
}

void ws_mark_dirty(Ctx *ctx, const char *name) { cur_exec(ctx)->ws[name].zeroed = false; }

void *pool_get(Ctx *ctx, size_t bytes, cudaError_t *e) {
  *e = cudaSuccess;
  auto it = ctx->pool.lower_bound(bytes);
  if (it != ctx->pool.end() && it->first <= 4 * std::max<size_t>(bytes, 4096)) {
    void *p = it->second;
    ctx->pool_bytes -= it->first;
    ctx->pool.erase(it);
    return p;
  }
  size_t cap = 4096;
  while (cap < bytes) cap *= 2;
  void *p = nullptr;
  *e = cudaMalloc(&p, cap);
  if (*e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->pool_cap[p] = cap;
  return p;
}

void pool_put(Ctx *ctx, void *p) {
  if (!p) return;
  auto it = ctx->pool_cap.find(p);
  if (it == ctx->pool_cap.end()) {
    cudaFree(p);
    return;
  }
  if (ctx->pool_bytes + it->second > (size_t(1) << 30)) {
    cudaFree(p);
    ctx->pool_cap.erase(it);
    return;
  }
  ctx->pool.emplace(it->second, p);
  ctx->pool_bytes += it->second;
}

void pool_release(Ctx *ctx) {
  for (auto &kv : ctx->pool) {
    cudaFree(kv.second);
    ctx->pool_cap.erase(kv.second);
  }
  ctx->pool.clear();
  ctx->pool_bytes = 0;
  for (auto &kv : ctx->hpool) {
    cudaFreeHost(kv.second);
    ctx->hpool_cap.erase(kv.second);
  }
  ctx->hpool.clear();
  ctx->hpool_bytes = 0;
}

void *hpool_get(Ctx *ctx, size_t bytes, cudaError_t *e) {
  *e = cudaSuccess;
  auto it = ctx->hpool.lower_bound(bytes);
  if (it != ctx->hpool.end() && it->first <= 4 * std::max<size_t>(bytes, 4096)) {
    void *p = it->second;
    ctx->hpool_bytes -= it->first;
    ctx->hpool.erase(it);
    return p;
  }
  size_t cap = 4096;
  while (cap < bytes) cap *= 2;
  void *p = nullptr;
  *e = cudaMallocHost(&p, cap);
  if (*e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->hpool_cap[p] = cap;
  return p;
}

void hpool_put(Ctx *ctx, void *p) {
  if (!p) return;
  auto it = ctx->hpool_cap.find(p);
  if (it == ctx->hpool_cap.end()) {
    cudaFreeHost(p);
    return;
  }
  if (ctx->hpool_bytes + it->second > (size_t(1) << 28)) {
    cudaFreeHost(p);
    ctx->hpool_cap.erase(it);
    return;
  }
  ctx->hpool.emplace(it->second, p);
  ctx->hpool_bytes += it->second;
}

void pairs_release(Ctx *ctx, pj_pairs *r) {
  if (r->pairs) {
    if (r->on_device) pool_put(ctx, r->pairs);
    else if (r->pairs_malloc) free(r->pairs);
    else hpool_put(ctx, r->pairs);
  }
  pool_put(ctx, r->flags);
  pool_put(ctx, r->cycles);
  memset(r, 0, sizeof(*r));
}

// ---------------------------------------------------------------------------
// Load kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t mesh_of(const int64_t *off, int64_t M, int64_t e) {
  // largest m with off[m] <= e (meshes may be empty)
  int64_t lo = 0, hi = M - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_validate_xyz(const float *xyz, int64_t n, unsigned long long *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f = xyz[i];
    bool ok = (f >= 0.f) && (f < 262144.f) && (f == floorf(f));
    if (!ok) atomicMin(bad, (unsigned long long)i);
  }
}

__global__ void k_convert_tris(const int32_t *tris_local, int64_t F,
                               const int64_t *voff, const int64_t *toff,
                               int64_t M, int32_t *tris_g,
                               unsigned long long *bad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t m = mesh_of(toff, M, t);
    int64_t nv = voff[m + 1] - voff[m];
    int a = tris_local[3 * t], b = tris_local[3 * t + 1], c = tris_local[3 * t + 2];
    bool ok = a >= 0 && b >= 0 && c >= 0 && a < nv && b < nv && c < nv &&
              a != b && b != c && a != c;
    if (!ok) {
      atomicMin(bad, (unsigned long long)t);
      a = b = c = 0;
    }
    tris_g[3 * t] = (int32_t)(voff[m] + a);
    tris_g[3 * t + 1] = (int32_t)(voff[m] + b);
    tris_g[3 * t + 2] = (int32_t)(voff[m] + c);
  }
}

// one block per mesh: closed bounding box of its vertices
// per-mesh record (see Dataset::d_mrec); runs after the boxes and the
// lexicographic order exist
__global__ void k_mesh_rec(const float *aabb, const float *xyz, const int32_t *lexorder,
                           const int64_t *voff, const int64_t *toff, int64_t M, float4 *rec) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    const float *b = aabb + 6 * m;
    const int64_t v0 = voff[m], nv = voff[m + 1] - v0;
    float x = 0.f, y = 0.f, z = 0.f;
    if (nv > 0) {
      const int64_t g = lexorder[v0];
      x = xyz[3 * g];
      y = xyz[3 * g + 1];
      z = xyz[3 * g + 2];
    }
    rec[3 * m] = make_float4(b[0], b[1], b[2], x);
    rec[3 * m + 1] = make_float4(b[3], b[4], b[5], y);
    rec[3 * m + 2] = make_float4(z, __int_as_float((int)toff[m]), __int_as_float((int)v0),
                                 __int_as_float((int)nv));
  }
}

__global__ void k_mesh_aabb(const float *xyz, const int64_t *voff, int64_t M,
                            float *aabb) {
  __shared__ float red[6][32];
  for (int64_t m = blockIdx.x; m < M; m += gridDim.x) {
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    for (int64_t v = voff[m] + threadIdx.x; v < voff[m + 1]; v += blockDim.x) {
      for (int d = 0; d < 3; ++d) {
        float f = xyz[3 * v + d];
        lo[d] = fminf(lo[d], f);
        hi[d] = fmaxf(hi[d], f);
      }
    }
    for (int d = 0; d < 3; ++d) {
      for (int o = 16; o > 0; o >>= 1) {
        lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
        hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
      }
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
      for (int d = 0; d < 3; ++d) { red[d][w] = lo[d]; red[3 + d][w] = hi[d]; }
    __syncthreads();
    if (threadIdx.x < 32) {
      int nw = blockDim.x >> 5;
      for (int d = 0; d < 3; ++d) {
        float a = l < nw ? red[d][l] : 3e38f, b = l < nw ? red[3 + d][l] : -3e38f;
        for (int o = 16; o > 0; o >>= 1) {
          a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
          b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (l == 0) { aabb[6 * m + d] = a; aabb[6 * m + 3 + d] = b; }
      }
    }
    __syncthreads();
  }
}

__global__ void k_halfedges(const int32_t *tris_g, int64_t F, uint64_t *keys,
                            uint32_t *vals) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F;
       t += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) {
      uint32_t a = (uint32_t)tris_g[3 * t + k], b = (uint32_t)tris_g[3 * t + (k + 1) % 3];
      uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
      keys[3 * t + k] = ((uint64_t)lo << 32) | hi;
      vals[3 * t + k] = (uint32_t)(3 * t + k);
    }
  }
}

// sorted half-edges: every key must occur exactly twice; the first of each
// run owns the edge
__global__ void k_edge_runs(const uint64_t *keys, const uint32_t *vals, int64_t n,
                            uint32_t *owner_bits, unsigned long long *n_unique,
                            unsigned long long *bad) {
  unsigned long long local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    if (i > 0 && keys[i - 1] == k) continue;  // not a run head
    bool two = (i + 1 < n) && keys[i + 1] == k && !((i + 2 < n) && keys[i + 2] == k);
    if (!two) atomicMin(bad, (unsigned long long)vals[i]);
    uint32_t v = vals[i];
    atomicOr(&owner_bits[v / 3], 1u << (v % 3));
    ++local;
  }
  if (local) atomicAdd(n_unique, local);
}

__global__ void k_pack_u8(const uint32_t *in, uint8_t *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint8_t)in[i];
}

__global__ void k_lex_keys(const float *xyz, int64_t V, const int64_t *voff,
                           int64_t M, uint64_t *kxyz, uint32_t *kmesh,
                           int32_t *ids) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x = (uint64_t)xyz[3 * v], y = (uint64_t)xyz[3 * v + 1],
             z = (uint64_t)xyz[3 * v + 2];
    kxyz[v] = (x << 36) | (y << 18) | z;
    kmesh[v] = (uint32_t)mesh_of(voff, M, v);
    ids[v] = (int32_t)v;
  }
}

__global__ void k_gather_u32(const uint32_t *src, const int32_t *idx, uint32_t *dst,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

static int nblk(Ctx *ctx, int64_t n, int t = 256) {
  int64_t b = (n + t - 1) / t;
  int64_t cap = (int64_t)ctx->num_sms * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
static cudaError_t dalloc(T **p, int64_t n) {
  return cudaMalloc((void **)p, sizeof(T) * (size_t)(n > 0 ? n : 1));
}

void free_bvh(Bvh &b) {
  cudaFree(b.d_nodes);
  cudaFree(b.d_roots);
  cudaFree(b.d_tri_order);
  cudaFree(b.d_trirec);
  b = Bvh();
}

void free_dataset(Dataset *d) {
  for (auto &kv : d->bvhs) free_bvh(kv.second);
  for (auto &kv : d->dbvhs) free_bvh(kv.second);
  cudaFree(d->d_xyz);
  cudaFree(d->d_tris);
  cudaFree(d->d_voff);
  cudaFree(d->d_toff);
  cudaFree(d->d_aabb);
  cudaFree(d->d_lexorder);
  cudaFree(d->d_emask);
  cudaFree(d->d_mrec);
}

// RAII for temporary device buffers of the load pipeline
struct Tmp {
  std::vector<void *> p;
  ~Tmp() {
    for (void *q : p) cudaFree(q);
  }
  template <typename T>
  cudaError_t get(T **out, int64_t n) {
    cudaError_t e = dalloc(out, n);
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
};

pj_status load_impl(Ctx *ctx, const float *xyz, int64_t V,
                           const int32_t *tris, int64_t F, const int64_t *voff,
                           const int64_t *toff, int64_t M, int dev_ptrs,
                           Dataset *d) {
  cudaStream_t s = ctx->stream;
  if (M <= 0) return fail(ctx, PJ_ERR_INVALID_ARG, "n_meshes must be positive");
  if (!voff || !toff) return fail(ctx, PJ_ERR_INVALID_ARG, "offset arrays are required");
  if (voff[0] != 0 || toff[0] != 0 || voff[M] != V || toff[M] != F)
    return fail(ctx, PJ_ERR_INVALID_ARG, "offsets must start at 0 and end at n_verts / n_tris");
  for (int64_t m = 0; m < M; ++m) {
    if (voff[m + 1] < voff[m] || toff[m + 1] < toff[m])
      return fail(ctx, PJ_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (toff[m + 1] - toff[m] > (1 << 28) - 2)
      return fail(ctx, PJ_ERR_INVALID_ARG, "a mesh has more than 2^28 - 2 triangles");
    if (toff[m + 1] == toff[m])
      return fail(ctx, PJ_ERR_NOT_MANIFOLD, "mesh " + std::to_string(m) + " has no triangles");
  }
  if (V >= (1ll << 31) - 1 || F >= (1ll << 31) - 1 || 3 * F >= (1ll << 32))
    return fail(ctx, PJ_ERR_INVALID_ARG, "dataset too large (2^31 - 1 vertices / triangles)");
  if ((V > 0 && !xyz) || (F > 0 && !tris)) return fail(ctx, PJ_ERR_INVALID_ARG, "null input");

  d->M = M; d->V = V; d->F = F;
  d->h_voff.assign(voff, voff + M + 1);
  d->h_toff.assign(toff, toff + M + 1);
  PJ_CK(dalloc(&d->d_xyz, 3 * V));
  PJ_CK(dalloc(&d->d_tris, 3 * F));
  PJ_CK(dalloc(&d->d_voff, M + 1));
  PJ_CK(dalloc(&d->d_toff, M + 1));
  PJ_CK(dalloc(&d->d_aabb, 6 * M));
  PJ_CK(dalloc(&d->d_lexorder, V));
  PJ_CK(dalloc(&d->d_emask, F));
  PJ_CK(dalloc(&d->d_mrec, 3 * M));
  d->bytes = 12 * V + 12 * F + 16 * (M + 1) + 24 * M + 4 * V + F + 48 * M;

  Tmp tmp;
  int32_t *tris_local = nullptr;
  cudaMemcpyKind k = dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  PJ_CK(cudaMemcpyAsync(d->d_xyz, xyz, sizeof(float) * 3 * V, k, s));
  PJ_CK(tmp.get(&tris_local, 3 * F));
  PJ_CK(cudaMemcpyAsync(tris_local, tris, sizeof(int32_t) * 3 * F, k, s));
  PJ_CK(cudaMemcpyAsync(d->d_voff, voff, sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, s));
  PJ_CK(cudaMemcpyAsync(d->d_toff, toff, sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, s));

  unsigned long long *d_flags = nullptr;  // [0] bad coord, [1] bad tri, [2] bad edge, [3] n unique
  PJ_CK(tmp.get(&d_flags, 4));
  unsigned long long init[4] = {~0ull, ~0ull, ~0ull, 0ull};
  PJ_CK(cudaMemcpyAsync(d_flags, init, sizeof(init), cudaMemcpyHostToDevice, s));

  if (V > 0) k_validate_xyz<<<nblk(ctx, 3 * V), 256, 0, s>>>(d->d_xyz, 3 * V, d_flags);
  k_convert_tris<<<nblk(ctx, F), 256, 0, s>>>(tris_local, F, d->d_voff, d->d_toff, M,
                                              d->d_tris, d_flags + 1);
  PJ_CK(cudaGetLastError());
  unsigned long long hf[4];
  PJ_CK(cudaMemcpyAsync(hf, d_flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  if (hf[0] != ~0ull) {
    int64_t i = (int64_t)hf[0];
    char buf[160];
    snprintf(buf, sizeof(buf), "vertex %lld coordinate %lld is not an integer in [0, 2^18)",
             (long long)(i / 3), (long long)(i % 3));
    return fail(ctx, PJ_ERR_NOT_QUANTIZED, buf);
  }
  if (hf[1] != ~0ull) {
    int64_t t = (int64_t)hf[1];
    int64_t m = std::upper_bound(d->h_toff.begin(), d->h_toff.end(), t) - d->h_toff.begin() - 1;
    char buf[200];
    snprintf(buf, sizeof(buf), "triangle %lld of mesh %lld has a vertex id out of range "
             "or repeats a vertex", (long long)(t - d->h_toff[m]), (long long)m);
    return fail(ctx, PJ_ERR_NOT_MANIFOLD, buf);
  }

  k_mesh_aabb<<<(int)std::min<int64_t>(M, 65535), 256, 0, s>>>(d->d_xyz, d->d_voff, M, d->d_aabb);
  PJ_CK(cudaGetLastError());

  // unique edges and the closed-manifold check
  {
    int64_t n = 3 * F;
    uint64_t *k0, *k1;
    uint32_t *v0, *v1, *bits;
    PJ_CK(tmp.get(&k0, n));
    PJ_CK(tmp.get(&k1, n));
    PJ_CK(tmp.get(&v0, n));
    PJ_CK(tmp.get(&v1, n));
    PJ_CK(tmp.get(&bits, F));
    PJ_CK(cudaMemsetAsync(bits, 0, sizeof(uint32_t) * F, s));
    k_halfedges<<<nblk(ctx, F), 256, 0, s>>>(d->d_tris, F, k0, v0);
    size_t tb = 0;
    PJ_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, k0, k1, v0, v1, (int)n, 0, 64, s));
    void *tstore;
    PJ_CK(tmp.get((char **)&tstore, (int64_t)tb));
    PJ_CK(cub::DeviceRadixSort::SortPairs(tstore, tb, k0, k1, v0, v1, (int)n, 0, 64, s));
    k_edge_runs<<<nblk(ctx, n), 256, 0, s>>>(k1, v1, n, bits, d_flags + 3, d_flags + 2);
    k_pack_u8<<<nblk(ctx, F), 256, 0, s>>>(bits, d->d_emask, F);
    PJ_CK(cudaGetLastError());
  }
  // per-mesh lexicographic vertex order: stable sort by (x, y, z), then
  // stable sort by mesh
  if (V > 0) {
    uint64_t *kx, *kx2;
    uint32_t *km, *km2;
    int32_t *ids, *ids2;
    PJ_CK(tmp.get(&kx, V));
    PJ_CK(tmp.get(&kx2, V));
    PJ_CK(tmp.get(&km, V));
    PJ_CK(tmp.get(&km2, V));
    PJ_CK(tmp.get(&ids, V));
    PJ_CK(tmp.get(&ids2, V));
    k_lex_keys<<<nblk(ctx, V), 256, 0, s>>>(d->d_xyz, V, d->d_voff, M, kx, km, ids);
    size_t tb = 0;
    PJ_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, kx, kx2, ids, ids2, (int)V, 0, 54, s));
    size_t tb2 = 0;
    PJ_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb2, km, km2, ids2, d->d_lexorder, (int)V, 0, 32, s));
    void *tstore;
    PJ_CK(tmp.get((char **)&tstore, (int64_t)std::max(tb, tb2)));
    PJ_CK(cub::DeviceRadixSort::SortPairs(tstore, tb, kx, kx2, ids, ids2, (int)V, 0, 54, s));
    // mesh ids in the xyz-sorted order
    k_gather_u32<<<nblk(ctx, V), 256, 0, s>>>(km, ids2, km2, V);
    PJ_CK(cub::DeviceRadixSort::SortPairs(tstore, tb2, km2, km, ids2, d->d_lexorder, (int)V, 0, 32, s));
    PJ_CK(cudaGetLastError());
  }
  if (M > 0) {
    k_mesh_rec<<<nblk(ctx, M), 256, 0, s>>>(d->d_aabb, d->d_xyz, d->d_lexorder, d->d_voff,
                                            d->d_toff, M, d->d_mrec);
    PJ_CK(cudaGetLastError());
  }
  PJ_CK(cudaMemcpyAsync(hf, d_flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  if (hf[2] != ~0ull) {
    int64_t t = (int64_t)(hf[2] / 3);
    int64_t m = std::upper_bound(d->h_toff.begin(), d->h_toff.end(), t) - d->h_toff.begin() - 1;
    char buf[200];
    snprintf(buf, sizeof(buf), "mesh %lld is not a closed manifold: an edge of its triangle "
             "%lld is not shared by exactly two triangles", (long long)m,
             (long long)(t - d->h_toff[m]));
    return fail(ctx, PJ_ERR_NOT_MANIFOLD, buf);
  }
  d->E = (int64_t)hf[3];
  d->h_aabb.resize(6 * (size_t)M);
  if (M > 0)
    PJ_CK(cudaMemcpy(d->h_aabb.data(), d->d_aabb, sizeof(float) * 6 * M, cudaMemcpyDeviceToHost));
  // the admission grid: per cell the meshes whose box touches it, then the
  // summed-area table of those counts
  const int G = kOccG, G1 = kOccG + 1;
  const double cw = 262144.0 / G;
  std::vector<int64_t> cnt((size_t)G * G * G, 0);
  for (int64_t m = 0; m < M; ++m) {
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(G - 1, std::max(0, (int)(d->h_aabb[6 * m + k] / cw)));
      hi[k] = std::min(G - 1, std::max(0, (int)(d->h_aabb[6 * m + 3 + k] / cw)));
    }
    for (int x = lo[0]; x <= hi[0]; ++x)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int z = lo[2]; z <= hi[2]; ++z) cnt[((size_t)x * G + y) * G + z] += 1;
  }
  d->occ_sat.assign((size_t)G1 * G1 * G1, 0);
  auto S = [&](int x, int y, int z) -> int64_t & { return d->occ_sat[((size_t)x * G1 + y) * G1 + z]; };
  for (int x = 1; x <= G; ++x)
    for (int y = 1; y <= G; ++y)
      for (int z = 1; z <= G; ++z)
        S(x, y, z) = cnt[((size_t)(x - 1) * G + (y - 1)) * G + (z - 1)] + S(x - 1, y, z) +
                     S(x, y - 1, z) + S(x, y, z - 1) - S(x - 1, y - 1, z) - S(x - 1, y, z - 1) -
                     S(x, y - 1, z - 1) + S(x - 1, y - 1, z - 1);
  return PJ_OK;
}

int64_t window_mesh_bound(const Dataset *d, const int32_t *wlo, const int32_t *whi) {
  const int G = kOccG, G1 = kOccG + 1;
  if (d->occ_sat.size() != (size_t)G1 * G1 * G1) return d->M;
  const double cw = 262144.0 / G;
  int a[3], b[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = std::min(G - 1, std::max(0, (int)(wlo[k] / cw)));
    b[k] = std::min(G - 1, std::max(0, (int)(whi[k] / cw))) + 1;
  }
  auto S = [&](int x, int y, int z) { return d->occ_sat[((size_t)x * G1 + y) * G1 + z]; };
  const int64_t sum = S(b[0], b[1], b[2]) - S(a[0], b[1], b[2]) - S(b[0], a[1], b[2]) -
                      S(b[0], b[1], a[2]) + S(a[0], a[1], b[2]) + S(a[0], b[1], a[2]) +
                      S(b[0], a[1], a[2]) - S(a[0], a[1], a[2]);
  return std::min(sum, d->M);
}

}  // namespace pj

using namespace pj;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

pj_status pj_create(const pj_config *cfg, pj_ctx **out) {
  if (!out) return PJ_ERR_INVALID_ARG;
  *out = nullptr;
  Ctx *ctx = new (std::nothrow) Ctx();
  if (!ctx) return PJ_ERR_NO_MEMORY;
  if (cfg) ctx->cfg = *cfg;
  ctx->device = cfg ? cfg->device : 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counters, sizeof(unsigned long long) * C_NUM);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * C_NUM);
  if (e != cudaSuccess || exec_init(ctx, &ctx->main) != PJ_OK) {
    cudaGetLastError();
    exec_free(&ctx->main);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? PJ_ERR_NO_MEMORY : PJ_ERR_CUDA;
  }
  *out = reinterpret_cast<pj_ctx *>(ctx);
  return PJ_OK;
}

pj_status pj_destroy(pj_ctx *h) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return PJ_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  serve_stop(ctx);
  // work that reads the datasets may sit on any stream of the device (the
  // allocation-free join runs on the caller's), so wait for all of it
  cudaDeviceSynchronize();
  for (auto &kv : ctx->datasets) free_dataset(kv.second.get());
  for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
  exec_free(&ctx->main);
  pool_release(ctx);
  cudaFree(ctx->d_counters);
  cudaStreamDestroy(ctx->stream);
  delete ctx;
  return PJ_OK;
}

const char *pj_last_error(pj_ctx *h) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

pj_status pj_load_meshes(pj_ctx *h, const float *xyz, int64_t n_verts,
                         const int32_t *tris, int64_t n_tris,
                         const int64_t *mesh_vert_off, const int64_t *mesh_tri_off,
                         int64_t n_meshes, int32_t ptr_is_device, pj_dataset *out) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  if (n_verts < 0 || n_tris < 0) return fail(ctx, PJ_ERR_INVALID_ARG, "negative size");
  cudaSetDevice(ctx->device);
  std::unique_ptr<Dataset> d(new Dataset());
  pj_status st = load_impl(ctx, xyz, n_verts, tris, n_tris, mesh_vert_off, mesh_tri_off,
                           n_meshes, ptr_is_device, d.get());
  if (st != PJ_OK) {
    cudaStreamSynchronize(ctx->stream);
    free_dataset(d.get());
    return st;
  }
  std::unique_lock<std::shared_mutex> wl(ctx->ds_rw);
  int id = ctx->next_ds++;
  ctx->datasets[id] = std::move(d);
  *out = id;
  return PJ_OK;
}

static Dataset *get_ds(Ctx *ctx, pj_dataset id) {
  auto it = ctx->datasets.find(id);
  return it == ctx->datasets.end() ? nullptr : it->second.get();
}

pj_status pj_free_dataset(pj_ctx *h, pj_dataset id) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::unique_lock<std::shared_mutex> wl(ctx->ds_rw);
  Dataset *d = get_ds(ctx, id);
  if (!d) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  if (serve_uses(ctx, d))
    return fail(ctx, PJ_ERR_BUSY, "serving queries on this dataset have not been polled yet");
  cudaSetDevice(ctx->device);
  // joins that read this dataset may still run on a caller's stream (the
  // allocation-free join returns once its work is queued): wait for the
  // whole device, not only the context's stream
  cudaDeviceSynchronize();
  free_dataset(d);
  ctx->datasets.erase(id);
  for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
  ctx->graphs.clear();
  return PJ_OK;
}

pj_status pj_build_bvh(pj_ctx *h, pj_dataset id, const pj_bvh_params *p) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::unique_lock<std::shared_mutex> wl(ctx->ds_rw);
  clear_err(ctx);
  Dataset *d = get_ds(ctx, id);
  if (!d) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  int W = p && p->width ? p->width : 4, L = p && p->leaf_size ? p->leaf_size : 4;
  if (!(W == 2 || W == 4 || W == 8) || !(L == 1 || L == 2 || L == 4 || L == 8))
    return fail(ctx, PJ_ERR_INVALID_ARG, "width must be 2, 4 or 8 and leaf size 1, 2, 4 or 8");
  cudaSetDevice(ctx->device);
  if (d->bvhs.count({W, L})) {
    d->last_bvh = {W, L};
    return PJ_OK;
  }
  pj_status st = build_bvh(ctx, d, W, L, ctx->stream);
  if (st == PJ_OK) d->last_bvh = {W, L};
  return st;
}

pj_status pj_dataset_info_get(pj_ctx *h, pj_dataset id, pj_dataset_info *out) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  Dataset *d = get_ds(ctx, id);
  if (!d) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  memset(out, 0, sizeof(*out));
  out->n_meshes = d->M;
  out->n_verts = d->V;
  out->n_tris = d->F;
  out->n_edges = d->E;
  out->device_bytes = d->bytes;
  auto it = d->bvhs.find(d->last_bvh);
  if (it != d->bvhs.end()) {
    out->bvh_nodes = it->second.n_nodes;
    out->bvh_width = it->second.W;
    out->bvh_leaf_size = it->second.L;
    out->bvh_max_depth = it->second.max_depth;
  }
  for (auto &kv : d->bvhs) out->device_bytes += kv.second.bytes;
  return PJ_OK;
}

pj_status pj_join_intersects(pj_ctx *h, pj_dataset a, pj_dataset b,
                             const int32_t *cand, int64_t n_cand, int32_t self_join,
                             void *stream, pj_pairs *out) {
  return pj_join_intersects_ex(h, a, b, cand, nullptr, n_cand, 0, self_join, nullptr,
                               stream, out);
}

pj_status pj_join_intersects_ex(pj_ctx *h, pj_dataset a, pj_dataset b,
                                const int32_t *cand, const int32_t *cand_off,
                                int64_t n_cand, int32_t cand_on_device,
                                int32_t self_join, const pj_join_opts *opts,
                                void *stream, pj_pairs *out) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  memset(out, 0, sizeof(*out));
  Dataset *A = get_ds(ctx, a), *B = get_ds(ctx, b);
  if (!A || !B) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  if (self_join && a != b) return fail(ctx, PJ_ERR_INVALID_ARG, "self_join needs a == b");
  if (cand && n_cand < 0) return fail(ctx, PJ_ERR_INVALID_ARG, "negative n_cand");
  if (!cand && cand_off) return fail(ctx, PJ_ERR_INVALID_ARG, "offsets need explicit candidates");
  cudaSetDevice(ctx->device);
  pj_join_opts o{};
  if (opts) o = *opts;
  return run_join(ctx, A, B, cand, cand_off, cand ? n_cand : -1, cand_on_device, self_join,
                  &o, stream ? (cudaStream_t)stream : ctx->stream, out);
}

pj_status pj_join_intersects_noalloc(pj_ctx *h, pj_dataset a, pj_dataset b,
                                     const int32_t *d_cand, int64_t n_cand, uint8_t *d_flags,
                                     int32_t *d_pairs, int64_t *d_count, void *stream) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  Dataset *A = get_ds(ctx, a), *B = get_ds(ctx, b);
  if (!A || !B) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  cudaSetDevice(ctx->device);
  return run_join_noalloc(ctx, A, B, d_cand, n_cand, d_flags, d_pairs, d_count,
                          stream ? (cudaStream_t)stream : ctx->stream);
}

pj_status pj_join_tiled(pj_ctx *h, const pj_host_meshes *a, const pj_host_meshes *b,
                        int32_t self_join, const pj_tiled_opts *opts, pj_pairs *out,
                        pj_tiled_stats *stats) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out || !a || (!self_join && !b)) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  memset(out, 0, sizeof(*out));
  cudaSetDevice(ctx->device);
  pj_tiled_opts o{};
  if (opts) o = *opts;
  return run_join_tiled(ctx, a, b, self_join, &o, out, stats);
}

pj_status pj_dataset_join(pj_ctx *h, pj_dataset a, pj_dataset b, int32_t self_join,
                          const pj_dsjoin_opts *opts, pj_pairs *out, pj_dsjoin_stats *stats) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  memset(out, 0, sizeof(*out));
  Dataset *A = get_ds(ctx, a), *B = get_ds(ctx, b);
  if (!A || !B) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  if (self_join && a != b) return fail(ctx, PJ_ERR_INVALID_ARG, "self_join needs a == b");
  cudaSetDevice(ctx->device);
  pj_dsjoin_opts o{};
  if (opts) o = *opts;
  return run_dataset_join(ctx, A, B, self_join, &o, out, stats, ctx->stream);
}

pj_status pj_estimate_join(pj_ctx *h, pj_dataset a, pj_dataset b, int32_t grid,
                           double *cells_out, pj_estimate *out) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  Dataset *A = get_ds(ctx, a), *B = get_ds(ctx, b);
  if (!A || !B) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  if (grid < 0) return fail(ctx, PJ_ERR_INVALID_ARG, "negative grid");
  cudaSetDevice(ctx->device);
  return run_estimate(ctx, A, B, grid, cells_out, out, ctx->stream);
}

pj_status pj_submit(pj_ctx *h, const pj_query *q, pj_ticket *out) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !q || !out) return PJ_ERR_INVALID_ARG;
  *out = 0;
  std::shared_lock<std::shared_mutex> rl(ctx->ds_rw);
  auto ia = ctx->datasets.find(q->a), ib = ctx->datasets.find(q->b);
  if (ia == ctx->datasets.end() || ib == ctx->datasets.end()) return PJ_ERR_INVALID_ARG;
  if (q->self_join && q->a != q->b) return PJ_ERR_INVALID_ARG;
  return serve_submit(ctx, ia->second.get(), ib->second.get(), q, out);
}

pj_status pj_poll(pj_ctx *h, pj_ticket t, int32_t wait, pj_pairs *out, pj_query_stats *stats) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  return serve_poll(ctx, t, wait, out, stats);
}

pj_status pj_free_pairs(pj_ctx *h, pj_pairs *res) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !res) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  pairs_release(ctx, res);
  return PJ_OK;
}

pj_status pj_autotune(pj_ctx *h, pj_dataset a, pj_dataset b, const int32_t *cand,
                      int64_t n_cand, int32_t self_join, const pj_tune_space *space,
                      pj_join_opts *best, pj_tune_entry *table, int32_t table_cap,
                      int32_t *table_n) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !space || !best) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::unique_lock<std::shared_mutex> wl(ctx->ds_rw);
  clear_err(ctx);
  Dataset *A = get_ds(ctx, a), *B = get_ds(ctx, b);
  if (!A || !B) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  if (self_join && a != b) return fail(ctx, PJ_ERR_INVALID_ARG, "self_join needs a == b");
  cudaSetDevice(ctx->device);
  int n = 0;
  pj_status st = run_autotune(ctx, A, B, cand, cand ? n_cand : -1, self_join, space, best, table,
                              table ? table_cap : 0, &n);
  if (table_n) *table_n = n;
  return st;
}

pj_status pj_get_counters(pj_ctx *h, pj_counters *out) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !out) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  unsigned long long c[C_NUM];
  cudaError_t e = cudaMemcpy(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pj_get_counters");
  memset(out, 0, sizeof(*out));
  out->pairs_refined = c[C_PAIRS];
  out->node_pairs = c[C_NODE_PAIRS];
  out->box_tests = c[C_BOX_TESTS];
  out->leaf_pairs = c[C_LEAF_PAIRS];
  out->edge_slab_tests = c[C_SLAB_TESTS];
  out->segtri_tests = c[C_SEGTRI];
  out->exact_fallbacks = c[C_FALLBACK];
  out->parity_rays = c[C_PARITY_RAYS];
  out->parity_nodes = c[C_PARITY_NODES];
  out->parity_tri_tests = c[C_PARITY_TRIS];
  out->bytes_fetched = c[C_BYTES];
  out->pairs_hit = c[C_HITS];
  out->kernel_launches = ctx->launches.load();
  out->tasks_spilled = c[C_SPILLED];
  out->tasks_resumed = c[C_TASKS];
  out->bytes_tasks = c[C_BYTES_TASKS];
  out->bytes_parity = c[C_BYTES_PARITY];
  out->bytes_expand = c[C_BYTES_EXPAND];
  out->bytes_leaf = c[C_BYTES_LEAF];
  out->parity_handed_over = c[C_PAR_HANDOVER];
  return PJ_OK;
}

pj_status pj_reset_counters(pj_ctx *h) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * C_NUM);
  ctx->launches = 0;
  return e == cudaSuccess ? PJ_OK : cuda_fail(ctx, e, "pj_reset_counters");
}

pj_status pj_segtri_batch(pj_ctx *h, const float *pq, const float *abc, int64_t n,
                          int32_t mode, uint8_t *res, int64_t *n_fallback, void *stream) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || n < 0 || (n > 0 && (!pq || !abc || !res))) return PJ_ERR_INVALID_ARG;
  if (mode != PJ_LEAF_FILTERED && mode != PJ_LEAF_EXACT && mode != PJ_LEAF_STATIC)
    return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  clear_err(ctx);
  cudaSetDevice(ctx->device);
  return run_segtri_batch(ctx, pq, abc, n, mode, res, n_fallback,
                          stream ? (cudaStream_t)stream : ctx->stream);
}

pj_status pj_export_bvh(pj_ctx *h, pj_dataset id, int32_t W, int32_t L, int32_t *nodes,
                        int32_t *roots, int32_t *tri_order, int64_t *n_nodes) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx || !n_nodes) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  Dataset *d = get_ds(ctx, id);
  if (!d) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  auto it = d->bvhs.find({W, L});
  if (it == d->bvhs.end()) return fail(ctx, PJ_ERR_INVALID_ARG, "no BVH with that width / leaf size");
  Bvh &b = it->second;
  cudaSetDevice(ctx->device);
  *n_nodes = b.n_nodes;
  int sw = node_stride_words(W);
  if (nodes) PJ_CK(cudaMemcpy(nodes, b.d_nodes, 4 * (size_t)b.n_nodes * sw, cudaMemcpyDeviceToHost));
  if (roots) PJ_CK(cudaMemcpy(roots, b.d_roots, 4 * d->M, cudaMemcpyDeviceToHost));
  if (tri_order) {
    PJ_CK(cudaMemcpy(tri_order, b.d_tri_order, 4 * d->F, cudaMemcpyDeviceToHost));
    for (int64_t m = 0; m < d->M; ++m)
      for (int64_t t = d->h_toff[m]; t < d->h_toff[m + 1]; ++t)
        tri_order[t] -= (int32_t)d->h_toff[m];
  }
  return PJ_OK;
}

pj_status pj_export_mesh_data(pj_ctx *h, pj_dataset id, float *aabb, int32_t *lex_first,
                              uint8_t *edge_owner) {
  Ctx *ctx = reinterpret_cast<Ctx *>(h);
  if (!ctx) return PJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  Dataset *d = get_ds(ctx, id);
  if (!d) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown dataset");
  cudaSetDevice(ctx->device);
  if (aabb) PJ_CK(cudaMemcpy(aabb, d->d_aabb, sizeof(float) * 6 * d->M, cudaMemcpyDeviceToHost));
  if (edge_owner) PJ_CK(cudaMemcpy(edge_owner, d->d_emask, d->F, cudaMemcpyDeviceToHost));
  if (lex_first) {
    std::vector<int32_t> lo((size_t)d->V);
    PJ_CK(cudaMemcpy(lo.data(), d->d_lexorder, 4 * d->V, cudaMemcpyDeviceToHost));
    for (int64_t m = 0; m < d->M; ++m)
      lex_first[m] = d->h_voff[m + 1] > d->h_voff[m]
                         ? lo[d->h_voff[m]] - (int32_t)d->h_voff[m] : -1;
  }
  return PJ_OK;
}

}  // extern "C"
