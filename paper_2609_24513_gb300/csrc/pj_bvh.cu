// Per-mesh BVH build on the GPU: an LBVH (Karras, "Maximizing Parallelism in
// the Construction of BVHs, Octrees, and k-d Trees", HPG 2012) over 30-bit
// Morton codes of triangle centroids normalised to the mesh box, exact
// integer-valued boxes by a bottom-up refit, then a top-down collapse of the
// binary tree into W-wide nodes whose leaves hold at most L triangles (a leaf
// is a subtree, so its triangles are contiguous in the sorted order).
//
// The paper builds one OptiX acceleration structure per dataset (Sec. 4.1);
// here each mesh gets its own tree because the refinement works per
// candidate pair.  Build time is not part of the query time (Sec. 4.2
// "Measurement").
#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "pj_internal.cuh"

namespace pj {

__device__ __forceinline__ int64_t mesh_of_b(const int64_t *off, int64_t M, int64_t e) {
  int64_t lo = 0, hi = M - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_morton(const float *xyz, const int32_t *tris, int64_t F,
                         const int64_t *toff, int64_t M, const float *aabb,
                         uint64_t *keys, int32_t *ids) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t m = mesh_of_b(toff, M, t);
    uint32_t q[3];
    for (int d = 0; d < 3; ++d) {
      double c = (double)xyz[3 * tris[3 * t] + d] + xyz[3 * tris[3 * t + 1] + d] +
                 xyz[3 * tris[3 * t + 2] + d];
      double lo = 3.0 * aabb[6 * m + d], ext = 3.0 * (aabb[6 * m + 3 + d] - aabb[6 * m + d]);
      double u = ext > 0 ? (c - lo) / ext : 0.0;
      int iq = (int)(u * 1024.0);
      q[d] = (uint32_t)min(max(iq, 0), 1023);
    }
    uint32_t code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    keys[t] = ((uint64_t)m << 30) | code;
    ids[t] = (int32_t)t;
  }
}

// binary radix tree node arrays (per dataset, internal nodes of mesh m at
// [ioff[m], ioff[m] + n_m - 1) with ioff[m] = toff[m] - m)
struct BinTree {
  int32_t *left, *right;   // >= 0 local internal index, < 0: leaf -(pos + 1)
  int32_t *first, *last;   // local sorted range
  int32_t *par_int;        // parent (global internal) of internal node, -1 root
  int32_t *par_leaf;       // parent (global internal) of sorted leaf, -1 none
  float *box;              // 6 per internal node
  float *leaf_box;         // 6 per sorted leaf
  int32_t *visits;
};

__device__ __forceinline__ int delta(const uint64_t *keys, int64_t base, int n,
                                     int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint32_t ki = (uint32_t)(keys[base + i] & 0x3FFFFFFFu);
  uint32_t kj = (uint32_t)(keys[base + j] & 0x3FFFFFFFu);
  if (ki != kj) return __clz(ki ^ kj);
  return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__global__ void k_karras(const uint64_t *keys, const int64_t *toff,
                         const int64_t *ioff, int64_t M, int64_t n_int,
                         BinTree T) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_int;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t m = mesh_of_b(ioff, M, g);
    int64_t base = toff[m];
    int n = (int)(toff[m + 1] - toff[m]);
    int i = (int)(g - ioff[m]);
    int d = (delta(keys, base, n, i, i + 1) - delta(keys, base, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, base, n, i, i - d);
    int lmax = 2;
    while (delta(keys, base, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (delta(keys, base, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, base, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
      int t = (l + div - 1) / div;
      if (delta(keys, base, n, i, i + (s + t) * d) > dnode) s += t;
      if (t <= 1) break;
    }
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int64_t ib = ioff[m];
    int32_t left, right;
    if (lo == gamma) {
      left = -(gamma + 1);
      T.par_leaf[base + gamma] = (int32_t)g;
    } else {
      left = gamma;
      T.par_int[ib + gamma] = (int32_t)g;
    }
    if (hi == gamma + 1) {
      right = -(gamma + 2);
      T.par_leaf[base + gamma + 1] = (int32_t)g;
    } else {
      right = gamma + 1;
      T.par_int[ib + gamma + 1] = (int32_t)g;
    }
    T.left[g] = left;
    T.right[g] = right;
    T.first[g] = lo;
    T.last[g] = hi;
    if (i == 0) T.par_int[g] = -1;
  }
}

__global__ void k_leaf_boxes(const float *xyz, const int32_t *tris,
                             const int32_t *sorted, int64_t F, float *leaf_box) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < F;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = sorted[s];
    for (int d = 0; d < 3; ++d) {
      float a = xyz[3 * tris[3 * t] + d], b = xyz[3 * tris[3 * t + 1] + d],
            c = xyz[3 * tris[3 * t + 2] + d];
      leaf_box[6 * s + d] = fminf(a, fminf(b, c));
      leaf_box[6 * s + 3 + d] = fmaxf(a, fmaxf(b, c));
    }
  }
}

// bottom-up union of child boxes; the second thread to reach a node computes
// it (no waiting: the first one stops)
__global__ void k_refit(const int64_t *toff, const int64_t *ioff, int64_t M,
                        int64_t F, BinTree T) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < F;
       s += (int64_t)gridDim.x * blockDim.x) {
    int32_t g = T.par_leaf[s];
    while (g >= 0) {
      __threadfence();
      if (atomicAdd(&T.visits[g], 1) == 0) break;
      __threadfence();
      int64_t m = mesh_of_b(ioff, M, g);
      int64_t base = toff[m], ib = ioff[m];
      float b[6];
      for (int c = 0; c < 2; ++c) {
        int32_t ch = c == 0 ? T.left[g] : T.right[g];
        const float *src = ch < 0 ? T.leaf_box + 6 * (base + (-ch - 1)) : T.box + 6 * (ib + ch);
        for (int d = 0; d < 6; ++d) {
          float v = __ldcg(src + d);
          if (c == 0) b[d] = v;
          else b[d] = d < 3 ? fminf(b[d], v) : fmaxf(b[d], v);
        }
      }
      for (int d = 0; d < 6; ++d) __stcg(T.box + 6 * (int64_t)g + d, b[d]);
      g = T.par_int[g];
    }
  }
}

__global__ void k_count_big(const int32_t *first, const int32_t *last, int64_t n,
                            int L, unsigned long long *cnt) {
  unsigned long long c = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x)
    c += (last[g] - first[g] + 1) > L;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

struct QEntry {
  int32_t bin;    // binary ref: >= 0 local internal, < 0 leaf -(pos + 1)
  int32_t mesh;
  int32_t wide;   // wide node id to fill
  int32_t depth;
};

__global__ void k_collapse(const QEntry *qin, const unsigned int *qin_n,
                           QEntry *qout, unsigned int *qout_n,
                           unsigned int *node_ctr, int64_t node_cap,
                           const int64_t *toff, const int64_t *ioff, BinTree T,
                           float *nodes, int W, int L, int *max_depth, int *err) {
  int n = (int)*qin_n;
  int sw = node_stride_words(W);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    QEntry q = qin[e];
    int64_t base = toff[q.mesh], ib = ioff[q.mesh];
    int32_t fr[8];
    int nf = 0;
    auto count_of = [&](int32_t r) -> int {
      return r < 0 ? 1 : (T.last[ib + r] - T.first[ib + r] + 1);
    };
    auto box_of = [&](int32_t r) -> const float * {
      return r < 0 ? T.leaf_box + 6 * (base + (-r - 1)) : T.box + 6 * (ib + r);
    };
    if (count_of(q.bin) <= L) {
      fr[nf++] = q.bin;
    } else {
      fr[nf++] = T.left[ib + q.bin];
      fr[nf++] = T.right[ib + q.bin];
      while (nf < W) {
        int best = -1;
        float best_a = -1.f;
        for (int k = 0; k < nf; ++k) {
          if (count_of(fr[k]) <= L) continue;
          const float *b = box_of(fr[k]);
          float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
          float a = dx * dy + dy * dz + dz * dx;
          if (a > best_a) { best_a = a; best = k; }
        }
        if (best < 0) break;
        int32_t r = fr[best];
        fr[best] = T.left[ib + r];
        fr[nf++] = T.right[ib + r];
      }
    }
    float *node = nodes + (int64_t)q.wide * sw;
    {
      const float *b = box_of(q.bin);
      for (int d = 0; d < 6; ++d) node[d] = b[d];
      node[6] = 0.f;
      node[7] = 0.f;
    }
    for (int k = 0; k < W; ++k) {
      float *slot = node + 8 * (k + 1);
      uint32_t *child = reinterpret_cast<uint32_t *>(slot + 6);
      slot[7] = 0.f;
      if (k >= nf) {
        for (int d = 0; d < 3; ++d) {
          slot[d] = 3e38f;
          slot[3 + d] = -3e38f;
        }
        *child = kEmpty;
        continue;
      }
      int32_t r = fr[k];
      const float *b = box_of(r);
      for (int d = 0; d < 6; ++d) slot[d] = b[d];
      int c = count_of(r);
      if (c <= L) {
        int first = r < 0 ? (-r - 1) : T.first[ib + r];
        *child = kLeafBit | ((uint32_t)first << 3) | (uint32_t)(c - 1);
      } else {
        unsigned int id = atomicAdd(node_ctr, 1u);
        if ((int64_t)id >= node_cap) {
          atomicExch(err, 1);
          *child = kEmpty;
          continue;
        }
        *child = id;
        unsigned int qs = atomicAdd(qout_n, 1u);
        QEntry o;
        o.bin = r;
        o.mesh = q.mesh;
        o.wide = (int32_t)id;
        o.depth = q.depth + 1;
        qout[qs] = o;
      }
    }
    atomicMax(max_depth, q.depth);
  }
}

__global__ void k_trirec(const float *xyz, const int32_t *tris, const int32_t *sorted,
                         const uint8_t *emask, const int64_t *toff, int64_t M,
                         int64_t F, float4 *rec) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < F;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = sorted[s];
    int64_t m = mesh_of_b(toff, M, t);
    const float *a = xyz + 3 * tris[3 * t], *b = xyz + 3 * tris[3 * t + 1],
                *c = xyz + 3 * tris[3 * t + 2];
    rec[3 * s] = make_float4(a[0], a[1], a[2], b[0]);
    rec[3 * s + 1] = make_float4(b[1], b[2], c[0], c[1]);
    rec[3 * s + 2] = make_float4(c[2], __int_as_float((int)emask[t]),
                                 __int_as_float((int)(t - toff[m])), 0.f);
  }
}

__global__ void k_iota_roots(int32_t *roots, int64_t M) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x)
    roots[m] = (int32_t)m;
}

__global__ void k_init_queue(QEntry *q, int64_t M, const int64_t *toff) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    QEntry e;
    e.mesh = (int32_t)m;
    e.wide = (int32_t)m;
    e.depth = 1;
    e.bin = (toff[m + 1] - toff[m] > 1) ? 0 : -1;  // internal 0 is the root
    q[m] = e;
  }
}

struct TmpB {
  std::vector<void *> p;
  ~TmpB() {
    for (void *q : p) cudaFree(q);
  }
  template <typename T>
  cudaError_t get(T **out, int64_t n) {
    cudaError_t e = cudaMalloc((void **)out, sizeof(T) * (size_t)(n > 0 ? n : 1));
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
};

pj_status build_bvh(Ctx *ctx, Dataset *ds, int W, int L, cudaStream_t s) {
  const int64_t M = ds->M, F = ds->F;
  const int64_t n_int = F - M;
  auto nb = [&](int64_t n) {
    int64_t b = (n + 255) / 256, cap = (int64_t)ctx->num_sms * 32;
    return (int)std::max<int64_t>(1, std::min(b, cap));
  };
  TmpB tmp;
  Bvh bvh;
  bvh.W = W;
  bvh.L = L;
  // 1. Morton keys, sorted per mesh
  uint64_t *k0, *k1;
  int32_t *i0;
  PJ_CK(tmp.get(&k0, F));
  PJ_CK(tmp.get(&k1, F));
  PJ_CK(tmp.get(&i0, F));
  PJ_CK(cudaMalloc(&bvh.d_tri_order, sizeof(int32_t) * (size_t)std::max<int64_t>(F, 1)));
  struct Guard {
    Bvh *b;
    bool ok = false;
    ~Guard() {
      if (!ok) {
        cudaFree(b->d_nodes);
        cudaFree(b->d_roots);
        cudaFree(b->d_tri_order);
        cudaFree(b->d_trirec);
      }
    }
  } guard{&bvh};
  k_morton<<<nb(F), 256, 0, s>>>(ds->d_xyz, ds->d_tris, F, ds->d_toff, M, ds->d_aabb, k0, i0);
  int mbits = 1;
  while ((1ll << mbits) <= M) ++mbits;
  size_t tb = 0;
  PJ_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, k0, k1, i0, bvh.d_tri_order, (int)F, 0,
                                        30 + mbits, s));
  char *tstore;
  PJ_CK(tmp.get(&tstore, (int64_t)tb));
  PJ_CK(cub::DeviceRadixSort::SortPairs(tstore, tb, k0, k1, i0, bvh.d_tri_order, (int)F, 0,
                                        30 + mbits, s));
  // 2. binary radix trees
  std::vector<int64_t> h_ioff(M + 1);
  for (int64_t m = 0; m <= M; ++m) h_ioff[m] = ds->h_toff[m] - m;
  int64_t *d_ioff;
  PJ_CK(tmp.get(&d_ioff, M + 1));
  PJ_CK(cudaMemcpyAsync(d_ioff, h_ioff.data(), sizeof(int64_t) * (M + 1),
                        cudaMemcpyHostToDevice, s));
  BinTree T;
  PJ_CK(tmp.get(&T.left, n_int));
  PJ_CK(tmp.get(&T.right, n_int));
  PJ_CK(tmp.get(&T.first, n_int));
  PJ_CK(tmp.get(&T.last, n_int));
  PJ_CK(tmp.get(&T.par_int, n_int));
  PJ_CK(tmp.get(&T.par_leaf, F));
  PJ_CK(tmp.get(&T.box, 6 * n_int));
  PJ_CK(tmp.get(&T.leaf_box, 6 * F));
  PJ_CK(tmp.get(&T.visits, n_int));
  PJ_CK(cudaMemsetAsync(T.par_leaf, 0xff, sizeof(int32_t) * F, s));
  PJ_CK(cudaMemsetAsync(T.visits, 0, sizeof(int32_t) * std::max<int64_t>(n_int, 1), s));
  if (n_int > 0)
    k_karras<<<nb(n_int), 256, 0, s>>>(k1, ds->d_toff, d_ioff, M, n_int, T);
  k_leaf_boxes<<<nb(F), 256, 0, s>>>(ds->d_xyz, ds->d_tris, bvh.d_tri_order, F, T.leaf_box);
  // 3. exact boxes bottom-up
  if (n_int > 0) k_refit<<<nb(F), 256, 0, s>>>(ds->d_toff, d_ioff, M, F, T);
  PJ_CK(cudaGetLastError());
  // 4. collapse to W-wide nodes
  unsigned long long *d_big;
  PJ_CK(tmp.get(&d_big, 1));
  PJ_CK(cudaMemsetAsync(d_big, 0, 8, s));
  if (n_int > 0) k_count_big<<<nb(n_int), 256, 0, s>>>(T.first, T.last, n_int, L, d_big);
  unsigned long long big = 0;
  PJ_CK(cudaMemcpyAsync(&big, d_big, 8, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  const int64_t node_cap = (int64_t)big + M;
  const int sw = node_stride_words(W);
  float *nodes_tmp;
  PJ_CK(tmp.get(&nodes_tmp, node_cap * sw));
  QEntry *qa, *qb;
  PJ_CK(tmp.get(&qa, node_cap));
  PJ_CK(tmp.get(&qb, node_cap));
  unsigned int *ctr;  // [0] qa count, [1] qb count, [2] node counter
  int *dflag;         // [0] max depth, [1] error
  PJ_CK(tmp.get(&ctr, 4));
  PJ_CK(tmp.get(&dflag, 2));
  unsigned int init[4] = {(unsigned int)M, 0u, (unsigned int)M, 0u};
  PJ_CK(cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, s));
  PJ_CK(cudaMemsetAsync(dflag, 0, 8, s));
  k_init_queue<<<nb(M), 256, 0, s>>>(qa, M, ds->d_toff);
  int64_t pending = M;
  int level = 0;
  unsigned int *qin_n = ctr, *qout_n = ctr + 1;
  while (pending > 0) {
    PJ_CK(cudaMemsetAsync(qout_n, 0, 4, s));
    k_collapse<<<nb(pending), 256, 0, s>>>(qa, qin_n, qb, qout_n, ctr + 2, node_cap,
                                          ds->d_toff, d_ioff, T, nodes_tmp, W, L, dflag,
                                          dflag + 1);
    PJ_CK(cudaGetLastError());
    unsigned int nxt = 0;
    PJ_CK(cudaMemcpyAsync(&nxt, qout_n, 4, cudaMemcpyDeviceToHost, s));
    PJ_CK(cudaStreamSynchronize(s));
    pending = nxt;
    std::swap(qa, qb);
    std::swap(qin_n, qout_n);
    if (++level > 4096) return fail(ctx, PJ_ERR_INTERNAL, "BVH collapse did not terminate");
  }
  unsigned int n_nodes = 0;
  int hflag[2];
  PJ_CK(cudaMemcpyAsync(&n_nodes, ctr + 2, 4, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaMemcpyAsync(hflag, dflag, 8, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  if (hflag[1]) return fail(ctx, PJ_ERR_INTERNAL, "BVH node capacity exceeded");
  if ((int64_t)n_nodes * W >= (1ll << 30))
    return fail(ctx, PJ_ERR_INVALID_ARG, "dataset too large for 30-bit BVH slot ids");
  bvh.n_nodes = n_nodes;
  bvh.max_depth = hflag[0];
  PJ_CK(cudaMalloc(&bvh.d_nodes, sizeof(float) * (size_t)n_nodes * sw));
  PJ_CK(cudaMemcpyAsync(bvh.d_nodes, nodes_tmp, sizeof(float) * (size_t)n_nodes * sw,
                        cudaMemcpyDeviceToDevice, s));
  PJ_CK(cudaMalloc(&bvh.d_roots, sizeof(int32_t) * (size_t)M));
  k_iota_roots<<<nb(M), 256, 0, s>>>(bvh.d_roots, M);
  // 5. triangle records in leaf order
  PJ_CK(cudaMalloc(&bvh.d_trirec, sizeof(float4) * 3 * (size_t)std::max<int64_t>(F, 1)));
  k_trirec<<<nb(F), 256, 0, s>>>(ds->d_xyz, ds->d_tris, bvh.d_tri_order, ds->d_emask,
                                 ds->d_toff, M, F, bvh.d_trirec);
  PJ_CK(cudaGetLastError());
  PJ_CK(cudaStreamSynchronize(s));
  bvh.bytes = (int64_t)n_nodes * sw * 4 + 4 * M + 4 * F + 48 * F;
  guard.ok = true;
  ds->bvhs[{W, L}] = bvh;
  return PJ_OK;
}

}  // namespace pj
