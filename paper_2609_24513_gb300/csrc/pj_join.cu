// The join's hot path: bounding-box filter join, pair refinement (crossing
// by edge piercing + containment by +z parity), result compaction.
//
// Paper mapping:
//   - Alg. 1 (edge ray tracing) run in both directions (Sec. 3.2) becomes,
//     per candidate pair, a simultaneous descent of the two meshes' BVHs: a
//     node of the source mesh is a packet of edge segments bounded by the
//     node's box, so a (source node, target node) step prunes every edge of
//     the packet against the target subtree at once.  At a (leaf, leaf) step
//     each owned edge of one leaf is tested against the other leaf's box (a
//     slab test, or in the streaming kernel an overlap test of the edge's
//     box) and then exactly against its triangles, in both directions.  The
//     first crossing ends the pair.
//   - Alg. 2's parity test (Sec. 3.3) runs in both directions (Sec. 3.4: not
//     filtered by crossings, but a crossing already decides the
//     intersection predicate).  The streaming (default) and breadth-first
//     front ends run it first, so that a contained pair skips the traversal;
//     the per-warp passes run it for the pairs their traversal left without a
//     crossing.
//   - Result materialisation (Sec. 3.5) is one flag per candidate followed
//     by a prefix-sum compaction, so nothing needs deduplication.
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>

#include "pj_geom.cuh"
#include "pj_internal.cuh"

namespace pj {

constexpr unsigned FULL = 0xffffffffu;

// Programmatic dependent launch (sm_90 and later): a kernel launched with
// launch_pdl may be scheduled while the previous kernel on the stream is
// still draining.  Every kernel of the join calls pdl_wait() before its
// first access to memory that an earlier kernel wrote (it returns once that
// kernel has completed and its writes are visible; without the launch
// attribute it returns at once), then pdl_trigger() to let the next kernel
// be scheduled as this one's blocks retire.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 (three-phase: block scan, scan of block sums, add)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    int64_t u = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// block-wide exclusive scan of one value per thread (blockDim.x == SCAN_T)
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
  __shared__ int64_t wsum[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = warp_incl_scan(v, lane);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    s = warp_incl_scan(s, lane);
    wsum[lane] = s;
  }
  __syncthreads();
  int64_t base = w > 0 ? wsum[w - 1] : 0;
  if (total) *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + inc - v;
}

__global__ void k_scan_blocks(const int64_t *in, int64_t *out, int64_t n, int64_t *bsum) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  int64_t tot;
  int64_t e = block_excl_scan(v, &tot);
  if (i < n) out[i] = e;
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *boff) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

__global__ void k_scan_total(const int64_t *in, const int64_t *out, int64_t n, int64_t *total) {
  pdl_wait();
  pdl_trigger();
  *total = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

// One block scans up to SCAN_T * SCAN_SMALL values: each thread sums a run
// of consecutive values, the block scans the run sums, each thread writes its
// run's exclusive prefixes; thread 0 also writes the total.
constexpr int SCAN_SMALL = 32;

__global__ void __launch_bounds__(SCAN_T) k_scan_small(const int64_t *in, int64_t *out, int64_t n,
                                                       int64_t *total) {
  pdl_wait();
  pdl_trigger();
  const int64_t per = (n + SCAN_T - 1) / SCAN_T;
  const int64_t b = threadIdx.x * per, e = min(n, b + per);
  int64_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += in[i];
  int64_t tot;
  int64_t run = block_excl_scan(sum, &tot);
  for (int64_t i = b; i < e; ++i) {
    const int64_t v = in[i];
    out[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) *total = tot;
}

pj_status scan_i64(Ctx *ctx, const int64_t *d_in, int64_t *d_out, int64_t n,
                   int64_t *d_total, cudaStream_t s) {
  if (n <= (int64_t)SCAN_T * SCAN_SMALL) {
    cudaError_t e = launch_pdl(k_scan_small, 1, SCAN_T, 0, s, d_in, d_out, n, d_total);
    ++ctx->launches;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scan");
    return PJ_OK;
  }
  // level buffers: block sums and their scans
  std::vector<int64_t> sizes;
  int64_t m = n;
  while (m > SCAN_T) {
    m = (m + SCAN_T - 1) / SCAN_T;
    sizes.push_back(m);
  }
  int64_t need = 0;
  for (int64_t z : sizes) need += 2 * z;
  pj_status st;
  int64_t *buf = (int64_t *)ws_get(ctx, "scan", sizeof(int64_t) * (size_t)(need + 2), &st);
  if (!buf) return st;
  // up-sweep
  const int64_t *cur_in = d_in;
  int64_t *cur_out = d_out;
  int64_t cur_n = n;
  std::vector<int64_t *> lv_in, lv_out;
  int64_t off = 0;
  for (size_t l = 0; l <= sizes.size(); ++l) {
    int nb = (int)((cur_n + SCAN_T - 1) / SCAN_T);
    if (nb < 1) nb = 1;
    int64_t *bsum = buf + need;  // scratch for the final single block
    if (l < sizes.size()) bsum = buf + off;
    k_scan_blocks<<<nb, SCAN_T, 0, s>>>(cur_in, cur_out, cur_n, bsum);
    ++ctx->launches;
    if (l == sizes.size()) break;
    int64_t *bscan = buf + off + sizes[l];
    lv_in.push_back(bsum);
    lv_out.push_back(bscan);
    cur_in = bsum;
    cur_out = bscan;
    cur_n = sizes[l];
    off += 2 * sizes[l];
  }
  // down-sweep: add scanned block sums
  for (int l = (int)sizes.size() - 1; l >= 0; --l) {
    int64_t *target = l == 0 ? d_out : lv_out[l - 1];
    int64_t tn = l == 0 ? n : sizes[l - 1];
    int nb = (int)((tn + SCAN_T - 1) / SCAN_T);
    k_scan_add<<<nb, SCAN_T, 0, s>>>(target, tn, lv_out[l]);
    ++ctx->launches;
  }
  k_scan_total<<<1, 1, 0, s>>>(d_in, d_out, n, d_total);
  ++ctx->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan");
  return PJ_OK;
}

// ---------------------------------------------------------------------------
// Bounding-box filter join (the paper's filter step, Sec. 1 / Sec. 2):
// candidates (i, j) whose closed mesh boxes meet, in lexicographic order.
// ---------------------------------------------------------------------------
constexpr int MBB_T = 256;

// One warp per A mesh; lanes sweep the B boxes 32 at a time.  The count pass
// and the emit pass make the same tests, and the emit pass writes each warp's
// hits in j order (ballot prefix), so candidates come out sorted by (i, j).
// B boxes staged in shared memory per tile
constexpr int MBB_TILE = 1024;
// single-pass box join tiles: MBB_RPW A meshes per warp, MBB_TA per tile (a
// tile is one block's unit of look-back; fewer, larger tiles fit the
// resident grid in one round)
constexpr int MBB_RPW = 2;
constexpr int MBB_TA = (MBB_T / 32) * MBB_RPW;

template <bool EMIT>
__global__ void __launch_bounds__(MBB_T) k_mbb(const float *aabbA, int64_t MA,
                                              const float *aabbB, int64_t MB, int self_join,
                                              int64_t *counts, const int64_t *offsets,
                                              int32_t *cand) {
  pdl_wait();
  pdl_trigger();
  // a tile of B boxes is copied to shared memory once per block (coalesced)
  // and tested by every warp's A mesh from there
  __shared__ float sb[MBB_TILE * 6];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  constexpr int WPB = MBB_T / 32;
  for (int64_t i0 = blockIdx.x * (int64_t)WPB; i0 < MA; i0 += (int64_t)gridDim.x * WPB) {
    const int64_t i = i0 + wib;
    const bool has = i < MA;
    float ax0 = 0.f, ay0 = 0.f, az0 = 0.f, ax1 = -1.f, ay1 = -1.f, az1 = -1.f;
    if (has) {
      const float *a = aabbA + 6 * i;
      ax0 = a[0], ay0 = a[1], az0 = a[2], ax1 = a[3], ay1 = a[4], az1 = a[5];
    }
    int64_t cnt = 0, pos = (EMIT && has) ? offsets[i] : 0;
    // in a self join only j > i counts: tiles below the block's first i are skipped
    const int64_t jstart = self_join ? ((i0 + 1) / MBB_TILE) * MBB_TILE : 0;
    for (int64_t t0 = jstart; t0 < MB; t0 += MBB_TILE) {
      const int n = MB - t0 < MBB_TILE ? (int)(MB - t0) : MBB_TILE;
      __syncthreads();  // the previous tile is no longer read
      for (int k = threadIdx.x; k < n * 6; k += MBB_T) sb[k] = aabbB[6 * t0 + k];
      __syncthreads();
      if (!has) continue;
      for (int j0 = 0; j0 < n; j0 += 32) {
        const int jj = j0 + lane;
        const int64_t j = t0 + jj;
        bool ov = false;
        if (jj < n && (!self_join || j > i)) {
          const float *bb = sb + 6 * jj;
          ov = ax0 <= bb[3] && bb[0] <= ax1 && ay0 <= bb[4] && bb[1] <= ay1 && az0 <= bb[5] &&
               bb[2] <= az1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ov);
        if (EMIT && ov) {
          const int64_t p = pos + __popc(m & ((1u << lane) - 1u));
          cand[2 * p] = (int32_t)i;
          cand[2 * p + 1] = (int32_t)j;
        }
        if (EMIT) pos += __popc(m);
        else cnt += __popc(m);
      }
    }
    if (!EMIT && has && lane == 0) counts[i] = cnt;
  }
}

// ---------------------------------------------------------------------------
// Candidate validation (explicit candidates): ids in range, translated
// meshes on the grid.
// ---------------------------------------------------------------------------
__global__ void k_check_cand(const int32_t *cand, const int32_t *off, int64_t n,
                             int64_t MA, int64_t MB, const float *aabbB, int *err) {
  pdl_wait();
  pdl_trigger();
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    int a = cand[2 * c], b = cand[2 * c + 1];
    if (a < 0 || a >= MA || b < 0 || b >= MB) {
      atomicCAS(err + 1, 0, 1);
      continue;
    }
    if (off) {
      for (int d = 0; d < 3; ++d) {
        float lo = aabbB[6 * (int64_t)b + d] + (float)off[3 * c + d];
        float hi = aabbB[6 * (int64_t)b + 3 + d] + (float)off[3 * c + d];
        if (lo < 0.f || hi > 262143.f) atomicCAS(err + 2, 0, 1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Refinement kernel
// ---------------------------------------------------------------------------
struct Side {
  const float *nodes;
  const int32_t *roots;
  const float4 *trirec;
  const int64_t *toff;
  const int64_t *voff;
  const float *aabb;
  const float *xyz;
  const int32_t *lexorder;
  const float4 *mrec;        // per-mesh record: box, first lexicographic vertex, offsets
};

struct RefineArgs {
  Side A, B;
  const int32_t *cand;
  const int32_t *cand_off;
  const int64_t *n_cand;     // device count
  uint8_t *flags;
  unsigned long long *work;  // work counter
  unsigned long long *counters;
  int *err;
  int stack_cap;             // task entries per warp
  int max_pop;               // tasks popped per traversal step (1 = plain DFS)
  int warps_per_pair;        // 1, 2 or 4
  int64_t MA, MB;            // mesh counts (candidate ids are checked)
  long long single;          // >= 0: process only this candidate
  unsigned int *cycles;      // per-candidate SM cycles, or null
  // pass 1 spill queue and budget; later passes read q_in
  uint4 *q_out;
  unsigned int *q_out_n;
  unsigned int q_cap;
  long long budget;          // SM cycles a warp spends on a pair or task before spilling
  const uint4 *q_in;
  const unsigned int *q_in_n;
  unsigned int *q_in_pos;
  unsigned int q_in_cap;
  // parity rays handed over by the per-thread parity kernel (pass 1 only)
  const uint4 *q_par;
  const unsigned int *q_par_n;
  unsigned int *q_par_pos;
  unsigned int q_par_cap;
  // join predicate (PJ_PRED_*); with contains / within the containment
  // result goes to pflags and flags keeps the crossing result
  int predicate;
  uint8_t *pflags;
};

struct Cnt {
  unsigned long long v[C_WARP_NUM];
};

// Work handed from one refinement pass to the next: when a pair exceeds its
// step budget its remaining traversal tasks go to a queue of
// (candidate, itemA, itemB) entries that the next pass spreads over warps.
struct Spill {
  uint4 *q;                  // queue to append to (null: never spill)
  unsigned int *q_n;         // its fill counter
  unsigned int q_cap;
  long long budget;          // SM cycles before spilling (0: unbounded)
  const volatile uint8_t *flag;  // this pair's result, polled for early exit
  uint32_t cand;
};

// Traversal items (32-bit):
//   internal node: node index (bits 0-29), bit 30 = expand this side next
//   leaf:          bit 31 | slot id = node * W + child (bits 0-29)
constexpr uint32_t kExpand = 0x40000000u;
constexpr uint32_t kIdx = 0x3FFFFFFFu;

template <int W>
struct Cfg {
  static constexpr int SW = 8 * (W + 1);  // node stride in words
  static constexpr int LQ = 128;          // leaf-pair queue entries
  static constexpr int TQ = 32;           // tasks popped per step
  // per-warp shared memory besides the task stack
  static constexpr int extra_bytes = LQ * 8 /*queue*/ + LQ * 8 /*descriptors*/ +
                                     (LQ + 1) * 4 /*unit prefix*/ + TQ * 8 /*popped*/ +
                                     (TQ + 1) * 4 /*test prefix*/;
};

template <int W>
__host__ __device__ constexpr int warp_smem_bytes(int stack_cap) {
  return ((stack_cap * 8 + Cfg<W>::extra_bytes) + 15) / 16 * 16;
}

struct WarpMem {
  uint2 *stk;
  uint2 *lq;
  uint2 *ldesc;
  uint2 *tq;
  int *lpre;
  int *tpre;
};

template <int W>
__device__ __forceinline__ WarpMem carve(unsigned char *base, int stack_cap) {
  WarpMem m;
  m.stk = reinterpret_cast<uint2 *>(base);
  m.lq = m.stk + stack_cap;
  m.ldesc = m.lq + Cfg<W>::LQ;
  m.tq = m.ldesc + Cfg<W>::LQ;
  m.lpre = reinterpret_cast<int *>(m.tq + Cfg<W>::TQ);
  m.tpre = m.lpre + Cfg<W>::LQ + 1;
  return m;
}



// slot k of a node (k = -1: the node's own box): box and child word
template <int W>
__device__ __forceinline__ void load_slot(const float *nodes, uint32_t node, int k, F3 off,
                                          Box &b, uint32_t &child) {
  const float4 *p = reinterpret_cast<const float4 *>(nodes + (int64_t)node * Cfg<W>::SW +
                                                     8 * (k + 1));
  float4 u = __ldg(p), v = __ldg(p + 1);
  b.lo = add(mkf3(u.x, u.y, u.z), off);
  b.hi = add(mkf3(u.w, v.x, v.y), off);
  child = __float_as_uint(v.z);
}

// Open (strict) overlap on every axis.  Exact for the crossing traversal:
// if on some axis the boxes of a segment (or of a subtree's segments) and of
// a triangle only touch at a value c, a strict crossing point would have
// coordinate c, an extreme of both the open segment and the open triangle,
// which forces both into the plane at c -- a coplanar configuration the
// strict test rejects.  So boxes that only touch hold no crossing, and
// pruning them loses nothing (pinned on the CPU against the oracle's strict
// predicate on configurations full of exact contacts).
__device__ __forceinline__ bool overlap_open(const Box &a, const Box &b) {
  return a.lo.x < b.hi.x && b.lo.x < a.hi.x && a.lo.y < b.hi.y && b.lo.y < a.hi.y &&
         a.lo.z < b.hi.z && b.lo.z < a.hi.z;
}

__device__ __forceinline__ bool overlap(const Box &a, const Box &b) {
  return a.lo.x <= b.hi.x && b.lo.x <= a.hi.x && a.lo.y <= b.hi.y && b.lo.y <= a.hi.y &&
         a.lo.z <= b.hi.z && b.lo.z <= a.hi.z;
}

__device__ __forceinline__ float extent(const Box &b) {
  return fmaxf(fmaxf(b.hi.x - b.lo.x, b.hi.y - b.lo.y), b.hi.z - b.lo.z);
}

// Build a task from two items (flags stripped) and their boxes: a leaf never
// expands; of two internal nodes, the one more than twice as large expands
// alone, otherwise both do (simultaneous descent).
__device__ __forceinline__ uint2 make_task(uint32_t a, const Box &ba, uint32_t b,
                                          const Box &bb) {
  const bool la = a & kLeafBit, lb = b & kLeafBit;
  const float ea = extent(ba), eb = extent(bb);
  const bool xa = !la && (lb || !(eb > 2.f * ea));
  const bool xb = !lb && (la || !(ea > 2.f * eb));
  return make_uint2(a | (xa ? kExpand : 0u), b | (xb ? kExpand : 0u));
}

// Algorithmic bytes of one (node, node) step: the W child slots of each side
// that expands, the one box slot of each side that does not (32 B a slot).
template <int W>
__device__ __forceinline__ unsigned node_pair_bytes(bool xa, bool xb) {
  return (unsigned)((xa ? W : 1) + (xb ? W : 1)) * 32u;
}

__device__ __forceinline__ int task_tests(uint2 t, int W) {
  return ((t.x & kExpand) ? W : 1) * ((t.y & kExpand) ? W : 1);
}

__device__ __forceinline__ void load_tri(const float4 *rec, int64_t s, F3 off, F3 &a,
                                         F3 &b, F3 &c, int &own) {
  float4 r0 = __ldg(rec + 3 * s), r1 = __ldg(rec + 3 * s + 1), r2 = __ldg(rec + 3 * s + 2);
  a = add(mkf3(r0.x, r0.y, r0.z), off);
  b = add(mkf3(r0.w, r1.x, r1.y), off);
  c = add(mkf3(r1.z, r1.w, r2.x), off);
  own = __float_as_int(r2.y);
}

// element t of a small register array without dynamic indexing (which would
// move the array to local memory)
template <int N>
__device__ __forceinline__ F3 sel_f3(const F3 (&a)[N], int t) {
  F3 r = a[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (t == k) r = a[k];
  return r;
}
template <int N>
__device__ __forceinline__ uint32_t sel_u32(const uint32_t (&a)[N], int t) {
  uint32_t r = a[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (t == k) r = a[k];
  return r;
}

// warp-wide inclusive scan of small ints
__device__ __forceinline__ int warp_scan_incl(int v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Leaf-pair work: one unit = (leaf pair, direction, source triangle).
template <int W, bool EXACT>
__device__ bool leaf_units(const Side &A, const Side &B, int64_t tA, int64_t tB, F3 off,
                           WarpMem &sm, int nlq, int lane, Cnt &cnt) {
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  // descriptors (child words of the two leaf slots) and unit counts
  int run = 0;
  if (lane == 0) sm.lpre[0] = 0;
  for (int e0 = 0; e0 < nlq; e0 += 32) {
    int e = e0 + lane;
    int u = 0;
    if (e < nlq) {
      uint2 q = sm.lq[e];
      uint32_t sa = q.x & kIdx, sb = q.y & kIdx;
      const float *pa = A.nodes + (int64_t)(sa / W) * Cfg<W>::SW + 8 * (sa % W + 1);
      const float *pb = B.nodes + (int64_t)(sb / W) * Cfg<W>::SW + 8 * (sb % W + 1);
      uint32_t da = __float_as_uint(__ldg(pa + 6)), db = __float_as_uint(__ldg(pb + 6));
      sm.ldesc[e] = make_uint2(da, db);
      u = (int)(da & 7u) + 1 + (int)(db & 7u) + 1;
    }
    int inc = warp_scan_incl(u, lane);
    if (e < nlq) sm.lpre[e + 1] = run + inc;
    run += __shfl_sync(FULL, inc, 31);
  }
  __syncwarp();
  const int U = run;
  if (lane == 0) {
    cnt.v[C_LEAF_PAIRS] += nlq;
    cnt.v[C_BYTES] += 8ull * nlq;
  }
  bool hit = false;
  for (int base = 0; base < U; base += 32) {
    int u = base + lane;
    if (u < U && !hit) {
      int lo = 0, hi = nlq - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sm.lpre[mid] <= u) lo = mid; else hi = mid - 1;
      }
      const int e = lo;
      const int k = u - sm.lpre[e];
      const uint2 q = sm.lq[e];
      const uint2 d = sm.ldesc[e];
      const int nA = (int)(d.x & 7u) + 1;
      const bool dirA = k < nA;  // source triangle from A, target leaf in B
      const Side &S = dirA ? A : B;
      const Side &T = dirA ? B : A;
      const uint32_t sdesc = dirA ? d.x : d.y, tdesc = dirA ? d.y : d.x;
      const uint32_t tslot = (dirA ? q.y : q.x) & kIdx;
      const int64_t sbase = dirA ? tA : tB, tbase = dirA ? tB : tA;
      const F3 soff = dirA ? zero : off;
      const F3 toff = dirA ? off : zero;
      const int si = dirA ? k : k - nA;
      const int64_t s_rec = sbase + ((sdesc >> 3) & 0x0FFFFFFFu) + si;
      const int64_t t_first = tbase + ((tdesc >> 3) & 0x0FFFFFFFu);
      const int t_n = (int)(tdesc & 7u) + 1;
      Box tb;
      uint32_t tdummy;
      load_slot<W>(T.nodes, tslot / W, (int)(tslot % W), toff, tb, tdummy);
      F3 v[3];
      int own;
      load_tri(S.trirec, s_rec, soff, v[0], v[1], v[2], own);
      cnt.v[C_BYTES] += 48 + 32;
      for (int ek = 0; ek < 3 && !hit; ++ek) {
        if (!((own >> ek) & 1)) continue;
        F3 p = v[ek], qv = v[ek == 2 ? 0 : ek + 1];
        Seg sg = make_seg(p, qv);
        cnt.v[C_SLAB_TESTS] += 1;
        if (!slab_hit(sg, tb.lo, tb.hi)) continue;
        F3 elo = mkf3(fminf(p.x, qv.x), fminf(p.y, qv.y), fminf(p.z, qv.z));
        F3 ehi = mkf3(fmaxf(p.x, qv.x), fmaxf(p.y, qv.y), fmaxf(p.z, qv.z));
        for (int t = 0; t < t_n; ++t) {
          F3 a, b, c;
          int town;
          load_tri(T.trirec, t_first + t, toff, a, b, c, town);
          cnt.v[C_BYTES] += 48;
          float lx = fminf(a.x, fminf(b.x, c.x)), hx = fmaxf(a.x, fmaxf(b.x, c.x));
          float ly = fminf(a.y, fminf(b.y, c.y)), hy = fmaxf(a.y, fmaxf(b.y, c.y));
          float lz = fminf(a.z, fminf(b.z, c.z)), hz = fmaxf(a.z, fmaxf(b.z, c.z));
          if (lx > ehi.x || elo.x > hx || ly > ehi.y || elo.y > hy || lz > ehi.z || elo.z > hz)
            continue;
          cnt.v[C_SEGTRI] += 1;
          bool r;
          if (EXACT) {
            r = segtri_exact_staged(p, qv, a, b, c);
          } else {
            bool ex = false;
            r = segtri_filtered(p, qv, a, b, c, &ex);
            cnt.v[C_FALLBACK] += ex ? 1 : 0;
          }
          if (r) {
            hit = true;
            break;
          }
        }
      }
    }
    if (__any_sync(FULL, hit)) return true;
  }
  return false;
}

// Crossing test of one pair by descending both BVHs (larger node first,
// simultaneously when comparable).  Each step pops up to 32 tasks and spreads
// their child-box tests over the lanes.  Returns 1 on a crossing, 0 if none,
// -1 if the task stack would overflow.
template <int W, bool EXACT>
__device__ int pair_cross(const Side &A, const Side &B, int ia, int ib, F3 off,
                          WarpMem &sm, int lane, int stack_cap, int max_pop, Cnt &cnt,
                          volatile int *group_hit, int rank, int nrank, const Spill &spill,
                          bool from_root, uint2 start) {
  constexpr int LQ = Cfg<W>::LQ;
  const int64_t tA = A.toff[ia], tB = B.toff[ib];
  const unsigned lt = (1u << lane) - 1u;
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  if (from_root) {
    const uint32_t ra = (uint32_t)A.roots[ia], rb = (uint32_t)B.roots[ib];
    Box ba, bb;
    ba.lo = ld3(A.aabb + 6 * (int64_t)ia);
    ba.hi = ld3(A.aabb + 6 * (int64_t)ia + 3);
    bb.lo = add(ld3(B.aabb + 6 * (int64_t)ib), off);
    bb.hi = add(ld3(B.aabb + 6 * (int64_t)ib + 3), off);
    if (lane == 0) sm.stk[0] = make_task(ra, ba, rb, bb);
  } else if (lane == 0) {
    sm.stk[0] = start;
  }
  int sp = 1, nlq = 0;
  __syncwarp();
  bool split_done = nrank <= 1;
  unsigned iters = 0;
  const long long t_begin = clock64();
  while (sp > 0 || nlq > 0) {
    if (++iters > (1u << 26)) return -1;  // defensive bound: a tree walk is finite
    if (group_hit) {
      int gh = __shfl_sync(FULL, *group_hit, 0);
      if (gh) return 1;
    }
    if (spill.flag && (iters & 15u) == 0) {
      // another warp may already have found a crossing of this pair
      int f = lane == 0 ? (int)*spill.flag : 0;
      if (__shfl_sync(FULL, f, 0)) return 1;
    }
    if (spill.budget > 0 && sp > 0 && clock64() - t_begin > spill.budget) {
      // over budget: finish the queued leaf pairs, then hand the remaining
      // tasks to the next pass, where other warps take them
      if (nlq > 0) {
        bool h = leaf_units<W, EXACT>(A, B, tA, tB, off, sm, nlq, lane, cnt);
        nlq = 0;
        __syncwarp();
        if (h) return 1;
      }
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(spill.q_n, (unsigned)sp);
      base = __shfl_sync(FULL, base, 0);
      if ((uint64_t)base + (uint64_t)sp > (uint64_t)spill.q_cap) return -3;
      for (int e = lane; e < sp; e += 32) {
        uint2 t = sm.stk[e];
        spill.q[base + e] = make_uint4(spill.cand, t.x, t.y, 0u);
      }
      if (lane == 0) cnt.v[C_SPILLED] += sp;
      return -2;
    }
    if (sp > 0 && nlq + 64 <= LQ) {
      // pop up to max_pop tasks whose tests add up to at most 32 (at least one)
      const int e = sp - 1 - lane;
      const bool valid = lane < max_pop && e >= 0;
      const uint2 t = valid ? sm.stk[e] : make_uint2(0u, 0u);
      const int nt = valid ? task_tests(t, W) : 0;
      const int incl = warp_scan_incl(nt, lane);
      int npop = __popc(__ballot_sync(FULL, valid && incl <= 32));
      if (npop == 0) npop = 1;
      int T = __shfl_sync(FULL, incl, npop - 1);
      // the pushes must fit: shrink the batch, down to one task
      while (npop > 1 && sp - npop + T > stack_cap) {
        --npop;
        T = __shfl_sync(FULL, incl, npop - 1);
      }
      if (sp - npop + T > stack_cap) return -1;
      if (lane < npop) {
        sm.tq[lane] = t;
        sm.tpre[lane] = incl - nt;
        cnt.v[C_BYTES] += node_pair_bytes<W>(t.x & kExpand, t.y & kExpand);
      }
      __syncwarp();
      sp -= npop;
      for (int base = 0; base < T; base += 32) {
        const int u = base + lane;
        const bool act = u < T;
        int k = 0;
        if (act) {
          int lo = 0, hi = npop - 1;
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sm.tpre[mid] <= u) lo = mid; else hi = mid - 1;
          }
          k = lo;
        }
        const uint2 tk = act ? sm.tq[k] : make_uint2(0u, 0u);
        const int r = act ? u - sm.tpre[k] : 0;
        const bool xa = tk.x & kExpand, xb = tk.y & kExpand;
        const int nB = xb ? W : 1;
        const int i = r / nB, j = r - (r / nB) * nB;
        bool ok = act;
        Box ba, bb;
        uint32_t na = 0, nb = 0;
        if (act) {
          uint32_t ca, cb;
          const uint32_t ia2 = tk.x & kIdx, ib2 = tk.y & kIdx;
          if (xa) {
            load_slot<W>(A.nodes, ia2, i, zero, ba, ca);
            ok = ok && ca != kEmpty;
            na = (ca & kLeafBit) ? (kLeafBit | (ia2 * W + i)) : ca;
          } else if (tk.x & kLeafBit) {
            load_slot<W>(A.nodes, ia2 / W, (int)(ia2 % W), zero, ba, ca);
            na = tk.x;
          } else {
            load_slot<W>(A.nodes, ia2, -1, zero, ba, ca);
            na = tk.x & ~kExpand;
          }
          if (xb) {
            load_slot<W>(B.nodes, ib2, j, off, bb, cb);
            ok = ok && cb != kEmpty;
            nb = (cb & kLeafBit) ? (kLeafBit | (ib2 * W + j)) : cb;
          } else if (tk.y & kLeafBit) {
            load_slot<W>(B.nodes, ib2 / W, (int)(ib2 % W), off, bb, cb);
            nb = tk.y;
          } else {
            load_slot<W>(B.nodes, ib2, -1, off, bb, cb);
            nb = tk.y & ~kExpand;
          }
          ok = ok && overlap(ba, bb);
        }
        const bool both = ok && (na & kLeafBit) && (nb & kLeafBit);
        const bool push = ok && !both;
        const unsigned m1 = __ballot_sync(FULL, push), m2 = __ballot_sync(FULL, both);
        if (push) sm.stk[sp + __popc(m1 & lt)] = make_task(na, ba, nb, bb);
        if (both) sm.lq[nlq + __popc(m2 & lt)] = make_uint2(na, nb);
        sp += __popc(m1);
        nlq += __popc(m2);
      }
      if (lane == 0) {
        cnt.v[C_NODE_PAIRS] += npop;
        cnt.v[C_BOX_TESTS] += T;
      }
      __syncwarp();
      if (!split_done) {
        // several warps share this pair: after the first expansion each keeps
        // every nrank-th task and leaf pair
        split_done = true;
        int nsp = 0, nl = 0;
        for (int e0 = 0; e0 < sp; e0 += 32) {
          int ee = e0 + lane;
          bool keep = ee < sp && (ee % nrank) == rank;
          uint2 v = keep ? sm.stk[ee] : make_uint2(0, 0);
          unsigned m = __ballot_sync(FULL, keep);
          __syncwarp();
          if (keep) sm.stk[nsp + __popc(m & lt)] = v;
          nsp += __popc(m);
          __syncwarp();
        }
        for (int e0 = 0; e0 < nlq; e0 += 32) {
          int ee = e0 + lane;
          bool keep = ee < nlq && ((sp + ee) % nrank) == rank;
          uint2 v = keep ? sm.lq[ee] : make_uint2(0, 0);
          unsigned m = __ballot_sync(FULL, keep);
          __syncwarp();
          if (keep) sm.lq[nl + __popc(m & lt)] = v;
          nl += __popc(m);
          __syncwarp();
        }
        sp = nsp;
        nlq = nl;
      }
    }
    if (nlq > 0 && (sp == 0 || nlq + 64 > LQ || nlq >= 32)) {
      bool h = leaf_units<W, EXACT>(A, B, tA, tB, off, sm, nlq, lane, cnt);
      nlq = 0;
      __syncwarp();
      if (h) return 1;
    }
  }
  return 0;
}

// +z parity traversal from the exact point v against mesh `it` of side T
// (translated by toff).  Returns bit 0 = parity, bit 1 = v on the surface,
// or -1 on a capacity error.
template <int W>
__device__ int parity_query(const Side &T, int it, F3 toff, F3 vf, int ax, int dir, WarpMem &sm,
                            int lane, int stack_cap, int max_pop, Cnt &cnt) {
  constexpr int LQ = Cfg<W>::LQ;
  const int64_t tbase = T.toff[it];
  const I3 v = toi(vf);
  const unsigned lt = (1u << lane) - 1u;
  int sp = 1, nlq = 0;
  if (lane == 0) sm.stk[0].x = (uint32_t)T.roots[it];
  __syncwarp();
  bool on = false;
  int par = 0;
  if (lane == 0) cnt.v[C_PARITY_RAYS] += 1;
  unsigned iters = 0;
  while (sp > 0 || nlq > 0) {
    if (++iters > (1u << 26)) return -1;  // defensive bound: a tree walk is finite
    if (sp > 0 && nlq + 32 <= LQ) {
      int P = min(min(sp, 32 / W), max_pop);
      while (P > 0 && sp - P + P * W > stack_cap) --P;
      if (P == 0) return -1;
      const int ni = lane / W, c = lane % W;
      bool ok = ni < P;
      const uint32_t node = ok ? sm.stk[sp - 1 - ni].x : 0u;
      __syncwarp();
      sp -= P;
      uint32_t ch = kEmpty;
      if (ok) {
        Box b;
        load_slot<W>(T.nodes, node, c, toff, b, ch);
        ok = ch != kEmpty && ray_axis_box(vf, b, ax, dir);
      }
      const bool leaf = ok && (ch & kLeafBit);
      const bool inner = ok && !leaf;
      const unsigned m1 = __ballot_sync(FULL, inner), m2 = __ballot_sync(FULL, leaf);
      if (inner) sm.stk[sp + __popc(m1 & lt)].x = ch;
      if (leaf) sm.lq[nlq + __popc(m2 & lt)] = make_uint2(node * W + c, ch);
      sp += __popc(m1);
      nlq += __popc(m2);
      if (lane == 0) {
        cnt.v[C_PARITY_NODES] += P;
        cnt.v[C_BYTES] += (unsigned long long)P * W * 32;
      }
      __syncwarp();
    }
    if (nlq > 0 && (sp == 0 || nlq + 32 > LQ)) {
      // flatten the queued leaves' triangles over the lanes
      int run = 0;
      if (lane == 0) sm.lpre[0] = 0;
      for (int e0 = 0; e0 < nlq; e0 += 32) {
        int e = e0 + lane;
        int u = e < nlq ? (int)(sm.lq[e].y & 7u) + 1 : 0;
        int inc = warp_scan_incl(u, lane);
        if (e < nlq) sm.lpre[e + 1] = run + inc;
        run += __shfl_sync(FULL, inc, 31);
      }
      __syncwarp();
      for (int base = 0; base < run; base += 32) {
        int u = base + lane;
        if (u < run) {
          int lo = 0, hi = nlq - 1;
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sm.lpre[mid] <= u) lo = mid; else hi = mid - 1;
          }
          const uint32_t d = sm.lq[lo].y;
          const int64_t s = tbase + ((d >> 3) & 0x0FFFFFFFu) + (u - sm.lpre[lo]);
          F3 a, b, c;
          int own;
          load_tri(T.trirec, s, toff, a, b, c, own);
          I3 ai = toi(a), bi = toi(b), ci = toi(c);
          on = on || on_triangle(v, ai, bi, ci);
          par ^= ray_axis_hit(v, ai, bi, ci, ax, dir) ? 1 : 0;
          cnt.v[C_PARITY_TRIS] += 1;
          cnt.v[C_BYTES] += 48;
        }
      }
      nlq = 0;
      __syncwarp();
    }
  }
  bool on_any = __any_sync(FULL, on);
  int parity = __popc(__ballot_sync(FULL, par != 0)) & 1;
  return parity | (on_any ? 2 : 0);
}

// Whether the exact point v lies on a triangle of mesh `it` of side T
// (translated by toff), by one thread: a descent through the nodes whose
// closed box contains v.  Every triangle through v lies in a leaf whose box
// contains v, and a parity ray from v visits those leaves too, so this is
// the ray walk's on-surface answer without the rest of the ray.  Returns 1 /
// 0, or -1 when its stack (kPointStack entries) would overflow.
constexpr int kPointStack = 64;

template <int W>
__device__ int point_on_surface(const Side &T, int it, int64_t tbase, F3 toff, F3 vf,
                               unsigned long long &nodes, unsigned long long &tris) {
  const I3 v = toi(vf);
  uint32_t stk[kPointStack];
  int sp = 0;
  stk[sp++] = (uint32_t)T.roots[it];
  while (sp > 0) {
    const uint32_t node = stk[--sp];
    nodes += 1;
#pragma unroll 1
    for (int c = 0; c < W; ++c) {
      Box b;
      uint32_t ch;
      load_slot<W>(T.nodes, node, c, toff, b, ch);
      if (ch == kEmpty || vf.x < b.lo.x || vf.x > b.hi.x || vf.y < b.lo.y || vf.y > b.hi.y ||
          vf.z < b.lo.z || vf.z > b.hi.z)
        continue;
      if (ch & kLeafBit) {
        const int64_t first = tbase + ((ch >> 3) & 0x0FFFFFFFu);
        const int cntl = (int)(ch & 7u) + 1;
        for (int t = 0; t < cntl; ++t) {
          F3 a, bb, cc;
          int own;
          load_tri(T.trirec, first + t, toff, a, bb, cc, own);
          tris += 1;
          if (on_triangle(v, toi(a), toi(bb), toi(cc))) return 1;
        }
      } else {
        if (sp >= kPointStack) return -1;
        stk[sp++] = ch;
      }
    }
  }
  return 0;
}

// inside(Q_iq, T_it): representative vertex of Q (lexicographically smallest
// not on T's surface) has odd +z parity against T.  A vertex outside T's
// closed box is off T's surface and has even parity (T is closed), which
// ends the search.  The first vertex takes one ray (it decides in most
// pairs); if it lies on T's surface, the following vertices are checked 32 at
// a time, one per lane, by point queries, and a ray runs for the first that
// is not on the surface (a vertex whose query overflowed takes the ray,
// which then decides whether it is on the surface).  Returns 1/0, or -1 on a
// capacity error.
template <int W>
__device__ int pair_inside(const Side &Q, int iq, F3 qoff, const Side &T, int it, F3 toff,
                           WarpMem &sm, int lane, int stack_cap, int max_pop, Cnt &cnt) {
  const int64_t v0 = Q.voff[iq], nv = Q.voff[iq + 1] - v0;
  const float *tb = T.aabb + 6 * (int64_t)it;
  F3 lo = add(ld3(tb), toff), hi = add(ld3(tb + 3), toff);
  auto outside = [&](F3 v) {
    return v.x < lo.x || v.x > hi.x || v.y < lo.y || v.y > hi.y || v.z < lo.z || v.z > hi.z;
  };
  if (nv <= 0) return 0;
  {
    const F3 v = add(ld3(Q.xyz + 3 * Q.lexorder[v0]), qoff);
    if (lane == 0) cnt.v[C_BYTES] += 16;
    if (outside(v)) return 0;
    int ax, dir;
    ray_axis_choice(v, lo, hi, ax, dir);
    const int r = parity_query<W>(T, it, toff, v, ax, dir, sm, lane, stack_cap, max_pop, cnt);
    if (r < 0) return -1;
    if (!(r & 2)) return r & 1;
  }
  const int64_t tbase = T.toff[it];
  for (int64_t k0 = 1; k0 < nv; k0 += 32) {
    const int64_t k = k0 + lane;
    // 0: on T's surface (skipped), 1: outside T's box, 2: off the surface,
    // 3: not known (the query's stack overflowed)
    int status = 0;
    F3 v = mkf3(0.f, 0.f, 0.f);
    if (k < nv) {
      v = add(ld3(Q.xyz + 3 * Q.lexorder[v0 + k]), qoff);
      if (outside(v)) {
        status = 1;
      } else {
        unsigned long long nn = 0, tt = 0;
        const int on = point_on_surface<W>(T, it, tbase, toff, v, nn, tt);
        status = on == 1 ? 0 : (on == 0 ? 2 : 3);
        cnt.v[C_PARITY_NODES] += nn;
        cnt.v[C_PARITY_TRIS] += tt;
        cnt.v[C_BYTES] += nn * W * 32 + tt * 48;
      }
      cnt.v[C_BYTES] += 16;
    }
    unsigned m = __ballot_sync(FULL, status != 0);
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      const int st = __shfl_sync(FULL, status, l);
      if (st == 1) return 0;
      const F3 vl = mkf3(__shfl_sync(FULL, v.x, l), __shfl_sync(FULL, v.y, l),
                         __shfl_sync(FULL, v.z, l));
      int ax, dir;
      ray_axis_choice(vl, lo, hi, ax, dir);
      const int r = parity_query<W>(T, it, toff, vl, ax, dir, sm, lane, stack_cap, max_pop, cnt);
      if (r < 0) return -1;
      if (!(r & 2)) return r & 1;
    }
  }
  return 0;
}

// Some vertex of Q_iq strictly inside T_it: off T's surface with odd ray
// parity (the any-vertex completeness mode).  Vertices outside T's closed box
// are outside T.  Returns 1/0, or -1 on a capacity error.
template <int W>
__device__ int pair_any_inside(const Side &Q, int iq, F3 qoff, const Side &T, int it, F3 toff,
                               WarpMem &sm, int lane, int stack_cap, int max_pop, Cnt &cnt) {
  const int64_t v0 = Q.voff[iq], nv = Q.voff[iq + 1] - v0;
  const float *tb = T.aabb + 6 * (int64_t)it;
  F3 lo = add(ld3(tb), toff), hi = add(ld3(tb + 3), toff);
  for (int64_t k = 0; k < nv; ++k) {
    F3 v = add(ld3(Q.xyz + 3 * (v0 + k)), qoff);
    if (lane == 0) cnt.v[C_BYTES] += 12;
    if (v.x < lo.x || v.x > hi.x || v.y < lo.y || v.y > hi.y || v.z < lo.z || v.z > hi.z)
      continue;
    int ax, dir;
    ray_axis_choice(v, lo, hi, ax, dir);
    int r = parity_query<W>(T, it, toff, v, ax, dir, sm, lane, stack_cap, max_pop, cnt);
    if (r < 0) return -1;
    if (r == 1) return 1;
  }
  return 0;
}

__device__ __forceinline__ void bar_group(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int W, bool EXACT>
__global__ void __launch_bounds__(128, 4) k_refine(RefineArgs P) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int group_flag[4];
  __shared__ long long group_cand[4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int k = P.warps_per_pair;
  const int grp = wib / k, rank = wib % k;
  WarpMem sm = carve<W>(smem + (size_t)wib * warp_smem_bytes<W>(P.stack_cap), P.stack_cap);
  Cnt cnt;
  for (int i = 0; i < C_WARP_NUM; ++i) cnt.v[i] = 0;
  const int64_t n = *P.n_cand;
  bool first = true;
  for (;;) {
    long long c;
    if (P.single >= 0) {
      c = first ? P.single : n;
      first = false;
    } else {
      if (k > 1) {
        if (rank == 0 && lane == 0) {
          group_cand[grp] = (long long)atomicAdd(P.work, 1ull);
          group_flag[grp] = 0;
        }
        bar_group(1 + grp, 32 * k);
        c = group_cand[grp];
      } else {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(P.work, 1ull);
        c = (long long)__shfl_sync(FULL, w, 0);
      }
    }
    if (c >= n) break;
    const long long t_start = clock64();
    const int ia = P.cand[2 * c], ib = P.cand[2 * c + 1];
    if (ia < 0 || ia >= P.MA || ib < 0 || ib >= P.MB) {
      // reported by the candidate check; never dereference a bad id
      if (rank == 0 && lane == 0) P.flags[c] = 0;
      continue;
    }
    F3 off = mkf3(0.f, 0.f, 0.f);
    if (P.cand_off)
      off = mkf3((float)P.cand_off[3 * c], (float)P.cand_off[3 * c + 1], (float)P.cand_off[3 * c + 2]);
    const float *ba = P.A.aabb + 6 * (int64_t)ia, *bb = P.B.aabb + 6 * (int64_t)ib;
    bool overlap = ba[0] <= bb[3] + off.x && bb[0] + off.x <= ba[3] && ba[1] <= bb[4] + off.y &&
                   bb[1] + off.y <= ba[4] && ba[2] <= bb[5] + off.z && bb[2] + off.z <= ba[5];
    volatile int *gflag = k > 1 ? &group_flag[grp] : nullptr;
    Spill spill;
    spill.q = P.q_out;
    spill.q_n = P.q_out_n;
    spill.q_cap = P.q_cap;
    spill.budget = (k == 1 && P.q_out) ? P.budget : 0;
    spill.flag = nullptr;
    spill.cand = (uint32_t)c;
    int res = 0;
    if (overlap)
      res = pair_cross<W, EXACT>(P.A, P.B, ia, ib, off, sm, lane, P.stack_cap, P.max_pop, cnt,
                                 gflag, rank, k, spill, true, make_uint2(0u, 0u));
    if (res == -2) {
      res = 0;  // the crossing test continues in the next pass
    } else if (res < 0) {
      if (lane == 0) atomicCAS(P.err, 0, res == -3 ? DERR_QUEUE : DERR_STACK);
      res = 0;
    }
    if (k > 1) {
      if (res == 1 && lane == 0) group_flag[grp] = 1;
      bar_group(1 + grp, 32 * k);
      res = group_flag[grp];
      bar_group(1 + grp, 32 * k);
    }
    // containment (Sec. 3.3): both directions for intersects, one for
    // contains (B_j inside A_i) or within (A_i inside B_j), none for overlap;
    // with several warps per pair, ranks 0 and 1 take one direction each
    const bool dBA = P.predicate != PJ_PRED_OVERLAP && P.predicate != PJ_PRED_WITHIN;
    const bool dAB = P.predicate != PJ_PRED_OVERLAP && P.predicate != PJ_PRED_CONTAINS;
    int ins = 0;
    if (!res && (dBA || dAB)) {
      int r1 = 0, r2 = 0;
      F3 zero = mkf3(0.f, 0.f, 0.f);
      if (rank == 0 && dBA)
        r1 = pair_inside<W>(P.B, ib, off, P.A, ia, zero, sm, lane, P.stack_cap, P.max_pop, cnt);
      if (dAB && ((k == 1 && r1 == 0) || (k > 1 && rank == 1)))
        r2 = pair_inside<W>(P.A, ia, zero, P.B, ib, off, sm, lane, P.stack_cap, P.max_pop, cnt);
      if (r1 < 0 || r2 < 0) {
        if (lane == 0) atomicCAS(P.err, 0, DERR_STACK);
        r1 = r2 = 0;
      }
      ins = (r1 > 0 || r2 > 0) ? 1 : 0;
      if (k > 1) {
        if (ins && lane == 0) group_flag[grp] = 1;
        bar_group(1 + grp, 32 * k);
        ins = group_flag[grp];
        bar_group(1 + grp, 32 * k);
      }
    }
    if (P.pflags) {
      if (rank == 0 && lane == 0) P.pflags[c] = (uint8_t)ins;  // flags[c] = the crossing
    } else {
      res = res || ins;
    }
    if (rank == 0 && lane == 0) {
      if (P.cycles) {
        long long dt = clock64() - t_start;
        P.cycles[c] = dt > 0xFFFFFFFFll ? 0xFFFFFFFFu : (unsigned int)dt;
      }
      P.flags[c] = (uint8_t)res;
      cnt.v[C_PAIRS] += 1;
      cnt.v[C_BYTES] += 8 + 1 + 48;
    }
  }
  // flush counters (warp-aggregated)
  for (int i = 0; i < C_WARP_NUM; ++i) {
    unsigned long long v = cnt.v[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(P.counters + i, v);
  }
}

// ---------------------------------------------------------------------------
// Wavefront front end.  Most candidate pairs are decided in the top few
// levels of the two BVHs (boxes stop overlapping, or the parity ray finds
// little); handing each of them a whole warp leaves most lanes idle on memory
// latency.  The front end therefore runs the first levels breadth-first with
// one thread per child test, the parity rays with one thread per (pair,
// direction) and the leaf-pair tests with one thread per source triangle;
// whatever is left after those levels goes to the warp-DFS passes as queued
// (candidate, itemA, itemB) tasks.
// ---------------------------------------------------------------------------
struct WaveArgs {
  Side A, B;
  const int32_t *cand;
  const int32_t *cand_off;
  const int64_t *n_cand;
  uint8_t *flags;
  unsigned long long *counters;
  int *err;
  unsigned int q_cap;
  int lshift;                // log2 of the leaf size L: 2L threads per leaf pair
  int64_t MA, MB;
  uint4 *q_par;              // parity rays over the per-thread node budget
  unsigned int *q_par_n;
  unsigned int q_par_cap;
  int par_dirs;              // parity rays cast: bit 0 inside(B, A), bit 1 inside(A, B)
  uint8_t *pflags;           // where parity results go (null: flags)
  const uint8_t *need;       // non-null: only candidates with need[c] != 0 are traversed
};

__device__ __forceinline__ F3 cand_offset(const WaveArgs &P, int64_t c) {
  if (!P.cand_off) return mkf3(0.f, 0.f, 0.f);
  return mkf3((float)P.cand_off[3 * c], (float)P.cand_off[3 * c + 1], (float)P.cand_off[3 * c + 2]);
}

// warp-aggregated append of `cnt` entries; returns this lane's first index
__device__ __forceinline__ unsigned warp_append(unsigned *ctr, unsigned cnt, int lane) {
  unsigned incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  unsigned total = __shfl_sync(FULL, incl, 31);
  unsigned base = 0;
  if (lane == 31 && total) base = atomicAdd(ctr, total);
  base = __shfl_sync(FULL, base, 31);
  return base + incl - cnt;
}

// Block-aggregated append of two per-thread counts to two queues (one atomic
// per queue and block instead of one per warp: the queue counters are single
// addresses that every block hits).  Every thread of the block calls it with
// block-uniform control flow.  Per-thread counts are below 2^16 / blockDim.x.
// Returns this thread's first index in each queue.
__device__ __forceinline__ uint2 block_append2(unsigned *ctr0, unsigned cnt0, unsigned *ctr1,
                                               unsigned cnt1) {
  __shared__ unsigned s_off[32];
  __shared__ unsigned s_base[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned mine = cnt0 | (cnt1 << 16);
  unsigned incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_off[w] = incl;
  __syncthreads();
  if (w == 0) {
    const unsigned v = lane < nw ? s_off[lane] : 0u;
    unsigned inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    s_off[lane] = inc - v;
    const unsigned tot = __shfl_sync(FULL, inc, 31);
    if (lane == 0) s_base[0] = (tot & 0xFFFFu) ? atomicAdd(ctr0, tot & 0xFFFFu) : 0u;
    if (lane == 1) s_base[1] = (tot >> 16) ? atomicAdd(ctr1, tot >> 16) : 0u;
  }
  __syncthreads();
  const unsigned ex = s_off[w] + incl - mine;
  const uint2 r = make_uint2(s_base[0] + (ex & 0xFFFFu), s_base[1] + (ex >> 16));
  __syncthreads();  // s_off / s_base are reused by the next call
  return r;
}

// Sum N per-thread counter values over the block and add them to the device
// counters `slot[i]`: one atomic per block and counter.  Every thread of the
// block calls it.
template <int N>
__device__ __forceinline__ void block_flush(unsigned long long *dst, const int (&slot)[N],
                                            const unsigned long long (&v)[N]) {
  __shared__ unsigned long long s_sum[N];
  __syncwarp();
  if (threadIdx.x < N) s_sum[threadIdx.x] = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < N; ++i) {
    unsigned long long x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if (lane == 0 && x) atomicAdd(&s_sum[i], x);
  }
  __syncthreads();
  if (threadIdx.x < N && s_sum[threadIdx.x]) atomicAdd(dst + slot[threadIdx.x], s_sum[threadIdx.x]);
}

__device__ __forceinline__ void flush_counters(unsigned long long *dst, const unsigned long long *v,
                                               int lane, int n) {
  for (int i = 0; i < n; ++i) {
    unsigned long long x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if (lane == 0 && x) atomicAdd(dst + i, x);
  }
}

// root task of every candidate whose mesh boxes meet
__global__ void k_wave_init(WaveArgs P, uint4 *q, unsigned *q_n) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = *P.n_cand;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0 && n > 0)
    atomicAdd(P.counters + C_PAIRS, (unsigned long long)n);
  for (int64_t g0 = blockIdx.x * (int64_t)blockDim.x; g0 < n; g0 += stride) {
    const int64_t g = g0 + threadIdx.x;
    bool push = false;
    uint2 t = make_uint2(0u, 0u);
    if (g < n && (!P.need || P.need[g])) {
      const int ia = P.cand[2 * g], ib = P.cand[2 * g + 1];
      if (ia >= 0 && ia < P.MA && ib >= 0 && ib < P.MB) {
        const F3 off = cand_offset(P, g);
        Box ba, bb;
        const float4 a0 = P.A.mrec[3 * (int64_t)ia], a1 = P.A.mrec[3 * (int64_t)ia + 1];
        const float4 b0 = P.B.mrec[3 * (int64_t)ib], b1 = P.B.mrec[3 * (int64_t)ib + 1];
        ba.lo = mkf3(a0.x, a0.y, a0.z);
        ba.hi = mkf3(a1.x, a1.y, a1.z);
        bb.lo = add(mkf3(b0.x, b0.y, b0.z), off);
        bb.hi = add(mkf3(b1.x, b1.y, b1.z), off);
        if (overlap(ba, bb)) {
          t = make_task((uint32_t)P.A.roots[ia], ba, (uint32_t)P.B.roots[ib], bb);
          push = true;
        }
      }
    }
    const unsigned pos = block_append2(q_n, push ? 1u : 0u, q_n, 0u).x;
    if (push && pos < P.q_cap) q[pos] = make_uint4((uint32_t)g, t.x, t.y, 0u);
    if (push && pos >= P.q_cap) atomicCAS(P.err, 0, DERR_QUEUE);
  }
}

// box of an item (an internal node's own box, or a leaf's slot box)
template <int W>
__device__ __forceinline__ void item_box(const float *nodes, uint32_t item, F3 off, Box &b) {
  uint32_t dummy;
  const uint32_t idx = item & kIdx;
  if (item & kLeafBit) load_slot<W>(nodes, idx / W, (int)(idx % W), off, b, dummy);
  else load_slot<W>(nodes, idx, -1, off, b, dummy);
}

// box and child word of an item's slot (the word is a leaf's descriptor;
// for an internal node's own box it is unused)
template <int W>
__device__ __forceinline__ void item_box_w(const float *nodes, uint32_t item, F3 off, Box &b,
                                           uint32_t &word) {
  const uint32_t idx = item & kIdx;
  if (item & kLeafBit) load_slot<W>(nodes, idx / W, (int)(idx % W), off, b, word);
  else load_slot<W>(nodes, idx, -1, off, b, word);
}

// One breadth-first level: W threads per task; thread i tests child i of
// the expanding side (against every child of the other side when both
// expand).  Surviving children become tasks of the next level, or leaf
// pairs.
template <int W>
__global__ void __launch_bounds__(256) k_wave_expand(WaveArgs P, const uint4 *qin,
                                                     const unsigned *qin_n, uint4 *qout,
                                                     unsigned *qout_n, uint4 *lq, unsigned *lq_n) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = (int64_t)min(*qin_n, P.q_cap) * W;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  unsigned long long cnt[3] = {0, 0, 0};  // node pairs, box tests, bytes
  for (int64_t g0 = blockIdx.x * (int64_t)blockDim.x; g0 < n; g0 += stride) {
    const int64_t g = g0 + threadIdx.x;
    unsigned task_mask = 0, leaf_mask = 0;
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    int i = 0;
    bool xa = false, xb = false;
    F3 off = zero;
    Box ba;
    uint32_t na = 0;
    bool live = false;
    if (g < n) {
      e = qin[g / W];
      i = (int)(g % W);
      live = P.flags[e.x] == 0;
      xa = e.y & kExpand;
      xb = e.z & kExpand;
      // with one side expanding only its W children are tested
      if (!(xa && xb) && !xa && !xb) live = false;
    }
    if (live) {
      off = cand_offset(P, e.x);
      if (xa) {
        uint32_t ca;
        load_slot<W>(P.A.nodes, e.y & kIdx, i, zero, ba, ca);
        if (ca == kEmpty) live = false;
        na = (ca & kLeafBit) ? (kLeafBit | ((e.y & kIdx) * W + i)) : ca;
      } else {
        item_box<W>(P.A.nodes, e.y, zero, ba);
        na = e.y & ~kExpand;
      }
      if (i == 0) {
        cnt[0] += 1;
        cnt[2] += node_pair_bytes<W>(xa, xb);
      }
    }
    if (live) {
      if (xb) {
        const int j0 = xa ? 0 : i, j1 = xa ? W : i + 1;
        for (int j = j0; j < j1; ++j) {
          Box bb;
          uint32_t cb;
          load_slot<W>(P.B.nodes, e.z & kIdx, j, off, bb, cb);
          cnt[1] += 1;
          if (cb == kEmpty || !overlap(ba, bb)) continue;
          const bool lb = cb & kLeafBit;
          if ((na & kLeafBit) && lb) leaf_mask |= 1u << j;
          else task_mask |= 1u << j;
        }
      } else {
        Box bb;
        item_box<W>(P.B.nodes, e.z, off, bb);
        cnt[1] += 1;
        if (overlap(ba, bb)) {
          if ((na & kLeafBit) && (e.z & kLeafBit)) leaf_mask = 1u;
          else task_mask = 1u;
        }
      }
    }
    // write the outputs (the B-side children are reloaded: L1 hits)
    const uint2 pos = block_append2(qout_n, __popc(task_mask), lq_n, __popc(leaf_mask));
    unsigned tpos = pos.x, lpos = pos.y;
    unsigned bits = task_mask | leaf_mask;
    while (bits) {
      const int j = __ffs(bits) - 1;
      bits &= bits - 1;
      Box bb;
      uint32_t nb;
      if (xb) {
        uint32_t cb;
        const int jj = xa ? j : i;
        load_slot<W>(P.B.nodes, e.z & kIdx, jj, off, bb, cb);
        nb = (cb & kLeafBit) ? (kLeafBit | ((e.z & kIdx) * W + jj)) : cb;
      } else {
        item_box<W>(P.B.nodes, e.z, off, bb);
        nb = e.z & ~kExpand;
      }
      if ((task_mask >> j) & 1u) {
        if (tpos < P.q_cap) {
          uint2 t = make_task(na, ba, nb, bb);
          qout[tpos] = make_uint4(e.x, t.x, t.y, 0u);
        } else {
          atomicCAS(P.err, 0, DERR_QUEUE);
        }
        ++tpos;
      } else {
        if (lpos < P.q_cap) lq[lpos] = make_uint4(e.x, na, nb, 0u);
        else atomicCAS(P.err, 0, DERR_QUEUE);
        ++lpos;
      }
    }
  }
  const int slots[4] = {C_NODE_PAIRS, C_BOX_TESTS, C_BYTES, C_BYTES_EXPAND};
  const unsigned long long v[4] = {cnt[0], cnt[1], cnt[2], cnt[2]};
  block_flush<4>(P.counters, slots, v);
}

// Per-thread counters of the leaf-pair work (32-bit: one thread's share of
// one launch stays far below 2^32).
struct LeafCnt {
  unsigned lp = 0, slab = 0, st = 0, fb = 0, bytes = 0;
};

// One unit of a leaf pair e = (candidate, leaf item A, leaf item B): unit u
// in [0, 2L) takes source triangle u mod L of side A (u < L) or of side B,
// slab-tests its owned edges against the other leaf's box and tests them
// exactly against the other leaf's triangles.  Returns true on a crossing.
template <int W, bool EXACT>
__device__ __forceinline__ bool leaf_unit(const WaveArgs &P, const uint4 e, const int u,
                                          LeafCnt &cn) {
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  const bool dirA = (u >> P.lshift) == 0;
  const int k = u & ((1 << P.lshift) - 1);
  const uint32_t sslot = (dirA ? e.y : e.z) & kIdx, tslot = (dirA ? e.z : e.y) & kIdx;
  const Side &S = dirA ? P.A : P.B;
  const Side &T = dirA ? P.B : P.A;
  Box sbox, tb;
  uint32_t sdesc, tdesc;
  load_slot<W>(S.nodes, sslot / W, (int)(sslot % W), zero, sbox, sdesc);
  if (k > (int)(sdesc & 7u)) return false;
  const int ia = P.cand[2 * (int64_t)e.x], ib = P.cand[2 * (int64_t)e.x + 1];
  const F3 off = cand_offset(P, e.x);
  const F3 soff = dirA ? zero : off, toff = dirA ? off : zero;
  load_slot<W>(T.nodes, tslot / W, (int)(tslot % W), toff, tb, tdesc);
  if (u == 0) cn.lp += 1;
  const int64_t sbase = __float_as_int(S.mrec[3 * (int64_t)(dirA ? ia : ib) + 2].y);
  const int64_t tbase = __float_as_int(T.mrec[3 * (int64_t)(dirA ? ib : ia) + 2].y);
  const int64_t s_rec = sbase + ((sdesc >> 3) & 0x0FFFFFFFu) + k;
  const int64_t t_first = tbase + ((tdesc >> 3) & 0x0FFFFFFFu);
  const int t_n = (int)(tdesc & 7u) + 1;
  F3 v[3];
  int own;
  load_tri(S.trirec, s_rec, soff, v[0], v[1], v[2], own);
  // the source triangle and the two leaf slots (source descriptor, target
  // box and descriptor)
  cn.bytes += 48 + 64;
  for (int ek = 0; ek < 3; ++ek) {
    if (!((own >> ek) & 1)) continue;
    const F3 p = v[ek], qv = v[ek == 2 ? 0 : ek + 1];
    Seg sg = make_seg(p, qv);
    cn.slab += 1;
    if (!slab_hit(sg, tb.lo, tb.hi)) continue;
    const F3 elo = mkf3(fminf(p.x, qv.x), fminf(p.y, qv.y), fminf(p.z, qv.z));
    const F3 ehi = mkf3(fmaxf(p.x, qv.x), fmaxf(p.y, qv.y), fmaxf(p.z, qv.z));
    for (int t = 0; t < t_n; ++t) {
      F3 a, b, c;
      int town;
      load_tri(T.trirec, t_first + t, toff, a, b, c, town);
      cn.bytes += 48;
      const float lx = fminf(a.x, fminf(b.x, c.x)), hx = fmaxf(a.x, fmaxf(b.x, c.x));
      const float ly = fminf(a.y, fminf(b.y, c.y)), hy = fmaxf(a.y, fmaxf(b.y, c.y));
      const float lz = fminf(a.z, fminf(b.z, c.z)), hz = fmaxf(a.z, fmaxf(b.z, c.z));
      if (lx > ehi.x || elo.x > hx || ly > ehi.y || elo.y > hy || lz > ehi.z || elo.z > hz)
        continue;
      cn.st += 1;
      bool r;
      if (EXACT) {
        r = segtri_exact_staged(p, qv, a, b, c);
      } else {
        bool ex = false;
        r = segtri_filtered(p, qv, a, b, c, &ex);
        cn.fb += ex ? 1 : 0;
      }
      if (r) return true;
    }
  }
  return false;
}

// Leaf pairs: 2L threads per pair (the L source triangles of each side).
template <int W, bool EXACT>
__global__ void __launch_bounds__(256, 3) k_wave_leaf(WaveArgs P, const uint4 *lq, const unsigned *lq_n) {
  pdl_wait();
  pdl_trigger();
  const int sh = P.lshift + 1;               // 2L = 1 << sh threads per pair
  const int64_t n = (int64_t)min(*lq_n, P.q_cap) << sh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  LeafCnt cn;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += stride) {
    const uint4 e = lq[g >> sh];
    const int u = (int)(g & ((1 << sh) - 1));
    if (P.flags[e.x]) continue;
    if (leaf_unit<W, EXACT>(P, e, u, cn)) P.flags[e.x] = 1;
  }
  const int slots[6] = {C_LEAF_PAIRS, C_SLAB_TESTS, C_SEGTRI, C_FALLBACK, C_BYTES, C_BYTES_LEAF};
  const unsigned long long v[6] = {cn.lp, cn.slab, cn.st, cn.fb, cn.bytes, cn.bytes};
  block_flush<6>(P.counters, slots, v);
}

// Parity rays, one thread per (pair, direction): inside(B, A) for even
// threads, inside(A, B) for odd ones.  Depth-first with a per-thread stack
// (bounded by 1 + (W - 1) * depth).  A ray that needs more than
// kParNodeBudget nodes (one that runs along a long tube, say) would hold its
// whole block back; it is handed to the warp passes instead (-2).
constexpr int kParNodeBudget = 4;
constexpr uint32_t kParItem = 0xFFFFFFFEu;  // queue entry: (c, kParItem, direction)

template <int W>
__device__ int thread_parity(const Side &T, int it, int64_t tbase, F3 toff, F3 vf, int ax, int dir,
                             uint32_t *stk, int cap, unsigned long long &nodes,
                             unsigned long long &tris) {
  const I3 v = toi(vf);
  int sp = 0;
  stk[sp++] = (uint32_t)T.roots[it];
  bool on = false;
  int par = 0;
  unsigned iters = 0;
  while (sp > 0) {
    if (++iters > (unsigned)kParNodeBudget) return -2;
    const uint32_t node = stk[--sp];
    nodes += 1;
    // the node's W child slots as one batch of independent loads (a thread
    // walks alone, so every serial load is a full memory latency)
    uint32_t ch[W];
    unsigned leaves = 0;
    {
      Box b[W];
#pragma unroll
      for (int c = 0; c < W; ++c) load_slot<W>(T.nodes, node, c, toff, b[c], ch[c]);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (ch[c] == kEmpty || !ray_axis_box(vf, b[c], ax, dir)) continue;
        if (ch[c] & kLeafBit) {
          leaves |= 1u << c;
        } else {
          if (sp >= cap) return -1;
          stk[sp++] = ch[c];
        }
      }
    }
    while (leaves) {
      const int c = __ffs(leaves) - 1;
      leaves &= leaves - 1;
      const uint32_t lc = sel_u32<W>(ch, c);
      const int64_t first = tbase + ((lc >> 3) & 0x0FFFFFFFu);
      const int cntl = (int)(lc & 7u) + 1;
      for (int t0 = 0; t0 < cntl; t0 += 4) {
        // up to four of the leaf's triangles per batch of loads
        F3 ta[4], tb[4], tc[4];
        int own;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t0 + t < cntl) load_tri(T.trirec, first + t0 + t, toff, ta[t], tb[t], tc[t], own);
        const int tn = min(4, cntl - t0);
#pragma unroll 1
        for (int t = 0; t < tn; ++t) {
          const I3 ai = toi(sel_f3<4>(ta, t)), bi = toi(sel_f3<4>(tb, t)), ci = toi(sel_f3<4>(tc, t));
          on = on || on_triangle(v, ai, bi, ci);
          par ^= ray_axis_hit(v, ai, bi, ci, ax, dir) ? 1 : 0;
          tris += 1;
        }
      }
    }
  }
  return par | (on ? 2 : 0);
}

template <int W>
__global__ void __launch_bounds__(128) k_wave_parity(WaveArgs P) {
  pdl_wait();
  pdl_trigger();
  // the node budget bounds the stack: each pop pushes at most W - 1 more
  constexpr int CAP = 1 + (W - 1) * kParNodeBudget;
  uint32_t stk[CAP];
  const int64_t n = *P.n_cand * 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  unsigned long long rays = 0, nodes = 0, tris = 0, bytes = 0, handed = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += stride) {
    const int64_t c = g >> 1;
    const bool bInA = (g & 1) == 0;
    if (!((P.par_dirs >> (bInA ? 0 : 1)) & 1)) continue;  // direction not asked for
    const int ia = P.cand[2 * c], ib = P.cand[2 * c + 1];
    if (ia < 0 || ia >= P.MA || ib < 0 || ib >= P.MB) continue;
    const F3 off = cand_offset(P, c);
    const Side &Q = bInA ? P.B : P.A;
    const Side &T = bInA ? P.A : P.B;
    const int iq = bInA ? ib : ia, it = bInA ? ia : ib;
    const F3 qoff = bInA ? off : zero, toff = bInA ? zero : off;
    // one fetch per side: T's box and first triangle, Q's first lexicographic
    // vertex and vertex range
    const float4 t0 = T.mrec[3 * (int64_t)it], t1 = T.mrec[3 * (int64_t)it + 1];
    const float4 t2 = T.mrec[3 * (int64_t)it + 2];
    const float4 q0 = Q.mrec[3 * (int64_t)iq], q1 = Q.mrec[3 * (int64_t)iq + 1];
    const float4 q2 = Q.mrec[3 * (int64_t)iq + 2];
    const int64_t tbase = __float_as_int(t2.y);
    const int64_t v0 = __float_as_int(q2.z), nv = __float_as_int(q2.w);
    const F3 lo = add(mkf3(t0.x, t0.y, t0.z), toff), hi = add(mkf3(t1.x, t1.y, t1.z), toff);
    bytes += 96;
    int res = 0;
    for (int64_t k = 0; k < nv; ++k) {
      F3 v;
      if (k == 0) {
        v = add(mkf3(q0.w, q1.w, q2.x), qoff);
      } else {
        const int64_t vid = Q.lexorder[v0 + k];
        v = add(ld3(Q.xyz + 3 * vid), qoff);
        bytes += 16;
      }
      if (v.x < lo.x || v.x > hi.x || v.y < lo.y || v.y > hi.y || v.z < lo.z || v.z > hi.z) break;
      rays += 1;
      const unsigned long long n0 = nodes, t0 = tris;
      int ax, dir;
      ray_axis_choice(v, lo, hi, ax, dir);
      const int r = thread_parity<W>(T, it, tbase, toff, v, ax, dir, stk, CAP, nodes, tris);
      bytes += (nodes - n0) * W * 32 + (tris - t0) * 48;
      if (r == -2) {
        // over the node budget: a warp redoes this direction from the start
        handed += 1;
        const unsigned pos = atomicAdd(P.q_par_n, 1u);
        if (pos < P.q_par_cap) P.q_par[pos] = make_uint4((uint32_t)c, kParItem, bInA ? 0u : 1u, 0u);
        else atomicCAS(P.err, 0, DERR_QUEUE);
        break;
      }
      if (r < 0) {
        atomicCAS(P.err, 0, DERR_STACK);
        break;
      }
      if (!(r & 2)) {
        res = r & 1;
        break;
      }
    }
    if (res) (P.pflags ? P.pflags : P.flags)[c] = 1;
  }
  const int slots[6] = {C_PARITY_RAYS, C_PARITY_NODES, C_PARITY_TRIS, C_BYTES, C_BYTES_PARITY,
                        C_PAR_HANDOVER};
  const unsigned long long v[6] = {rays, nodes, tris, bytes, bytes, handed};
  block_flush<6>(P.counters, slots, v);
}

// Later passes: warps pop spilled (candidate, itemA, itemB) tasks and continue
// the crossing test from there.  A crossing sets the candidate's flag (the
// first pass already stored the containment result; a crossing can only add
// to it).  Pairs already known to intersect are skipped.
template <int W, bool EXACT>
__global__ void __launch_bounds__(128, 4) k_refine_tasks(RefineArgs P) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpMem sm = carve<W>(smem + (size_t)wib * warp_smem_bytes<W>(P.stack_cap), P.stack_cap);
  Cnt cnt;
  for (int i = 0; i < C_WARP_NUM; ++i) cnt.v[i] = 0;
  // first the handed-over parity rays (the longest items), one warp each
  const unsigned int np = P.q_par ? min(*P.q_par_n, P.q_par_cap) : 0u;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0 && np) t = atomicAdd(P.q_par_pos, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= np) break;
    const uint4 e = P.q_par[t];
    const uint32_t c = e.x;
    volatile uint8_t *flag = (P.pflags ? P.pflags : P.flags) + c;
    int done = lane == 0 ? (int)*flag : 0;
    if (__shfl_sync(FULL, done, 0)) continue;
    const int ia = P.cand[2 * (int64_t)c], ib = P.cand[2 * (int64_t)c + 1];
    F3 off = mkf3(0.f, 0.f, 0.f);
    if (P.cand_off)
      off = mkf3((float)P.cand_off[3 * (int64_t)c], (float)P.cand_off[3 * (int64_t)c + 1],
                 (float)P.cand_off[3 * (int64_t)c + 2]);
    const F3 zero = mkf3(0.f, 0.f, 0.f);
    // direction 0: B's representative vertex against A; 1: A's against B
    const int r = e.z == 0u
        ? pair_inside<W>(P.B, ib, off, P.A, ia, zero, sm, lane, P.stack_cap, P.max_pop, cnt)
        : pair_inside<W>(P.A, ia, zero, P.B, ib, off, sm, lane, P.stack_cap, P.max_pop, cnt);
    if (r == 1) {
      if (lane == 0) *flag = 1;
    } else if (r < 0) {
      if (lane == 0) atomicCAS(P.err, 0, DERR_STACK);
    }
  }
  const unsigned long long par_bytes = cnt.v[C_BYTES];
  const unsigned int n = min(*P.q_in_n, P.q_in_cap);
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(P.q_in_pos, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= n) break;
    const uint4 e = P.q_in[t];
    const uint32_t c = e.x;
    volatile uint8_t *flag = P.flags + c;
    int done = lane == 0 ? (int)*flag : 0;
    if (__shfl_sync(FULL, done, 0)) continue;
    const int ia = P.cand[2 * (int64_t)c], ib = P.cand[2 * (int64_t)c + 1];
    F3 off = mkf3(0.f, 0.f, 0.f);
    if (P.cand_off)
      off = mkf3((float)P.cand_off[3 * (int64_t)c], (float)P.cand_off[3 * (int64_t)c + 1],
                 (float)P.cand_off[3 * (int64_t)c + 2]);
    Spill spill;
    spill.q = P.q_out;
    spill.q_n = P.q_out_n;
    spill.q_cap = P.q_cap;
    spill.budget = P.q_out ? P.budget : 0;
    spill.flag = flag;
    spill.cand = c;
    int res = pair_cross<W, EXACT>(P.A, P.B, ia, ib, off, sm, lane, P.stack_cap, P.max_pop, cnt,
                                   nullptr, 0, 1, spill, false, make_uint2(e.y, e.z));
    if (res == 1) {
      if (lane == 0) *flag = 1;
    } else if (res < -2 || res == -1) {
      if (lane == 0) atomicCAS(P.err, 0, res == -3 ? DERR_QUEUE : DERR_STACK);
    }
    if (lane == 0) cnt.v[C_TASKS] += 1;
  }
  cnt.v[C_BYTES_TASKS] = cnt.v[C_BYTES] - par_bytes;
  {
    unsigned long long v = par_bytes;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(P.counters + C_BYTES_PARITY, v);
  }
  for (int i = 0; i < C_WARP_NUM; ++i) {
    unsigned long long v = cnt.v[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(P.counters + i, v);
  }
}

// The any-vertex completeness mode: after the intersection join, each
// candidate not found intersecting is tested vertex by vertex, both ways
// (one warp per candidate, warp-cooperative parity rays).
template <int W>
__global__ void __launch_bounds__(128, 4) k_any_vertex(RefineArgs P) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpMem sm = carve<W>(smem + (size_t)wib * warp_smem_bytes<W>(P.stack_cap), P.stack_cap);
  Cnt cnt;
  for (int i = 0; i < C_WARP_NUM; ++i) cnt.v[i] = 0;
  const int64_t n = *P.n_cand;
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  for (;;) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(P.work, 1ull);
    const long long c = (long long)__shfl_sync(FULL, w, 0);
    if (c >= n) break;
    int done = lane == 0 ? (int)P.flags[c] : 0;
    if (__shfl_sync(FULL, done, 0)) continue;
    const int ia = P.cand[2 * c], ib = P.cand[2 * c + 1];
    if (ia < 0 || ia >= P.MA || ib < 0 || ib >= P.MB) continue;
    F3 off = zero;
    if (P.cand_off)
      off = mkf3((float)P.cand_off[3 * c], (float)P.cand_off[3 * c + 1], (float)P.cand_off[3 * c + 2]);
    int r = pair_any_inside<W>(P.B, ib, off, P.A, ia, zero, sm, lane, P.stack_cap, P.max_pop, cnt);
    if (r == 0)
      r = pair_any_inside<W>(P.A, ia, zero, P.B, ib, off, sm, lane, P.stack_cap, P.max_pop, cnt);
    if (r < 0 && lane == 0) atomicCAS(P.err, 0, DERR_STACK);
    if (r > 0 && lane == 0) P.flags[c] = 1;
  }
  for (int i = 0; i < C_WARP_NUM; ++i) {
    unsigned long long v = cnt.v[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(P.counters + i, v);
  }
}

// contains / within: a candidate is reported when its parity test holds and
// no crossing was found (Alg. 2): flags = pflags AND NOT flags
__global__ void k_pred_combine(uint8_t *flags, const uint8_t *pflags, const int64_t *n_dev) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (uint8_t)(pflags[i] != 0 && flags[i] == 0);
}

// ---------------------------------------------------------------------------
// Streaming refinement.  A persistent kernel whose warps each keep a task
// stack and a leaf-pair queue in shared memory holding the tasks of many
// candidate pairs at once, so that every traversal round is wide: an expand
// round copies the nodes of 16 (node, node) tasks (8 at W = 8) to shared
// memory with asynchronous copies issued all at once and tests their child
// pairs with 2 lanes per task (4 at W = 8); a leaf round does the same with
// the triangles of up to 24 leaf pairs (48 / L), filters (edge, triangle)
// tests by boxes and runs the exact tests that remain one per lane.  A round
// thus waits for one memory latency however many fetches it makes.  A warp
// takes 32 new candidates whenever its stack holds less than one round.
//
// Load balance.  A few pairs (a nucleus lying along a vessel wall over a
// large area) cost thousands of times the mean, and a warp that holds one
// would finish long after the others.  So the warps share a device task
// queue: a warp with no input and no tasks left becomes hungry and claims
// tasks from the queue; a straggler -- a warp that has not been able to take
// new work for `give_after` SM cycles, while most warps take some every few
// rounds -- that sees hungry warps gives the older half of its stack (the
// larger subtrees) to the queue, and so does a warp whose stack is nearly
// full.  A costly pair thus spreads over more and more warps.  At most
// `hungry_max` warps wait for tasks (a warp that finds that many waiting
// leaves): a heavy pair needs tens of helpers, not thousands of warps
// polling the same words.  A crossing sets the candidate's flag; the tasks
// of a flagged candidate are dropped when popped or claimed.
//
// Queue protocol.  Entries are uint4 (candidate, item A, item B, ready).  A
// producer reserves slots with an atomic add on `tail`, writes the first
// three words, fences, sets ready = 1, fences, and adds the count to
// `avail` (entries published, not yet claimed).  A consumer takes k of them
// by an atomic subtract on `avail` (undone if fewer than k were left), then
// an atomic add on `head` gives it k slot positions; every reserved slot is
// written without waiting on anything, so it waits for ready on each (a
// bounded wait), reads the slot through L2 and sets ready back to 0: the
// queue is all-zero again when the launch ends.  `active` counts the warps
// that hold work.  A waiting warp leaves once `active` is 0 and nothing is
// published, and a warp over the waiting cap leaves at once if nothing is
// published.  No warp leaves while published entries wait (a consumer whose
// subtract failed stays to retry), so whatever was pushed is taken by a
// warp that is still there, if need be by its producer: leaving early costs
// helpers, never work.  Every wait is bounded: on expiry the kernel records
// an error and the host redoes the join by plain depth-first traversal.
// ---------------------------------------------------------------------------
// 16-byte asynchronous copy global -> shared (bypassing L1), and the wait
// for all of this thread's copies
__device__ __forceinline__ void cp_async16(float4 *dst, const float4 *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// a staged triangle record (three float4, as in the BVH's triangle records)
__device__ __forceinline__ void stage_tri(const float4 *stage, int i, F3 off, F3 &a, F3 &b,
                                          F3 &c, int &own) {
  const float4 r0 = stage[3 * i], r1 = stage[3 * i + 1], r2 = stage[3 * i + 2];
  a = add(mkf3(r0.x, r0.y, r0.z), off);
  b = add(mkf3(r0.w, r1.x, r1.y), off);
  c = add(mkf3(r1.z, r1.w, r2.x), off);
  own = __float_as_int(r2.y);
}

// Leaf rounds stage the triangles of up to kLeafPairs leaf pairs (at most
// 48 / L) in shared memory: kStageF4 float4 = 4.5 KB per warp, which also
// holds an expand round's nodes (16 or 8 tasks x 2 nodes x W slots, padded).
constexpr int kLeafPairs = 24;
constexpr int kStageF4 = 288;
constexpr int kListMax = 384;  // queued (edge, triangle) tests: 32 units x 3 edges x 4 tests

template <int W>
struct StreamCfg {
  static constexpr int NT = W == 2 ? 16 : 64 / W;                  // tasks per expand round
  // staged node region of one (task, side): W slots of two float4 plus one
  // float4 of padding, so that regions start on different shared-memory banks
  static constexpr int RS = 2 * W + 1;
  static_assert(NT * 2 * RS <= kStageF4, "an expand round's nodes must fit the stage");
  static constexpr int SC = W == 8 ? 384 : 192;                    // stack entries
  static constexpr int LQ = 64;                                    // leaf-pair entries
  // per warp: stack, leaf queue (uint4 entries), triangle stage, boxes of
  // the staged triangles and of the leaves, pair offsets, pair entries, hit
  // words, test list
  static constexpr int warp_bytes = (SC + LQ) * 16 + kStageF4 * 16 + kStageF4 / 3 * 6 * 4 +
                                    kLeafPairs * 2 * 6 * 4 + kLeafPairs * 3 * 4 +
                                    kLeafPairs * 16 + kLeafPairs * 4 + kLeafPairs * 4 +
                                    kListMax * 2;
};

// control words of one launch (zeroed before it), each on its own 128-byte
// line: ctl[k * SQ_STRIDE]
enum { SQ_INTAKE = 0, SQ_TAIL, SQ_HEAD, SQ_AVAIL, SQ_ACTIVE, SQ_HUNGRY, SQ_NUM };
constexpr int SQ_STRIDE = 32;
constexpr int SQ_WORDS = SQ_NUM * SQ_STRIDE;

struct StreamArgs {
  WaveArgs w;               // meshes, candidates, flags, counters, error word
  unsigned int *ctl;        // SQ_* words
  uint4 *dq;                // shared task queue (all-zero between launches)
  int2 *cbase;              // per candidate: first triangle of each mesh
  unsigned int dq_cap;
  unsigned int spin_limit;  // bound on the polls of every wait (each sleeps <= 1 us)
  unsigned int hungry_max;  // warps that may wait for queued tasks
  long long give_after;     // SM cycles without new work that make a straggler
  // parity rays over the per-thread node budget (w.q_par, w.q_par_n): one
  // warp each, claimed at this position before the warp's first intake
  unsigned int *q_par_pos;
  int par_stack_cap;        // the rays' traversal stack, in the warp's own memory
};

// the launch's control word k
__device__ __forceinline__ unsigned *sq(const StreamArgs &P, int k) {
  return P.ctl + k * SQ_STRIDE;
}

template <int W>
__host__ __device__ constexpr int stream_warp_bytes() { return StreamCfg<W>::warp_bytes; }

// release store / acquire load at device scope: a queue slot's ready word
// publishes the entry its lane wrote before it, without a full fence
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_vol(const unsigned *p) {
  return *reinterpret_cast<volatile const unsigned *>(p);
}

// A queue entry's ready word: 1 for a traversal task (candidate, item A,
// item B); kLeafEntry | the leaf-queue counts word for a leaf pair
// (candidate, first triangle of A's leaf, first triangle of B's leaf).
constexpr unsigned kLeafEntry = 0x80000000u;

// queue entries a waiting warp claims at least (while there are as many)
constexpr int kClaimMin = 4;

// give src[0, n) to the queue (all lanes; n > 0), tasks or (leaves) leaf
// pairs; false if it is full
__device__ __forceinline__ bool queue_push(const StreamArgs &P, const uint4 *src, int n,
                                           int lane, bool leaves) {
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(sq(P, SQ_TAIL), (unsigned)n);
  base = __shfl_sync(FULL, base, 0);
  if ((uint64_t)base + (uint64_t)n > (uint64_t)P.dq_cap) return false;
  for (int k = lane; k < n; k += 32) {
    const uint4 v = src[k];
    uint4 *d = P.dq + base + k;
    d->x = v.x;
    d->y = v.y;
    d->z = v.z;
  }
  // each lane publishes the slots it wrote (a release store orders that
  // lane's entry before its ready word); no fence is needed before the
  // count either: a consumer waits for each slot's ready word, which may
  // become visible after the count
  for (int k = lane; k < n; k += 32)
    st_release(&P.dq[base + k].w, leaves ? (kLeafEntry | src[k].w) : 1u);
  __syncwarp();
  if (lane == 0) atomicAdd(reinterpret_cast<int *>(sq(P, SQ_AVAIL)), n);
  return true;
}

// drop stk[0, n) by moving stk[n, sp) down (all lanes)
__device__ __forceinline__ void stack_drop_bottom(uint4 *stk, int n, int sp, int lane) {
  __syncwarp();
  for (int k0 = 0; k0 < sp - n; k0 += 32) {
    const int k = k0 + lane;
    const uint4 v = k < sp - n ? stk[n + k] : make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    if (k < sp - n) stk[k] = v;
    __syncwarp();
  }
}


template <int W, bool EXACT>
__global__ void __launch_bounds__(128, 4) k_stream(StreamArgs P) {
  pdl_wait();
  pdl_trigger();
  using Cf = StreamCfg<W>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint4 *stk = reinterpret_cast<uint4 *>(smem + (size_t)wib * Cf::warp_bytes);
  uint4 *lq = stk + Cf::SC;
  float4 *stage = reinterpret_cast<float4 *>(lq + Cf::LQ);
  float *s_tbox = reinterpret_cast<float *>(stage + kStageF4);  // per staged triangle
  float *s_box = s_tbox + kStageF4 / 3 * 6;                       // per leaf
  float *s_off = s_box + kLeafPairs * 2 * 6;
  uint4 *s_pe = reinterpret_cast<uint4 *>(s_off + kLeafPairs * 3);
  volatile unsigned *s_hit = reinterpret_cast<volatile unsigned *>(s_pe + kLeafPairs);
  float *s_err = reinterpret_cast<float *>(const_cast<unsigned *>(s_hit) + kLeafPairs);
  unsigned short *s_list = reinterpret_cast<unsigned short *>(s_err + kLeafPairs);
  const WaveArgs &Q = P.w;
  const unsigned lt = (1u << lane) - 1u;
  const int lsh = Q.lshift;
  const int L = 1 << lsh;                         // leaf size
  const int pmax = min(kLeafPairs, 48 / L);       // leaf pairs per round (<= 32)
  const int upi = L == 8 ? 16 : 32;               // leaf units per filter iteration
  const F3 zero = mkf3(0.f, 0.f, 0.f);
  volatile const uint8_t *vflags = Q.flags;
  const int64_t n_in = *Q.n_cand;
  if (blockIdx.x == 0 && threadIdx.x == 0 && n_in > 0)
    atomicAdd(Q.counters + C_PAIRS, (unsigned long long)n_in);
  // counters: node pairs, box tests, tasks claimed from / given to the queue
  unsigned c_np = 0, c_bt = 0, c_res = 0, c_sp = 0;
  unsigned c_bx = 0;  // node bytes
  LeafCnt lc;
  int sp = 0, nlq = 0;
  bool more = true;   // candidates may be left
  long long t_new = clock64();  // when this warp last took (or tried to take) work
  int err = DERR_NONE;
  unsigned iters = 0;
  // Every 4th iteration lane 0 reads the intake position (a warp busy with a
  // costly pair takes no input and would not notice that it has run out) or,
  // once it has, the hungry count; the next iteration uses the value, so the
  // load overlaps one round of work.
  unsigned peek = 0;
  bool peeked = false, peek_more = false;
  bool registered = true;  // counted in SQ_ACTIVE
  if (lane == 0) atomicAdd(sq(P, SQ_ACTIVE), 1u);

  // The parity rays the per-thread kernel handed over: the longest rays,
  // taken first, one warp each, so that they overlap the crossing traversal
  // instead of forming a launch of their own.  The warp's stack, leaf queue
  // and stage are still empty here; the ray traversal borrows them.
  if (Q.q_par && Q.q_par_n && P.q_par_pos) {
    const unsigned npar = min(*Q.q_par_n, Q.q_par_cap);
    if (npar > 0) {
      constexpr int extra = Cfg<W>::extra_bytes;
      const int cap = min(P.par_stack_cap, (Cf::warp_bytes - extra) / 8 - 1);
      WarpMem pm = carve<W>(reinterpret_cast<unsigned char *>(stk), cap);
      Cnt pc;
      for (int i = 0; i < C_WARP_NUM; ++i) pc.v[i] = 0;
      for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(P.q_par_pos, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= npar) break;
        const uint4 e = Q.q_par[t];
        const uint32_t c = e.x;
        volatile uint8_t *flag = (Q.pflags ? Q.pflags : Q.flags) + c;
        const int done = lane == 0 ? (int)*flag : 0;
        if (__shfl_sync(FULL, done, 0)) continue;
        const int ia = Q.cand[2 * (int64_t)c], ib = Q.cand[2 * (int64_t)c + 1];
        const F3 off = cand_offset(Q, c);
        // direction 0: B's representative vertex against A; 1: A's against B
        const int r = e.z == 0u
            ? pair_inside<W>(Q.B, ib, off, Q.A, ia, zero, pm, lane, cap, 32, pc)
            : pair_inside<W>(Q.A, ia, zero, Q.B, ib, off, pm, lane, cap, 32, pc);
        if (r == 1) {
          if (lane == 0) *flag = 1;
        } else if (r < 0) {
          if (lane == 0) atomicCAS(Q.err, 0, DERR_STACK);  // the join is redone safely
          break;
        }
      }
      // their bytes count as parity bytes and as this launch's per-warp
      // passes (the bytes_tasks counter)
      const int ps[6] = {C_PARITY_RAYS, C_PARITY_NODES, C_PARITY_TRIS, C_BYTES, C_BYTES_PARITY,
                         C_BYTES_TASKS};
      const unsigned long long pv[6] = {pc.v[C_PARITY_RAYS], pc.v[C_PARITY_NODES],
                                        pc.v[C_PARITY_TRIS], pc.v[C_BYTES], pc.v[C_BYTES],
                                        pc.v[C_BYTES]};
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        unsigned long long v = pv[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0 && v) atomicAdd(Q.counters + ps[i], v);
      }
      __syncwarp();
    }
  }

  // one leaf round: the triangles of up to np leaf pairs from the top of the
  // queue are copied to shared memory (cp.async, all at once), each leaf's
  // box is taken from its triangles, every owned edge's box is tested against
  // the other leaf's box and its triangles' boxes, and the surviving (edge,
  // triangle) tests run one per lane.
  auto leaf_round = [&]() {
    const int np = min(nlq, pmax);
    uint4 pe = make_uint4(0u, 0u, 0u, 0u);
    if (lane < np) {
      pe = lq[nlq - 1 - lane];
      s_pe[lane] = pe;
    }
    __syncwarp();
    nlq -= np;
    // the pair's flag and offset load while the triangles are copied (a
    // pair found intersecting meanwhile is copied for nothing)
    uint8_t pfl = 1;
    F3 po = zero;
    if (lane < np) {
      pfl = vflags[pe.x];
      po = cand_offset(Q, pe.x);
    }
    // stage: the triangle records of each (pair p, side), contiguous in the
    // mesh, go to float4 ((p * 2 + side) * L + t) * 3 + k.  A (pair, side)
    // owns 4 L lanes of an iteration (at least its 3 L float4): lane h of
    // them copies float4 h, so that the lanes of one run read consecutive
    // addresses (one coalesced request per run instead of a lane copying it
    // piece by piece).
    {
      const int chs = lsh + 2, h = lane & ((1 << chs) - 1);
      for (int ps = lane >> chs; ps < 2 * np; ps += 32 >> chs) {
        const int side = ps & 1;
        const uint4 e = s_pe[ps >> 1];
        const int n3 = 3 * ((int)((side ? e.w >> 8 : e.w) & 7u) + 1);
        if (h < n3)
          cp_async16(stage + 3 * (ps << lsh) + h,
                     (side ? Q.B.trirec : Q.A.trirec) + 3 * (int64_t)(side ? e.z : e.y) + h);
      }
    }
    if (lane < np) {
      const bool alive = pfl == 0;
      s_hit[lane] = alive ? 0u : 1u;
      s_off[3 * lane] = po.x;
      s_off[3 * lane + 1] = po.y;
      s_off[3 * lane + 2] = po.z;
      if (alive) {
        lc.lp += 1;
        lc.bytes += 48u * ((pe.w & 7u) + ((pe.w >> 8) & 7u) + 2u);
      }
    }
    cp_async_wait_all();
    __syncwarp();
    // one lane per (pair, side): the boxes of the leaf's staged triangles
    // (B's translated by the pair's offset) and the leaf's box; the two sides
    // of a pair sit on adjacent lanes, which combine their leaf boxes into the
    // pair's static filter bound (from the box around both leaves)
    for (int ps0 = 0; ps0 < 2 * np; ps0 += 32) {
      const int ps = ps0 + lane, p = ps >> 1, side = ps & 1;
      float bx[6] = {3.4e38f, 3.4e38f, 3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
      const bool on = ps < 2 * np && !s_hit[p];  // the same for both sides
      if (on) {
        const uint4 e = s_pe[p];
        const int n = (int)((side ? e.w >> 8 : e.w) & 7u) + 1;
        const F3 o = side ? mkf3(s_off[3 * p], s_off[3 * p + 1], s_off[3 * p + 2]) : zero;
        for (int t = 0; t < n; ++t) {
          const int i = (ps << lsh) + t;
          F3 a, b, c;
          int own;
          stage_tri(stage, i, o, a, b, c, own);
          const float lx = fminf(a.x, fminf(b.x, c.x)), ly = fminf(a.y, fminf(b.y, c.y));
          const float lz = fminf(a.z, fminf(b.z, c.z)), hx = fmaxf(a.x, fmaxf(b.x, c.x));
          const float hy = fmaxf(a.y, fmaxf(b.y, c.y)), hz = fmaxf(a.z, fmaxf(b.z, c.z));
          float *bp = s_tbox + 6 * i;
          bp[0] = lx;
          bp[1] = ly;
          bp[2] = lz;
          bp[3] = hx;
          bp[4] = hy;
          bp[5] = hz;
          bx[0] = fminf(bx[0], lx);
          bx[1] = fminf(bx[1], ly);
          bx[2] = fminf(bx[2], lz);
          bx[3] = fmaxf(bx[3], hx);
          bx[4] = fmaxf(bx[4], hy);
          bx[5] = fmaxf(bx[5], hz);
        }
        float *bp = s_box + 6 * ps;
#pragma unroll
        for (int q = 0; q < 6; ++q) bp[q] = bx[q];
      }
      float ob[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) ob[q] = __shfl_xor_sync(FULL, bx[q], 1);
      if (on && side == 0) {
        const float D = fmaxf(fmaxf(fmaxf(bx[3], ob[3]) - fminf(bx[0], ob[0]),
                                    fmaxf(bx[4], ob[4]) - fminf(bx[1], ob[1])),
                              fmaxf(bx[5], ob[5]) - fminf(bx[2], ob[2]));
        s_err[p] = static_err(D);
      }
    }
    __syncwarp();
    // the queued (edge, triangle) tests, one per lane: code = p | dir << 5 |
    // s << 6 | k << 9 | t << 11
    int nlist = 0;
    auto flush = [&]() {
      for (int i0 = 0; i0 < nlist; i0 += 32) {
        const int i = i0 + lane;
        if (i < nlist) {
          const unsigned code = s_list[i];
          const int p = code & 31, dir = (code >> 5) & 1, si = (code >> 6) & 7;
          const int k = (code >> 9) & 3, t = (code >> 11) & 7;
          // every shared-memory read of the test is issued at once, before
          // the pair's hit word decides whether to run it
          const F3 o = mkf3(s_off[3 * p], s_off[3 * p + 1], s_off[3 * p + 2]);
          F3 v0, v1, v2, a, b, c;
          int own, town;
          stage_tri(stage, (p * 2 + dir) * L + si, dir ? o : zero, v0, v1, v2, own);
          stage_tri(stage, (p * 2 + (dir ^ 1)) * L + t, dir ? zero : o, a, b, c, town);
          const float err_p = s_err[p];
          if (!s_hit[p]) {
            const F3 pp = k == 0 ? v0 : (k == 1 ? v1 : v2);
            const F3 qq = k == 0 ? v1 : (k == 1 ? v2 : v0);
            lc.st += 1;
            bool r;
            if (EXACT) {
              r = segtri_exact_staged(pp, qq, a, b, c);
            } else {
              bool ex = false;
              r = segtri_static(pp, qq, a, b, c, err_p, &ex);
              lc.fb += ex ? 1 : 0;
            }
            if (r) {
              s_hit[p] = 1u;
              Q.flags[s_pe[p].x] = 1;
            }
          }
        }
        __syncwarp();
      }
      nlist = 0;
    };
    // units (p, dir, source triangle): the source's owned edges against the
    // target leaf
    const int nu = np * 2 * L;
    for (int u0 = 0; u0 < nu; u0 += upi) {
      const int u = lane < upi ? u0 + lane : nu;
      unsigned mask = 0;  // bit k * L + t: edge k against target triangle t
      int p = 0, dir = 0, si = 0;
      if (u < nu) {
        si = u & (L - 1);
        const int pd = u >> lsh;
        dir = pd & 1;
        p = pd >> 1;
        const uint4 e = s_pe[p];
        const int ns = (int)((dir ? e.w >> 8 : e.w) & 7u) + 1;
        const int nt = (int)((dir ? e.w : e.w >> 8) & 7u) + 1;
        if (!s_hit[p] && si < ns) {
          const F3 o = mkf3(s_off[3 * p], s_off[3 * p + 1], s_off[3 * p + 2]);
          F3 v[3];
          int own;
          stage_tri(stage, (p * 2 + dir) * L + si, dir ? o : zero, v[0], v[1], v[2], own);
          const float *bp = s_box + 6 * (p * 2 + (dir ^ 1));
          const F3 tlo = mkf3(bp[0], bp[1], bp[2]), thi = mkf3(bp[3], bp[4], bp[5]);
          const float *tbx = s_tbox + 6 * ((p * 2 + (dir ^ 1)) * L);
          // box filters only (no slab test: its reciprocals cost more here
          // than the exact tests it would save, which run one per lane)
          // each owned edge's box against the leaf's (bit k of ek), then
          // against each target triangle's box, read once for all edges
          F3 elo[3], ehi[3];
          unsigned ek = 0;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const F3 pp = v[k], qq = v[k == 2 ? 0 : k + 1];
            elo[k] = mkf3(fminf(pp.x, qq.x), fminf(pp.y, qq.y), fminf(pp.z, qq.z));
            ehi[k] = mkf3(fmaxf(pp.x, qq.x), fmaxf(pp.y, qq.y), fmaxf(pp.z, qq.z));
            if (!((own >> k) & 1)) continue;
            lc.slab += 1;
            if (!(elo[k].x >= thi.x || tlo.x >= ehi[k].x || elo[k].y >= thi.y ||
                  tlo.y >= ehi[k].y || elo[k].z >= thi.z || tlo.z >= ehi[k].z))
              ek |= 1u << k;  // open overlap (exact for crossings, see overlap_open)
          }
          for (int t = 0; ek && t < nt; ++t) {
            const float *tp = tbx + 6 * t;
            const float t0 = tp[0], t1 = tp[1], t2 = tp[2], t3 = tp[3], t4 = tp[4], t5 = tp[5];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              if (((ek >> k) & 1) && !(t0 >= ehi[k].x || elo[k].x >= t3 || t1 >= ehi[k].y ||
                                       elo[k].y >= t4 || t2 >= ehi[k].z || elo[k].z >= t5))
                mask |= 1u << (k * L + t);
            }
          }
        }
      }
      // append this lane's tests (at most 3 L), flushing first if they would
      // not fit
      const int cnt = __popc(mask);
      const int incl = warp_scan_incl(cnt, lane);
      const int tot = __shfl_sync(FULL, incl, 31);
      if (nlist + tot > kListMax) flush();
      int pos = nlist + incl - cnt;
      while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        const int k = b >> lsh, t = b & (L - 1);
        s_list[pos++] = (unsigned short)(p | (dir << 5) | (si << 6) | (k << 9) | (t << 11));
      }
      nlist += tot;
      __syncwarp();
    }
    flush();
  };

  // take the k claimed queue entries at position h (their producers may
  // still be writing them): tasks onto the stack, leaf pairs onto the leaf
  // queue, those of candidates found intersecting dropped; false if a
  // bounded wait ran out (k <= 32; the caller checked the room)
  auto take = [&](int64_t h, int k) -> bool {
    bool tpush = false, lpush = false, late = false;
    uint4 ent = make_uint4(0u, 0u, 0u, 0u);
    if (lane < k) {
      unsigned *rdy = &P.dq[h + lane].w;
      unsigned it = 0;
      unsigned w = 0;
      while ((w = ld_acquire(rdy)) == 0u) {  // acquire: the entry is visible after it
        if (++it >= P.spin_limit) {
          late = true;
          break;
        }
        __nanosleep(64);
      }
      if (!late) {
        ent = __ldcg(P.dq + h + lane);
        *reinterpret_cast<volatile unsigned *>(rdy) = 0u;
        const bool alive = vflags[ent.x] == 0;
        lpush = alive && (w & kLeafEntry);
        tpush = alive && !(w & kLeafEntry);
        ent.w = lpush ? (w & ~kLeafEntry) : 0u;
      }
    }
    if (__any_sync(FULL, late)) return false;
    c_res += lane == 0 ? (unsigned)k : 0u;
    const unsigned mt = __ballot_sync(FULL, tpush), ml = __ballot_sync(FULL, lpush);
    if (tpush) stk[sp + __popc(mt & lt)] = ent;
    if (lpush) lq[nlq + __popc(ml & lt)] = ent;
    sp += __popc(mt);
    nlq += __popc(ml);
    __syncwarp();
    return true;
  };

  // give the older half of the stack to the queue
  auto give_half = [&](int n) -> bool {
    if (!queue_push(P, stk, n, lane, false)) return false;
    c_sp += lane == 0 ? (unsigned)n : 0u;
    stack_drop_bottom(stk, n, sp, lane);
    sp -= n;
    return true;
  };
  // give the older leaf pairs of the leaf queue: leaf rounds are the costly
  // part of a heavy candidate, so its leaf pairs spread like its tasks
  auto give_leaves = [&](int n) -> bool {
    if (!queue_push(P, lq, n, lane, true)) return false;
    c_sp += lane == 0 ? (unsigned)n : 0u;
    stack_drop_bottom(lq, n, nlq, lane);
    nlq -= n;
    return true;
  };

  for (;;) {
    if (++iters > (1u << 24)) {  // defensive bound: a warp needs ~10^3 rounds at most here
      err = DERR_STACK;
      break;
    }
    bool give = false;
    if (peeked) {
      peeked = false;
      const unsigned v = __shfl_sync(FULL, peek, 0);
      if (peek_more) {
        if ((int64_t)v >= n_in) more = false;
      } else {
        give = v > 0 && __shfl_sync(FULL, (int)(clock64() - t_new > P.give_after), 0);
      }
    }
    if ((iters & 3u) == 0) {
      if (lane == 0) peek = ld_vol(sq(P, more ? SQ_INTAKE : SQ_HUNGRY));
      peeked = true;
      peek_more = more;
    }
    // 1. intake, while the stack holds less than one round
    if (more && sp < Cf::NT && nlq < pmax) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(sq(P, SQ_INTAKE), 32u);
      base = __shfl_sync(FULL, base, 0);
      t_new = clock64();
      if ((int64_t)base >= n_in) {
        more = false;
        continue;
      }
      const int64_t idx = (int64_t)base + lane;
      bool push = false;
      uint4 ent = make_uint4(0u, 0u, 0u, 0u);
      if (idx < n_in && vflags[idx] == 0 && (!Q.need || Q.need[idx])) {
        const int ia = Q.cand[2 * idx], ib = Q.cand[2 * idx + 1];
        if (ia >= 0 && ia < Q.MA && ib >= 0 && ib < Q.MB) {
          const F3 off = cand_offset(Q, idx);
          Box ba, bb;
          const float4 a0 = Q.A.mrec[3 * (int64_t)ia], a1 = Q.A.mrec[3 * (int64_t)ia + 1];
          const float4 b0 = Q.B.mrec[3 * (int64_t)ib], b1 = Q.B.mrec[3 * (int64_t)ib + 1];
          const float ta = Q.A.mrec[3 * (int64_t)ia + 2].y, tbs = Q.B.mrec[3 * (int64_t)ib + 2].y;
          const uint32_t ra = (uint32_t)Q.A.roots[ia], rb = (uint32_t)Q.B.roots[ib];
          ba.lo = mkf3(a0.x, a0.y, a0.z);
          ba.hi = mkf3(a1.x, a1.y, a1.z);
          bb.lo = add(mkf3(b0.x, b0.y, b0.z), off);
          bb.hi = add(mkf3(b1.x, b1.y, b1.z), off);
          if (overlap_open(ba, bb)) {  // crossings only (parity runs apart)
            const uint2 t = make_task(ra, ba, rb, bb);
            ent = make_uint4((uint32_t)idx, t.x, t.y, 0u);
            P.cbase[idx] = make_int2(__float_as_int(ta), __float_as_int(tbs));
            push = true;
          }
        }
      }
      // room: sp < NT <= 32 and 32 more stay below SC
      const unsigned m = __ballot_sync(FULL, push);
      if (push) stk[sp + __popc(m & lt)] = ent;
      sp += __popc(m);
      __syncwarp();
      continue;
    }
    // 2. out of work: claim tasks from the queue, or leave
    if (sp == 0 && nlq == 0) {
      if (more) continue;
      int64_t h = -1;
      int k = 0;
      if (lane == 0) {
        __threadfence();  // this warp's pushes before it stops counting as active
        atomicSub(sq(P, SQ_ACTIVE), 1u);
        // over the cap a warp may leave only while nothing is published:
        // entries it pushed itself might otherwise outlive every waiting warp
        int *avail = reinterpret_cast<int *>(sq(P, SQ_AVAIL));
        bool wait = atomicAdd(sq(P, SQ_HUNGRY), 1u) < P.hungry_max;
        if (!wait) wait = (int)ld_acquire(reinterpret_cast<const unsigned *>(avail)) > 0;
        unsigned nap = 128;
        for (unsigned it = 0; wait; ++it) {
          if (it >= P.spin_limit) {
            err = DERR_TIMEOUT;
            break;
          }
          if (ld_vol(reinterpret_cast<const unsigned *>(Q.err)) != 0u) break;  // failing
          const int av = *reinterpret_cast<volatile int *>(avail);
          if (av > 0) {
            // a share of what is published: the entries split over the
            // waiting warps, at least kClaimMin and at most NT of them
            // (claiming up to NT, or 2 NT, regardless left most waiting
            // warps without work in the tail)
            const unsigned hg = max(1u, ld_vol(sq(P, SQ_HUNGRY)));
            const int want = min(min(av, Cf::NT),
                                 max(kClaimMin, (int)(((unsigned)av + hg - 1u) / hg)));
            if (atomicSub(avail, want) >= want) {
              h = atomicAdd(sq(P, SQ_HEAD), (unsigned)want);
              atomicAdd(sq(P, SQ_ACTIVE), 1u);
              k = want;
              break;
            }
            atomicAdd(avail, want);  // fewer were left: undo, retry
            nap = 64;
          } else if (ld_acquire(sq(P, SQ_ACTIVE)) == 0u) {
            // a producer fences its pushes before it stops counting as
            // active, so with no warp active an acquire read of the count
            // sees everything published
            if ((int)ld_acquire(reinterpret_cast<const unsigned *>(avail)) <= 0) break;  // leave
          }
          __nanosleep(nap);
          nap = min(nap * 2, 1024u);
        }
        atomicSub(sq(P, SQ_HUNGRY), 1u);
      }
      err = __shfl_sync(FULL, err, 0);
      h = __shfl_sync(FULL, h, 0);
      k = __shfl_sync(FULL, k, 0);
      registered = h >= 0;
      if (h < 0) break;
      t_new = clock64();
      sp = 0;
      nlq = 0;
      if (!take(h, k)) {
        err = DERR_TIMEOUT;
        break;
      }
      continue;
    }
    // 3. a straggler and hungry warps: give the older half of the stack
    // (from NT / 2 entries: the costliest candidates end in rounds of fewer
    // than NT tasks, 0.257 against 0.265 ms) and of the leaf queue
    if (give && sp >= Cf::NT / 2) {
      if (!give_half(sp / 2)) {
        err = DERR_QUEUE;
        break;
      }
    }
    if (give && nlq >= pmax) {
      if (!give_leaves(nlq / 2)) {
        err = DERR_QUEUE;
        break;
      }
    }
    // 4. leaf pairs once a round's worth is queued (or nothing else is left)
    if (nlq >= pmax || sp == 0) {
      leaf_round();
      continue;
    }
    // 5. expand round: up to NT tasks; their nodes are copied to shared
    // memory (cp.async, all at once), then 32 / NT lanes per task test its
    // child pairs.  Leaf pairs that do not fit in the leaf queue go on the
    // stack as (leaf, leaf) tasks.
    constexpr int NT = Cf::NT;          // tasks per round
    constexpr int LPT = 32 / NT;        // lanes per task
    static_assert(W * W / LPT <= 32, "a lane's child pairs must fit one mask word");
    int npop = min(NT, sp);
    while (npop > 0 && sp - npop + npop * W * W > Cf::SC) --npop;
    if (npop == 0) {
      // the stack is nearly full: its older half goes to the queue
      if (!give_half(Cf::SC / 2)) {
        err = DERR_QUEUE;
        break;
      }
      continue;
    }
    const int ti = lane / LPT, gi = lane - ti * LPT;  // task of this lane, rank in it
    const bool act = ti < npop;
    const uint4 t = act ? stk[sp - 1 - ti] : make_uint4(0u, 0u, 0u, 0u);
    const bool xa = t.y & kExpand, xb = t.z & kExpand;
    // the candidate's flag, offset and first triangles are requested before
    // the node copies, so that they do not queue behind them
    const uint8_t fl = act ? vflags[t.x] : (uint8_t)1;
    const F3 off = act ? cand_offset(Q, t.x) : zero;
    const int2 cbv = act ? P.cbase[t.x] : make_int2(0, 0);  // for leaf pairs
    // stage: task i, side s, slot j (of W) at float4 index (i * 2 + s) * RS + 2 j;
    // one lane per (task, side) copies the W child slots of an expanding
    // node, or the one slot of the item's own box.  (Spreading a node's
    // pieces over consecutive lanes, so that each copy request is one
    // coalesced run, measured slower here: 0.281 against 0.265 ms on the
    // pathology step; the leaf triangles below do gain from it.)
    for (int is = lane; is < npop * 2; is += 32) {
      const int side = is & 1, i = is >> 1;
      const uint4 e = stk[sp - 1 - i];
      const uint32_t item = side ? e.z : e.y;
      const bool x = item & kExpand;
      const uint32_t idx = item & kIdx;
      int64_t word;  // float offset of the first slot in the node array
      if (x) word = (int64_t)idx * Cfg<W>::SW + 8;
      else if (item & kLeafBit) word = (int64_t)(idx / W) * Cfg<W>::SW + 8 * (idx % W + 1);
      else word = (int64_t)idx * Cfg<W>::SW;
      const float4 *src = reinterpret_cast<const float4 *>((side ? Q.B.nodes : Q.A.nodes) + word);
      float4 *dst = stage + is * Cf::RS;
      const int n = x ? 2 * W : 2;
      for (int h = 0; h < n; ++h) cp_async16(dst + h, src + h);
    }
    cp_async_wait_all();
    __syncwarp();
    sp -= npop;
    const bool live = act && fl == 0;
    if (live && gi == 0) {
      c_np += 1;
      c_bx += node_pair_bytes<W>(xa, xb);
    }
    // this lane's child pairs q = gi + k LPT, k < W * W / LPT <= 16, of the
    // NA x NB child slots (W for an expanding side, else 1): a = q / NB,
    // b = q % NB; bit k of the masks.  They are enumerated as (A slot ia,
    // B slot m) with k = ia * nbl + m, so that each box is read from shared
    // memory once: the lane's B slots are gi + m LPT (B expands) or the one
    // slot, its A slots all W (both expand), gi + ia LPT (only A expands) or
    // the one slot.
    constexpr int MB = (W + LPT - 1) / LPT;
    unsigned tmask = 0, lmask = 0;
    if (live && (xa || xb || gi == 0)) {
      const int nbl = xb ? MB : 1;
      const int nal = xa ? (xb ? W : MB) : 1;
      c_bt += (unsigned)(nal * nbl);
      Box bbx[MB];
      uint32_t bwd[MB];
#pragma unroll
      for (int m = 0; m < MB; ++m) {
        const int b = xb ? gi + m * LPT : 0;
        const float4 b0 = stage[(ti * 2 + 1) * Cf::RS + 2 * b];
        const float4 b1 = stage[(ti * 2 + 1) * Cf::RS + 2 * b + 1];
        bwd[m] = __float_as_uint(b1.z);
        bbx[m].lo = add(mkf3(b0.x, b0.y, b0.z), off);
        bbx[m].hi = add(mkf3(b0.w, b1.x, b1.y), off);
      }
      for (int ia = 0; ia < nal; ++ia) {
        const int a = xa ? (xb ? ia : gi + ia * LPT) : 0;
        const float4 a0 = stage[(ti * 2) * Cf::RS + 2 * a], a1 = stage[(ti * 2) * Cf::RS + 2 * a + 1];
        const uint32_t wa = __float_as_uint(a1.z);
        if (xa && wa == kEmpty) continue;
        Box ba;
        ba.lo = mkf3(a0.x, a0.y, a0.z);
        ba.hi = mkf3(a0.w, a1.x, a1.y);
        const bool la = xa ? (wa & kLeafBit) != 0 : (t.y & kLeafBit) != 0;
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          if (m >= nbl) break;
          if (xb && bwd[m] == kEmpty) continue;
          if (!overlap_open(ba, bbx[m])) continue;
          const bool lb = xb ? (bwd[m] & kLeafBit) != 0 : (t.z & kLeafBit) != 0;
          const int k = ia * nbl + m;
          if (la && lb) lmask |= 1u << k;
          else tmask |= 1u << k;
        }
      }
    }
    // positions of this lane's outputs (task and leaf counts packed)
    const unsigned mine = (unsigned)__popc(tmask) | ((unsigned)__popc(lmask) << 16);
    unsigned incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned tot = __shfl_sync(FULL, incl, 31);
    const unsigned ex = incl - mine;
    const int tt = (int)(tot & 0xFFFFu), tl = (int)(tot >> 16);
    const int room = Cf::LQ - nlq;  // leaf pairs past it go on the stack
    int tpos = sp + (int)(ex & 0xFFFFu), lr = (int)(ex >> 16);
    unsigned bits = tmask | lmask;
    while (bits) {
      const int k = __ffs(bits) - 1;
      bits &= bits - 1;
      const int q = gi + k * LPT;
      const int a = xb ? (int)((unsigned)q / W) : q, b = xb ? (int)((unsigned)q % W) : 0;
      const float4 a0 = stage[(ti * 2) * Cf::RS + 2 * a], a1 = stage[(ti * 2) * Cf::RS + 2 * a + 1];
      const float4 b0 = stage[(ti * 2 + 1) * Cf::RS + 2 * b];
      const float4 b1 = stage[(ti * 2 + 1) * Cf::RS + 2 * b + 1];
      const uint32_t wa = __float_as_uint(a1.z), wb = __float_as_uint(b1.z);
      // the child items: a leaf slot id or a node index (expanding side),
      // else the task's item itself
      const uint32_t na = xa ? ((wa & kLeafBit) ? (kLeafBit | ((t.y & kIdx) * W + a)) : wa)
                             : (t.y & ~kExpand);
      const uint32_t nb = xb ? ((wb & kLeafBit) ? (kLeafBit | ((t.z & kIdx) * W + b)) : wb)
                             : (t.z & ~kExpand);
      if ((tmask >> k) & 1u) {
        Box ba, bb;
        ba.lo = mkf3(a0.x, a0.y, a0.z);
        ba.hi = mkf3(a0.w, a1.x, a1.y);
        bb.lo = add(mkf3(b0.x, b0.y, b0.z), off);
        bb.hi = add(mkf3(b0.w, b1.x, b1.y), off);
        const uint2 nt = make_task(na, ba, nb, bb);
        stk[tpos++] = make_uint4(t.x, nt.x, nt.y, 0u);
      } else if (lr < room) {
        // leaf pair: absolute first triangles and counts (wa / wb are the
        // leaves' descriptors: for a side that does not expand, its slot's
        // child word)
        lq[nlq + lr] = make_uint4(t.x, (uint32_t)cbv.x + ((wa >> 3) & 0x0FFFFFFFu),
                                  (uint32_t)cbv.y + ((wb >> 3) & 0x0FFFFFFFu),
                                  (wa & 7u) | ((wb & 7u) << 8));
        ++lr;
      } else {
        stk[sp + tt + (lr - room)] = make_uint4(t.x, na, nb, 0u);
        ++lr;
      }
    }
    sp += tt + max(0, tl - room);
    nlq += min(tl, room);
    __syncwarp();
  }
  if (err != DERR_NONE && lane == 0) atomicCAS(Q.err, 0, err);
  // a warp that stops with an error still counted as active lets the others
  // go (they see the error word)
  if (registered && lane == 0) {
    __threadfence();
    atomicSub(sq(P, SQ_ACTIVE), 1u);
  }
  // counters: one atomic per warp and counter
  const unsigned long long cv[11] = {c_np, c_bt, lc.lp, lc.slab, lc.st, lc.fb,
                                     (unsigned long long)c_bx + lc.bytes, c_bx, lc.bytes,
                                     c_res, c_sp};
  const int slot[11] = {C_NODE_PAIRS, C_BOX_TESTS, C_LEAF_PAIRS, C_SLAB_TESTS, C_SEGTRI,
                        C_FALLBACK, C_BYTES, C_BYTES_EXPAND, C_BYTES_LEAF, C_TASKS, C_SPILLED};
#pragma unroll
  for (int i = 0; i < 11; ++i) {
    unsigned long long v = cv[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v) atomicAdd(Q.counters + slot[i], v);
  }
}

// ---------------------------------------------------------------------------
// Compaction: flags -> (idA, idB) in candidate order
// ---------------------------------------------------------------------------
constexpr int CMP_T = 256, CMP_PER = 16, CMP_CHUNK = CMP_T * CMP_PER;

__global__ void k_flag_count(const uint8_t *flags, const int64_t *n_dev, int64_t *bcount,
                             unsigned long long *hits) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = *n_dev;
  int64_t base = blockIdx.x * (int64_t)CMP_CHUNK;
  // the grid covers the candidate capacity; chunks past the count are empty
  if (base >= n) {
    if (threadIdx.x == 0) bcount[blockIdx.x] = 0;
    return;
  }
  int c = 0;
  for (int k = threadIdx.x; k < CMP_CHUNK; k += CMP_T) {
    int64_t i = base + k;
    if (i < n) c += flags[i] != 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
  __shared__ int ws[CMP_T / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < CMP_T / 32; ++w) s += ws[w];
    bcount[blockIdx.x] = s;
    if (hits && s) atomicAdd(hits, (unsigned long long)s);
  }
}

__global__ void k_flag_emit(const uint8_t *flags, const int64_t *n_dev, const int32_t *cand,
                            const int64_t *boff, int32_t *out) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = *n_dev;
  if (blockIdx.x * (int64_t)CMP_CHUNK >= n) return;  // an empty chunk (see k_flag_count)
  int64_t base = blockIdx.x * (int64_t)CMP_CHUNK + (int64_t)threadIdx.x * CMP_PER;
  int c = 0;
  uint8_t f[CMP_PER];
  for (int k = 0; k < CMP_PER; ++k) {
    int64_t i = base + k;
    f[k] = (i < n) ? flags[i] : 0;
    c += f[k] != 0;
  }
  // block exclusive scan of c
  __shared__ int ws[CMP_T / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = c;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int wbase = 0;
  for (int k = 0; k < w; ++k) wbase += ws[k];
  int64_t pos = boff[blockIdx.x] + wbase + inc - c;
  for (int k = 0; k < CMP_PER; ++k) {
    if (f[k]) {
      int64_t i = base + k;
      out[2 * pos] = cand[2 * i];
      out[2 * pos + 1] = cand[2 * i + 1];
      ++pos;
    }
  }
}

// ---------------------------------------------------------------------------
// Single-pass compaction and box join: output offsets by decoupled
// look-back (Merrill and Garland, "Single-pass Parallel Prefix Scan with
// Decoupled Look-back", 2016).  Tiles take ids from a ticket counter in the
// order blocks start them; a tile publishes its own count as soon as it has
// it (AGG) and its inclusive prefix once known (INC); it finds its exclusive
// prefix by summing its predecessors' words backwards, 32 at a time, down to
// the nearest inclusive prefix.  It only waits for tiles whose ids were
// taken before its own, by blocks that are running, so every wait ends; each
// is bounded all the same (on expiry the kernel records DERR_TIMEOUT and the
// host redoes the join with the multi-pass kernels).  The words and the
// ticket are zeroed before each launch.
// ---------------------------------------------------------------------------
constexpr unsigned long long LB_AGG = 1ull << 62, LB_INC = 2ull << 62,
                             LB_VAL = (1ull << 62) - 1;

__device__ __forceinline__ void lb_publish(unsigned long long *state, unsigned tile,
                                           unsigned long long word) {
  *reinterpret_cast<volatile unsigned long long *>(state + tile) = word;
}

// one warp (all lanes): the exclusive prefix of `tile`, or -1 if a bounded
// wait ran out
__device__ long long lb_exclusive(const unsigned long long *state, unsigned tile,
                                  unsigned spin_limit, int lane) {
  long long excl = 0;
  for (int64_t j0 = (int64_t)tile - 32;; j0 -= 32) {
    const int64_t j = j0 + lane;
    unsigned long long st = LB_INC;  // before tile 0: an inclusive prefix of 0
    bool late = false;
    if (j >= 0) {
      unsigned it = 0;
      while (((st = *reinterpret_cast<const volatile unsigned long long *>(state + j)) >> 62) ==
             0ull) {
        if (++it > spin_limit) {
          late = true;
          break;
        }
        __nanosleep(32);
      }
    }
    if (__any_sync(FULL, late)) return -1;
    const unsigned pm = __ballot_sync(FULL, (st >> 62) == 2ull);
    const int hp = pm ? 31 - __clz(pm) : 0;  // the nearest inclusive prefix
    long long v = lane >= hp ? (long long)(st & LB_VAL) : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    excl += v;
    if (pm) return excl;
  }
}

// flags -> (idA, idB) of the flagged candidates in candidate order, the pair
// count to *count and to the hit counter; one tile = CMP_CHUNK candidates
__global__ void __launch_bounds__(CMP_T) k_compact(const uint8_t *flags, const int64_t *n_dev,
                                                   const int32_t *cand, unsigned *ticket,
                                                   unsigned long long *state, int32_t *out,
                                                   int64_t *count, unsigned long long *hits,
                                                   int *err, unsigned spin_limit) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned s_tile;
  __shared__ int ws[CMP_T / 32];
  __shared__ long long s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const unsigned tile = s_tile;
  const int64_t n = *n_dev;
  const int64_t ntiles = (n + CMP_CHUNK - 1) / CMP_CHUNK;
  if ((int64_t)tile >= ntiles) {
    if (tile == 0 && threadIdx.x == 0) *count = 0;  // no candidates at all
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)tile * CMP_CHUNK + (int64_t)threadIdx.x * CMP_PER;
  // CMP_PER = 16 flags: one 16-byte load when the run is in range
  uint8_t f[CMP_PER];
  if (base + CMP_PER <= n) {
    const uint4 v = *reinterpret_cast<const uint4 *>(flags + base);
    const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < CMP_PER; ++k) f[k] = (uint8_t)(u[k >> 2] >> (8 * (k & 3)));
  } else {
#pragma unroll
    for (int k = 0; k < CMP_PER; ++k) f[k] = base + k < n ? flags[base + k] : 0;
  }
  int c = 0;
#pragma unroll
  for (int k = 0; k < CMP_PER; ++k) c += f[k] != 0;
  int inc = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int wbase = 0, agg = 0;
  for (int k = 0; k < CMP_T / 32; ++k) {
    wbase += k < w ? ws[k] : 0;
    agg += ws[k];
  }
  if (threadIdx.x == 0) lb_publish(state, tile, (tile == 0 ? LB_INC : LB_AGG) | (unsigned long long)agg);
  if (w == 0) {
    const long long e = tile == 0 ? 0 : lb_exclusive(state, tile, spin_limit, lane);
    if (lane == 0) {
      if (e < 0) {
        atomicCAS(err, 0, DERR_TIMEOUT);
      } else {
        if (tile > 0) lb_publish(state, tile, LB_INC | (unsigned long long)(e + agg));
        if ((int64_t)tile == ntiles - 1) *count = e + agg;
        if (hits && agg) atomicAdd(hits, (unsigned long long)agg);
      }
      s_excl = e;
    }
  }
  __syncthreads();
  if (s_excl < 0) return;
  int64_t pos = s_excl + wbase + inc - c;
#pragma unroll
  for (int k = 0; k < CMP_PER; ++k) {
    if (f[k]) {
      const int64_t i = base + k;
      out[2 * pos] = cand[2 * i];
      out[2 * pos + 1] = cand[2 * i + 1];
      ++pos;
    }
  }
}

// The bounding-box filter join in one launch: a tile is MBB_T / 32 A meshes
// (one warp each); its blocks count their candidates (the tests of k_mbb),
// take the tile's output offset by look-back, then test again and write.
// Persistent blocks take tiles from the ticket counter until none is left;
// the last tile writes the candidate count.
__global__ void __launch_bounds__(MBB_T, 5) k_mbb1(const float *aabbA, int64_t MA,
                                               const float *aabbB, int64_t MB, int self_join,
                                               unsigned *ticket, unsigned long long *state,
                                               int32_t *cand, int64_t *count, int *err,
                                               unsigned spin_limit) {
  pdl_wait();
  pdl_trigger();
  constexpr int WPB = MBB_T / 32;
  __shared__ float sb[MBB_TILE * 6];
  __shared__ unsigned s_tile;
  __shared__ long long s_wcnt[MBB_RPW][WPB];
  __shared__ long long s_excl;
  // when every B box fits one tile, the count pass keeps its ballot masks and
  // the emit pass writes from them (no second load and test of the boxes)
  __shared__ unsigned s_mask[MBB_RPW][WPB][MBB_TILE / 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ntiles = (MA + MBB_TA - 1) / MBB_TA;
  if (ntiles == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0;
    return;
  }
  for (;;) {
    __syncthreads();  // s_tile and s_excl of the previous tile are no longer read
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const unsigned tile = s_tile;
    if ((int64_t)tile >= ntiles) return;
    // the tile's A meshes i0 + r WPB + warp: candidate order is mesh order,
    // so the offsets run over (r, warp)
    const int64_t i0 = (int64_t)tile * MBB_TA;
    int64_t ii[MBB_RPW];
    bool has[MBB_RPW];
    float ab[MBB_RPW][6];
#pragma unroll
    for (int r = 0; r < MBB_RPW; ++r) {
      ii[r] = i0 + r * WPB + wib;
      has[r] = ii[r] < MA;
#pragma unroll
      for (int q = 0; q < 6; ++q) ab[r][q] = has[r] ? aabbA[6 * ii[r] + q] : (q < 3 ? 0.f : -1.f);
    }
    // in a self join only j > i counts: tiles below the block's first i are skipped
    const int64_t jstart = self_join ? ((i0 + 1) / MBB_TILE) * MBB_TILE : 0;
    const bool one = MB - jstart <= MBB_TILE;  // a single B tile: masks kept
    int64_t pos[MBB_RPW];
#pragma unroll
    for (int r = 0; r < MBB_RPW; ++r) pos[r] = 0;
    for (int pass = 0; pass < 2; ++pass) {
      int64_t cnt[MBB_RPW];
#pragma unroll
      for (int r = 0; r < MBB_RPW; ++r) cnt[r] = 0;
      for (int64_t t0 = jstart; t0 < MB; t0 += MBB_TILE) {
        const int n = MB - t0 < MBB_TILE ? (int)(MB - t0) : MBB_TILE;
        const bool kept = one && pass == 1;
        if (!kept) {
          __syncthreads();  // the previous tile is no longer read
          for (int k = threadIdx.x; k < n * 6; k += MBB_T) sb[k] = aabbB[6 * t0 + k];
          __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < MBB_RPW; ++r) {
          if (!has[r]) continue;
          const int64_t i = ii[r];
          for (int j0 = 0; j0 < n; j0 += 32) {
            const int jj = j0 + lane;
            const int64_t j = t0 + jj;
            unsigned m;
            bool ov;
            if (kept) {
              m = s_mask[r][wib][j0 >> 5];
              ov = (m >> lane) & 1u;
            } else {
              ov = false;
              if (jj < n && (!self_join || j > i)) {
                const float *bb = sb + 6 * jj;
                ov = ab[r][0] <= bb[3] && bb[0] <= ab[r][3] && ab[r][1] <= bb[4] &&
                     bb[1] <= ab[r][4] && ab[r][2] <= bb[5] && bb[2] <= ab[r][5];
              }
              m = __ballot_sync(FULL, ov);
              if (one && lane == 0) s_mask[r][wib][j0 >> 5] = m;
            }
            if (pass == 1 && ov) {
              const int64_t p = pos[r] + __popc(m & lt);
              cand[2 * p] = (int32_t)i;
              cand[2 * p + 1] = (int32_t)j;
            }
            if (pass == 1) pos[r] += __popc(m);
            else cnt[r] += __popc(m);
          }
        }
      }
      if (pass == 1) break;
      // the tile's count, its offset by look-back, each (r, warp)'s start
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < MBB_RPW; ++r) s_wcnt[r][wib] = cnt[r];
      }
      __syncthreads();
      long long agg = 0, before[MBB_RPW];
#pragma unroll
      for (int r = 0; r < MBB_RPW; ++r) before[r] = 0;
      for (int r2 = 0; r2 < MBB_RPW; ++r2)
        for (int k = 0; k < WPB; ++k) {
          const long long c = s_wcnt[r2][k];
          agg += c;
#pragma unroll
          for (int r = 0; r < MBB_RPW; ++r)
            if (r2 < r || (r2 == r && k < wib)) before[r] += c;
        }
      if (threadIdx.x == 0)
        lb_publish(state, tile, (tile == 0 ? LB_INC : LB_AGG) | (unsigned long long)agg);
      if (wib == 0) {
        const long long e = tile == 0 ? 0 : lb_exclusive(state, tile, spin_limit, lane);
        if (lane == 0) {
          if (e < 0) {
            atomicCAS(err, 0, DERR_TIMEOUT);
          } else {
            if (tile > 0) lb_publish(state, tile, LB_INC | (unsigned long long)(e + agg));
            if ((int64_t)tile == ntiles - 1) *count = e + agg;
          }
          s_excl = e;
        }
      }
      __syncthreads();
      if (s_excl < 0) return;  // (the whole block: s_excl is shared)
#pragma unroll
      for (int r = 0; r < MBB_RPW; ++r) pos[r] = s_excl + before[r];
    }
  }
}

// ---------------------------------------------------------------------------
// Leaf predicate on explicit inputs (tests of the filter and exact path)
// ---------------------------------------------------------------------------
__global__ void k_segtri_batch(const float *pq, const float *abc, int64_t n, int mode,
                               uint8_t *res, unsigned long long *nfb) {
  unsigned long long fb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    F3 p = ld3(pq + 6 * i), q = ld3(pq + 6 * i + 3);
    F3 a = ld3(abc + 9 * i), b = ld3(abc + 9 * i + 3), c = ld3(abc + 9 * i + 6);
    bool r;
    if (mode == PJ_LEAF_EXACT) {
      r = segtri_exact_staged(p, q, a, b, c);
    } else if (mode == PJ_LEAF_STATIC) {
      bool ex = false;
      const float D = fmaxf(
          fmaxf(fmaxf(fmaxf(p.x, q.x), fmaxf(a.x, fmaxf(b.x, c.x))) -
                    fminf(fminf(p.x, q.x), fminf(a.x, fminf(b.x, c.x))),
                fmaxf(fmaxf(p.y, q.y), fmaxf(a.y, fmaxf(b.y, c.y))) -
                    fminf(fminf(p.y, q.y), fminf(a.y, fminf(b.y, c.y)))),
          fmaxf(fmaxf(p.z, q.z), fmaxf(a.z, fmaxf(b.z, c.z))) -
              fminf(fminf(p.z, q.z), fminf(a.z, fminf(b.z, c.z))));
      r = segtri_static(p, q, a, b, c, static_err(D), &ex);
      fb += ex ? 1 : 0;
    } else {
      bool ex = false;
      r = segtri_filtered(p, q, a, b, c, &ex);
      fb += ex ? 1 : 0;
    }
    res[i] = r ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) fb += __shfl_xor_sync(FULL, fb, o);
  if ((threadIdx.x & 31) == 0 && fb) atomicAdd(nfb, fb);
}

pj_status run_segtri_batch(Ctx *ctx, const float *pq, const float *abc, int64_t n, int mode,
                           uint8_t *res, int64_t *n_fallback, cudaStream_t s) {
  pj_status st;
  unsigned long long *d = (unsigned long long *)ws_get(ctx, "segtri", 8, &st);
  if (!d) return st;
  PJ_CK(cudaMemsetAsync(d, 0, 8, s));
  if (n > 0) {
    int nb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 16);
    k_segtri_batch<<<nb, 256, 0, s>>>(pq, abc, n, mode, res, d);
    PJ_CK(cudaGetLastError());
  }
  unsigned long long h = 0;
  PJ_CK(cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  if (n_fallback) *n_fallback = (int64_t)h;
  return PJ_OK;
}

// ---------------------------------------------------------------------------
// Orchestration
// ---------------------------------------------------------------------------
typedef void (*RefineKernel)(RefineArgs);

static RefineKernel pick_kernel(int W, bool exact) {
  if (W == 2) return exact ? k_refine<2, true> : k_refine<2, false>;
  if (W == 4) return exact ? k_refine<4, true> : k_refine<4, false>;
  return exact ? k_refine<8, true> : k_refine<8, false>;
}

static RefineKernel pick_task_kernel(int W, bool exact) {
  if (W == 2) return exact ? k_refine_tasks<2, true> : k_refine_tasks<2, false>;
  if (W == 4) return exact ? k_refine_tasks<4, true> : k_refine_tasks<4, false>;
  return exact ? k_refine_tasks<8, true> : k_refine_tasks<8, false>;
}

typedef void (*WaveExpandKernel)(WaveArgs, const uint4 *, const unsigned *, uint4 *,
                                 unsigned *, uint4 *, unsigned *);
typedef void (*WaveLeafKernel)(WaveArgs, const uint4 *, const unsigned *);
typedef void (*WaveParityKernel)(WaveArgs);

static WaveExpandKernel pick_wave_expand(int W) {
  if (W == 2) return k_wave_expand<2>;
  if (W == 4) return k_wave_expand<4>;
  return k_wave_expand<8>;
}
static WaveLeafKernel pick_wave_leaf(int W, bool exact) {
  if (W == 2) return exact ? k_wave_leaf<2, true> : k_wave_leaf<2, false>;
  if (W == 4) return exact ? k_wave_leaf<4, true> : k_wave_leaf<4, false>;
  return exact ? k_wave_leaf<8, true> : k_wave_leaf<8, false>;
}
static WaveParityKernel pick_wave_parity(int W) {
  if (W == 2) return k_wave_parity<2>;
  if (W == 4) return k_wave_parity<4>;
  return k_wave_parity<8>;
}

typedef void (*StreamKernel)(StreamArgs);
typedef void (*AnyVertexKernel)(RefineArgs);
static AnyVertexKernel pick_any_vertex(int W) {
  if (W == 2) return k_any_vertex<2>;
  if (W == 4) return k_any_vertex<4>;
  return k_any_vertex<8>;
}

static StreamKernel pick_stream(int W, bool exact) {
  if (W == 2) return exact ? k_stream<2, true> : k_stream<2, false>;
  if (W == 4) return exact ? k_stream<4, true> : k_stream<4, false>;
  return exact ? k_stream<8, true> : k_stream<8, false>;
}
static int stream_smem_per_warp(int W) {
  return W == 2 ? stream_warp_bytes<2>() : (W == 4 ? stream_warp_bytes<4>() : stream_warp_bytes<8>());
}

static int smem_per_warp(int W, int cap) {
  if (W == 2) return warp_smem_bytes<2>(cap);
  if (W == 4) return warp_smem_bytes<4>(cap);
  return warp_smem_bytes<8>(cap);
}

static Side make_side(Dataset *d, Bvh &b) {
  Side s;
  s.nodes = b.d_nodes;
  s.roots = b.d_roots;
  s.trirec = b.d_trirec;
  s.toff = d->d_toff;
  s.voff = d->d_voff;
  s.aabb = d->d_aabb;
  s.xyz = d->d_xyz;
  s.lexorder = d->d_lexorder;
  s.mrec = d->d_mrec;
  return s;
}

// Blocks of `kern` resident per SM at (block, dynamic shared memory).  The
// first query for a kernel on a device also raises its dynamic shared-memory
// limit to the device's maximum, so that every later launch fits.  Both
// calls cost microseconds of host time ahead of a join's first launch, so
// the answers are kept per device, kernel and shape.
static cudaError_t occupancy(int device, const void *kern, int block, size_t smem, int *occ) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
  static std::map<std::pair<int, const void *>, bool> raised;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(device, kern, block, smem);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *occ = it->second;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (!raised[std::make_pair(device, kern)]) {
    // the limit covers dynamic memory only: the device's maximum less the
    // kernel's static shared memory
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) raised[std::make_pair(device, kern)] = true;
  }
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, block, smem);
  if (e == cudaSuccess) cache[key] = *occ;
  return e;
}

pj_status run_join(Ctx *ctx, Dataset *A, Dataset *B, const int32_t *cand,
                   const int32_t *cand_off, int64_t n_cand, int cand_on_device,
                   int self_join, const pj_join_opts *o, cudaStream_t s, pj_pairs *out,
                   bool safe) {
  // pick the BVH
  std::pair<int, int> key = o->width ? std::make_pair((int)o->width, (int)o->leaf_size)
                                     : A->last_bvh;
  auto ia = A->bvhs.find(key), ib = B->bvhs.find(key);
  if (ia == A->bvhs.end() || ib == B->bvhs.end())
    return fail(ctx, PJ_ERR_INVALID_ARG, "both datasets need a BVH of the requested width / "
                                         "leaf size (pj_build_bvh)");
  Bvh &bA = ia->second, &bB = ib->second;
  const int W = key.first;
  const int k = o->warps_per_pair ? o->warps_per_pair : 1;
  if (!(k == 1 || k == 2 || k == 4)) return fail(ctx, PJ_ERR_INVALID_ARG, "warps_per_pair must be 1, 2 or 4");
  const bool exact = o->leaf_mode == PJ_LEAF_EXACT;
  const int pred = o->predicate;
  if (pred < PJ_PRED_INTERSECTS || pred > PJ_PRED_ANY_VERTEX)
    return fail(ctx, PJ_ERR_INVALID_ARG, "unknown join predicate");
  // contains / within keep the parity result apart from the crossing result
  const bool split = pred == PJ_PRED_CONTAINS || pred == PJ_PRED_WITHIN;
  const bool parity_rays = pred != PJ_PRED_OVERLAP;

  pj_status st;
  // [0] n_cand, [1] K, [2] work counter, [3..4] spill queue counters, [5..7] wave counters
  int64_t *d_misc = (int64_t *)ws_get(ctx, "misc", 64, &st);
  if (!d_misc) return st;
  int64_t *h_misc = (int64_t *)cur_exec(ctx)->h_pinned;
  int *d_err = cur_exec(ctx)->d_err;

  // events: 0 start, 1 candidates ready, 2 refinement done, 3 end,
  // 4 parity done, 5 front end done (wavefront path, not in graph replays)
  cudaEvent_t *ev = cur_exec(ctx)->ev;
  bool phases = false;
  cudaEvent_t e0 = ev[0], e1 = ev[3];
  // the legacy default stream cannot be captured into a graph: order the
  // work on the context's stream after everything already queued on it
  if (o->use_graph && (s == cudaStreamLegacy || s == cudaStreamPerThread)) {
    PJ_CK(cudaEventRecord(ev[0], s));
    PJ_CK(cudaStreamWaitEvent(ctx->stream, ev[0], 0));
    s = ctx->stream;
  }
  PJ_CK(cudaMemsetAsync(d_err, 0, sizeof(int) * 4, s));
  PJ_CK(cudaEventRecord(e0, s));

  // 1. candidates.  C is the candidate count, Ccap what buffers and launches
  // are sized for: when every pair of the two datasets fits a modest buffer,
  // the device box join's count stays on the device (every later kernel
  // reads it there) and C is read back with the result, so the join runs
  // without a host round trip in the middle.
  int32_t *d_cand = nullptr;
  int32_t *d_off = nullptr;
  int64_t C = 0, Ccap = 0;
  bool count_on_host = true;
  // the single-pass box join, launched at the start of the device sequence
  std::function<cudaError_t()> mbb_in_graph;
  if (n_cand < 0) {
    // bounding-box filter join on the device
    const int64_t MA = A->M, MB = B->M;
    int64_t *counts = (int64_t *)ws_get(ctx, "mbb_counts", sizeof(int64_t) * (MA + 1), &st);
    if (!counts) return st;
    int64_t *offs = (int64_t *)ws_get(ctx, "mbb_offs", sizeof(int64_t) * (MA + 1), &st);
    if (!offs) return st;
    int nb = (int)std::min<int64_t>((MA + (MBB_T / 32) - 1) / (MBB_T / 32), (int64_t)ctx->num_sms * 64);
    const int64_t all = self_join ? MA * (MA - 1) / 2 : MA * MB;
    if (all <= (int64_t(1) << 24) && o->launch_mode != PJ_LAUNCH_PER_PAIR) {
      // every pair fits the buffers: the count stays on the device
      Ccap = std::max<int64_t>(all, 1);
      count_on_host = false;
    }
    if (!count_on_host && !safe) {
      // one launch: count, offset by look-back, emit (tiles of MBB_TA A meshes);
      // it is part of the device sequence below (captured with it)
      d_cand = (int32_t *)ws_get(ctx, "cand", sizeof(int32_t) * 2 * (size_t)Ccap, &st);
      if (!d_cand) return st;
      const int64_t tiles = (MA + MBB_TA - 1) / MBB_TA;
      unsigned long long *lb =
          (unsigned long long *)ws_get(ctx, "mbb_lookback", 8 * (size_t)(tiles + 1), &st);
      if (!lb) return st;
      int occ = 0;
      PJ_CK(occupancy(ctx->device, (const void *)k_mbb1, MBB_T, 0, &occ));
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)std::max(occ, 1) * ctx->num_sms));
      const float *aA = A->d_aabb, *aB = B->d_aabb;
      const unsigned polls = o->wait_polls > 0 ? (unsigned)o->wait_polls : (1u << 20);
      int32_t *dc = d_cand;
      int *de = d_err;
      mbb_in_graph = [=]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(lb, 0, 8 * (size_t)(tiles + 1), s);
        // the count is written by the last tile; zero until then, so that a
        // join whose look-back gave up refines nothing before it is redone
        if (e == cudaSuccess) e = cudaMemsetAsync(d_misc, 0, 8, s);
        if (e != cudaSuccess) return e;
        k_mbb1<<<grid, MBB_T, 0, s>>>(aA, MA, aB, MB, self_join,
                                      reinterpret_cast<unsigned *>(lb + tiles), lb, dc, d_misc,
                                      de, polls);
        return cudaGetLastError();
      };
    } else if (count_on_host && !safe) {
      // too many pairs to test them all: sort and sweep along x
      if ((st = mbb_sweep(ctx, A, B, self_join, s, d_misc, &d_cand, &C)) != PJ_OK) return st;
      Ccap = C;
    } else {
      k_mbb<false><<<nb, MBB_T, 0, s>>>(A->d_aabb, MA, B->d_aabb, MB, self_join, counts, nullptr, nullptr);
      ++ctx->launches;
      PJ_CK(cudaGetLastError());
      if ((st = scan_i64(ctx, counts, offs, MA, d_misc, s)) != PJ_OK) return st;
      if (count_on_host) {
        PJ_CK(cudaMemcpyAsync(h_misc, d_misc, 8, cudaMemcpyDeviceToHost, s));
        PJ_CK(cudaStreamSynchronize(s));
        C = Ccap = h_misc[0];
      }
      d_cand = (int32_t *)ws_get(ctx, "cand", sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(Ccap, 1), &st);
      if (!d_cand) return st;
      k_mbb<true><<<nb, MBB_T, 0, s>>>(A->d_aabb, MA, B->d_aabb, MB, self_join, nullptr, offs, d_cand);
      ++ctx->launches;
      PJ_CK(cudaGetLastError());
    }
  } else {
    C = Ccap = n_cand;
    if (cand_on_device) {
      d_cand = const_cast<int32_t *>(cand);
      d_off = const_cast<int32_t *>(cand_off);
    } else {
      d_cand = (int32_t *)ws_get(ctx, "cand", sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(C, 1), &st);
      if (!d_cand) return st;
      if (C > 0)
        PJ_CK(cudaMemcpyAsync(d_cand, cand, sizeof(int32_t) * 2 * C, cudaMemcpyHostToDevice, s));
      if (cand_off) {
        d_off = (int32_t *)ws_get(ctx, "cand_off", sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(C, 1), &st);
        if (!d_off) return st;
        if (C > 0)
          PJ_CK(cudaMemcpyAsync(d_off, cand_off, sizeof(int32_t) * 3 * C, cudaMemcpyHostToDevice, s));
      }
    }
    h_misc[0] = C;
    PJ_CK(cudaMemcpyAsync(d_misc, h_misc, 8, cudaMemcpyHostToDevice, s));
    if (C > 0)
      k_check_cand<<<std::min(blocks_for(C, 256), ctx->num_sms * 8), 256, 0, s>>>(
          d_cand, d_off, C, A->M, B->M, B->d_aabb, d_err);
    if (C > 0) ++ctx->launches;
  }
  uint8_t *d_flags = (uint8_t *)ws_get(ctx, "flags", (size_t)std::max<int64_t>(Ccap, 1), &st);
  if (!d_flags) return st;
  uint8_t *d_pflags = nullptr;
  if (split) {
    d_pflags = (uint8_t *)ws_get(ctx, "pflags", (size_t)std::max<int64_t>(Ccap, 1), &st);
    if (!d_pflags) return st;
  }
  unsigned long long *d_anyv = nullptr;  // work counter of the any-vertex pass
  if (pred == PJ_PRED_ANY_VERTEX) {
    d_anyv = (unsigned long long *)ws_get(ctx, "anyv_work", 8, &st);
    if (!d_anyv) return st;
  }
  int32_t *d_pairs = (int32_t *)ws_get(ctx, "pairs", sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(Ccap, 1), &st);
  if (!d_pairs) return st;
  int nchunks = (int)std::max<int64_t>(1, (Ccap + CMP_CHUNK - 1) / CMP_CHUNK);
  int64_t *bcount = (int64_t *)ws_get(ctx, "cmp_counts", sizeof(int64_t) * nchunks, &st);
  if (!bcount) return st;
  int64_t *boff = (int64_t *)ws_get(ctx, "cmp_offs", sizeof(int64_t) * nchunks, &st);
  if (!boff) return st;
  // single-pass compaction: look-back words of the tiles, then the ticket
  unsigned long long *cmp_lb =
      (unsigned long long *)ws_get(ctx, "cmp_lookback", 8 * (size_t)(nchunks + 1), &st);
  if (!cmp_lb) return st;

  PJ_CK(cudaEventRecord(ev[1], s));
  // 2. refinement
  const int depth = std::max(bA.max_depth, 1) + std::max(bB.max_depth, 1);
  // plain depth-first order needs at most 1 + (W^2 - 1) * depth entries; the
  // batched pops get 256 more and fall back to plain DFS if that is not enough
  int stack_cap = 1 + (W * W - 1) * depth + 256;
  const int per_warp = smem_per_warp(W, stack_cap);
  int threads = 128;
  if (per_warp * 4 > 200 * 1024) return fail(ctx, PJ_ERR_INTERNAL, "BVH too deep for the traversal stack");
  const int smem = per_warp * (threads / 32);
  RefineKernel kern = pick_kernel(W, exact);
  RefineKernel kern_tasks = pick_task_kernel(W, exact);
  {
    int occ_k = 0;
    PJ_CK(occupancy(ctx->device, (const void *)kern, threads, smem, &occ_k));
    PJ_CK(occupancy(ctx->device, (const void *)kern_tasks, threads, smem, &occ_k));
    if (pred == PJ_PRED_ANY_VERTEX)
      PJ_CK(occupancy(ctx->device, (const void *)pick_any_vertex(W), threads, smem, &occ_k));
  }
  // spill queues between the refinement passes
  const unsigned int q_cap = 1u << 22;
  uint4 *q1 = (uint4 *)ws_get(ctx, "spill1", sizeof(uint4) * (size_t)q_cap, &st);
  if (!q1) return st;
  uint4 *q2 = (uint4 *)ws_get(ctx, "spill2", sizeof(uint4) * (size_t)q_cap, &st);
  if (!q2) return st;
  unsigned int *qctr = reinterpret_cast<unsigned int *>(d_misc + 3);  // q1 n/pos, q2 n/pos
  // front end: 0 or PJ_FRONT_STREAM the streaming kernel, > 0 that many
  // breadth-first levels, PJ_FRONT_NONE none (the per-warp passes from the
  // candidates).  Both front ends start with the per-thread parity rays,
  // whose stack needs the BVH depth to stay within 64 levels.
  int wave_levels = o->wave_levels > 0 ? o->wave_levels : 0;
  bool stream = (o->wave_levels == 0 || o->wave_levels == PJ_FRONT_STREAM) &&
                o->launch_mode != PJ_LAUNCH_PER_PAIR;
  if (std::max(bA.max_depth, bB.max_depth) > 64 || safe) {
    wave_levels = 0;
    stream = false;
  }
  const unsigned int wq_cap = 1u << 23;
  uint4 *wqa = nullptr, *wqb = nullptr, *wlq = nullptr, *wpar = nullptr;
  // level counters, cleared by one memset: task count entering each level
  // [0, levels], leaf pairs found at each level, then the position of the
  // first warp pass in the last queue and the parity hand-over count/position
  unsigned int *wctr = nullptr;
  const int wctr_words = 2 * std::max(wave_levels, 0) + SQ_WORDS + 8;
  const unsigned int wpar_cap =
      (unsigned int)std::min<int64_t>(std::max<int64_t>(2 * Ccap, 1024), 1 << 22);
  int wave_grid[3] = {1, 1, 1};  // expand/init, leaf, parity: one resident wave
  bool front = (wave_levels > 0 || stream) && o->launch_mode != PJ_LAUNCH_PER_PAIR;
  int stream_grid = 1, stream_smem = 0;
  StreamKernel ks = pick_stream(W, exact);
  // the streaming launch's shared task queue (all-zero between launches)
  const unsigned int dq_cap = 1u << 22;
  uint4 *dq = nullptr;
  int2 *cbase = nullptr;
  if (stream && front) {
    dq = (uint4 *)ws_get_zeroed(ctx, "stream_queue", sizeof(uint4) * (size_t)dq_cap, s, &st);
    if (!dq) return st;
    cbase = (int2 *)ws_get(ctx, "cand_base", sizeof(int2) * (size_t)std::max<int64_t>(Ccap, 1), &st);
    if (!cbase) return st;
    stream_smem = 4 * stream_smem_per_warp(W);
    int occ = 0;
    PJ_CK(occupancy(ctx->device, (const void *)ks, 128, stream_smem, &occ));
    stream_grid = std::max(1, occ) * ctx->num_sms;
  }
  if (front) {
    int occ = 0;
    PJ_CK(occupancy(ctx->device, (const void *)pick_wave_expand(W), 256, 0, &occ));
    wave_grid[0] = std::max(1, occ) * ctx->num_sms;
    PJ_CK(occupancy(ctx->device, (const void *)pick_wave_leaf(W, exact), 256, 0, &occ));
    wave_grid[1] = std::max(1, occ) * ctx->num_sms;
    PJ_CK(occupancy(ctx->device, (const void *)pick_wave_parity(W), 128, 0, &occ));
    wave_grid[2] = std::max(1, occ) * ctx->num_sms;
    if (!stream) {
      wqa = (uint4 *)ws_get(ctx, "wave_a", sizeof(uint4) * (size_t)wq_cap, &st);
      if (!wqa) return st;
      wqb = (uint4 *)ws_get(ctx, "wave_b", sizeof(uint4) * (size_t)wq_cap, &st);
      if (!wqb) return st;
      wlq = (uint4 *)ws_get(ctx, "wave_leaf", sizeof(uint4) * (size_t)wq_cap, &st);
      if (!wlq) return st;
    }
    wpar = (uint4 *)ws_get(ctx, "wave_par", sizeof(uint4) * (size_t)wpar_cap, &st);
    if (!wpar) return st;
    wctr = (unsigned int *)ws_get(ctx, "wave_ctr", sizeof(unsigned int) * (size_t)wctr_words, &st);
    if (!wctr) return st;
  }
  unsigned int *d_cycles = nullptr;
  if (o->record_cycles) {
    d_cycles = (unsigned int *)ws_get(ctx, "cycles", sizeof(unsigned int) * (size_t)std::max<int64_t>(Ccap, 1), &st);
    if (!d_cycles) return st;
  }
  RefineArgs args;
  args.A = make_side(A, bA);
  args.B = make_side(B, bB);
  args.cand = d_cand;
  args.cand_off = d_off;
  args.cycles = d_cycles;
  args.n_cand = d_misc;
  args.flags = d_flags;
  args.work = (unsigned long long *)(d_misc + 2);
  args.counters = ctx->d_counters;
  args.err = d_err;
  args.stack_cap = stack_cap;
  args.max_pop = safe ? 1 : 32;
  args.warps_per_pair = k;
  args.MA = A->M;
  args.MB = B->M;
  args.single = -1;
  args.predicate = pred;
  args.pflags = d_pflags;
  const bool per_pair = o->launch_mode == PJ_LAUNCH_PER_PAIR;
  // pass 1 spills a pair after this many traversal steps; pass 2 after more;
  // pass 3 finishes everything
  long long budget1 = o->spill_budget > 0 ? o->spill_budget : (o->spill_budget < 0 ? 0 : 40000);
  if (safe) budget1 = 0;
  if (per_pair) budget1 = 0;
  const long long budget2 = budget1 > 0 ? 8 * budget1 : 0;
  args.q_cap = q_cap;
  args.q_in_cap = q_cap;
  args.q_in = nullptr;
  args.q_in_n = nullptr;
  args.q_in_pos = nullptr;
  args.q_par = nullptr;
  args.q_par_n = nullptr;
  args.q_par_pos = nullptr;
  args.q_par_cap = 0;
  int64_t blocks = 1;
  if (Ccap > 0 && o->launch_mode != PJ_LAUNCH_PER_PAIR) {
    int occ = 0;
    PJ_CK(occupancy(ctx->device, (const void *)kern, threads, smem, &occ));
    if (occ < 1) return fail(ctx, PJ_ERR_INTERNAL, "refinement kernel does not fit on an SM");
    blocks = std::min<int64_t>((int64_t)occ * ctx->num_sms, (Ccap * k * 32 + threads - 1) / threads);
    blocks = std::max<int64_t>(blocks, 1);
  }
  if (o->launch_mode == PJ_LAUNCH_PER_PAIR && k != 1)
    return fail(ctx, PJ_ERR_INVALID_ARG, "per-pair launches use one warp per pair");
  const bool graph = o->use_graph != 0;
  // optional per-launch events of the breadth-first levels (eager runs only)
  std::vector<cudaEvent_t> kev;
  struct KevGuard {
    std::vector<cudaEvent_t> *v;
    ~KevGuard() {
      for (auto e : *v) cudaEventDestroy(e);
    }
  } kg{&kev};
  bool kev_used = false;
  if (o->kernel_times && front) {
    kev.resize(stream ? 2 : 2 * (size_t)wave_levels + 1);
    for (auto &e : kev) PJ_CK(cudaEventCreate(&e));
  }
  auto make_wave_args = [&]() {
    WaveArgs wa;
    wa.A = args.A;
    wa.B = args.B;
    wa.cand = d_cand;
    wa.cand_off = d_off;
    wa.n_cand = d_misc;
    wa.flags = d_flags;
    wa.counters = ctx->d_counters;
    wa.err = d_err;
    wa.q_cap = wq_cap;
    wa.lshift = key.second == 1 ? 0 : (key.second == 2 ? 1 : (key.second == 4 ? 2 : 3));
    wa.MA = A->M;
    wa.MB = B->M;
    wa.q_par = wpar;
    wa.q_par_n = nullptr;
    wa.q_par_cap = wpar_cap;
    wa.par_dirs = pred == PJ_PRED_OVERLAP ? 0 : (pred == PJ_PRED_CONTAINS ? 1 : (pred == PJ_PRED_WITHIN ? 2 : 3));
    wa.pflags = d_pflags;
    wa.need = d_pflags;  // contains / within: traverse where the parity test holds
    return wa;
  };
  // everything from here to the compacted pairs is a fixed sequence of
  // stream operations (no host synchronisation), so it can be captured
  auto device_part = [&](bool timed) -> pj_status {
    if (mbb_in_graph) {
      PJ_CK(mbb_in_graph());
      ++ctx->launches;
      if (timed) PJ_CK(cudaEventRecord(ev[1], s));
    }
    if (d_pflags) PJ_CK(cudaMemsetAsync(d_pflags, 0, (size_t)Ccap, s));
    if (Ccap > 0) {
      if (o->launch_mode == PJ_LAUNCH_PER_PAIR) {
        args.q_out = nullptr;
        args.q_out_n = nullptr;
        args.budget = 0;
        for (int64_t c = 0; c < C; ++c) {
          args.single = c;
          kern<<<1, 32, per_warp, s>>>(args);
        }
        args.single = -1;
        ctx->launches += C;
      } else if (front && stream) {
        // parity rays per thread, then the streaming refinement in one
        // persistent launch, whose warps first take the rays the per-thread
        // kernel handed over
        PJ_CK(cudaMemsetAsync(wctr, 0, sizeof(unsigned int) * wctr_words, s));
        PJ_CK(cudaMemsetAsync(d_flags, 0, (size_t)Ccap, s));
        WaveArgs wa = make_wave_args();
        // words: [0, SQ_WORDS) the streaming launch's control words, then the
        // parity hand-over fill and claim position, a zero count and the
        // intake position of a hand-over launch
        unsigned int *sc = wctr, *hc = wctr + SQ_WORDS;
        wa.q_par_n = hc;
        // the long rays go to warps before the traversal: a containment-only
        // pair (no crossing to stop at) is the costliest kind to traverse.
        // (Running the parity launches on a second stream beside the
        // streaming one measured slower: its persistent grid holds the SMs,
        // so the parity flags came late -- 0.445 against 0.437 ms a step.)
        if (parity_rays) PJ_CK(launch_pdl(pick_wave_parity(W), wave_grid[2], 128, 0, s, wa));
        if (parity_rays && split) {
          // contains / within: the streaming intake reads the parity results
          // (it traverses only where they hold), so the long rays finish
          // first, in a launch of their own
          RefineArgs ap = args;
          ap.q_in = q1;
          ap.q_in_n = hc + 2;  // stays zero: no traversal tasks in this launch
          ap.q_in_pos = hc + 3;
          ap.q_out = nullptr;
          ap.q_out_n = nullptr;
          ap.budget = 0;
          ap.q_par = wpar;
          ap.q_par_n = hc;
          ap.q_par_pos = hc + 1;
          ap.q_par_cap = wpar_cap;
          PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, ap));
          ctx->launches += 1;
        }
        if (timed) PJ_CK(cudaEventRecord(ev[4], s));
        StreamArgs sa{};
        sa.w = wa;
        sa.ctl = sc;
        sa.dq = dq;
        sa.cbase = cbase;
        sa.dq_cap = dq_cap;
        sa.spin_limit = o->wait_polls > 0 ? (unsigned)o->wait_polls : (1u << 19);
        sa.hungry_max = 2u * (unsigned)ctx->num_sms;
        sa.give_after = 5000;
        sa.q_par_pos = split ? nullptr : hc + 1;
        sa.par_stack_cap = args.stack_cap;
        const bool kt = timed && !kev.empty();
        if (kt) PJ_CK(cudaEventRecord(kev[0], s));
        PJ_CK(launch_pdl(ks, stream_grid, 128, stream_smem, s, sa));
        if (kt) {
          PJ_CK(cudaEventRecord(kev[1], s));
          kev_used = true;
        }
        if (timed) {
          PJ_CK(cudaEventRecord(ev[5], s));
          phases = true;
        }
        ctx->launches += parity_rays ? 2 : 1;
      } else if (front) {
        // wavefront front end, then the warp passes over what is left
        PJ_CK(cudaMemsetAsync(d_misc + 2, 0, 48, s));  // work and spill counters
        PJ_CK(cudaMemsetAsync(wctr, 0, sizeof(unsigned int) * wctr_words, s));
        PJ_CK(cudaMemsetAsync(d_flags, 0, (size_t)Ccap, s));
        WaveArgs wa = make_wave_args();
        unsigned int *qn = wctr, *ln = wctr + wave_levels + 1, *misc = ln + wave_levels;
        wa.q_par_n = misc + 1;
        wa.q_par_cap = wpar_cap;
        WaveExpandKernel kx = pick_wave_expand(W);
        WaveLeafKernel kl = pick_wave_leaf(W, exact);
        WaveParityKernel kp = pick_wave_parity(W);
        const int wblocks = wave_grid[0], lblocks = wave_grid[1], pblocks = wave_grid[2];
        if (parity_rays) PJ_CK(launch_pdl(kp, pblocks, 128, 0, s, wa));
        // the rays over the per-thread node budget, one warp each, before
        // the front end: a containment-only pair (no crossing to stop at)
        // is the costliest kind to traverse, so its flag should be set early
        RefineArgs ap = args;
        ap.q_in = wqa;
        ap.q_in_n = misc + 3;  // stays zero: no traversal tasks in this launch
        ap.q_in_pos = misc + 4;
        ap.q_out = nullptr;
        ap.q_out_n = nullptr;
        ap.budget = 0;
        ap.q_par = wpar;
        ap.q_par_n = misc + 1;
        ap.q_par_pos = misc + 2;
        ap.q_par_cap = wpar_cap;
        if (parity_rays) PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, ap));
        if (timed) PJ_CK(cudaEventRecord(ev[4], s));
        // the roots after the parity rays: contains / within traverse only
        // the candidates whose parity test held
        k_wave_init<<<wblocks, 256, 0, s>>>(wa, wqa, qn);
        uint4 *qin = wqa, *qout = wqb;
        const bool kt = timed && !kev.empty();
        for (int lvl = 0; lvl < wave_levels; ++lvl) {
          if (kt) PJ_CK(cudaEventRecord(kev[2 * lvl], s));
          PJ_CK(launch_pdl(kx, wblocks, 256, 0, s, wa, (const uint4 *)qin,
                           (const unsigned *)(qn + lvl), qout, qn + lvl + 1, wlq, ln + lvl));
          if (kt) PJ_CK(cudaEventRecord(kev[2 * lvl + 1], s));
          PJ_CK(launch_pdl(kl, lblocks, 256, 0, s, wa, (const uint4 *)wlq,
                           (const unsigned *)(ln + lvl)));
          std::swap(qin, qout);
        }
        if (kt) {
          PJ_CK(cudaEventRecord(kev[2 * wave_levels], s));
          kev_used = true;
        }
        if (timed) {
          PJ_CK(cudaEventRecord(ev[5], s));
          phases = true;
        }
        RefineArgs a1 = args;
        a1.q_in = qin;
        a1.q_in_n = qn + wave_levels;
        a1.q_in_pos = misc;
        a1.q_in_cap = wq_cap;
        a1.q_par = nullptr;
        a1.q_out = budget1 > 0 ? q1 : nullptr;
        a1.q_out_n = qctr;
        a1.budget = budget1;
        PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, a1));
        RefineArgs a2 = args;
        a2.q_in = q1;
        a2.q_in_n = qctr;
        a2.q_in_pos = qctr + 1;
        a2.q_out = q2;
        a2.q_out_n = qctr + 2;
        a2.budget = budget2;
        PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, a2));
        RefineArgs a3 = args;
        a3.q_in = q2;
        a3.q_in_n = qctr + 2;
        a3.q_in_pos = qctr + 3;
        a3.q_out = nullptr;
        a3.q_out_n = nullptr;
        a3.budget = 0;
        PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, a3));
        ctx->launches += 6 + 2 * wave_levels;
      } else {
        PJ_CK(cudaMemsetAsync(d_misc + 2, 0, 24, s));  // work counter, queue counters
        RefineArgs a1 = args;
        a1.q_out = budget1 > 0 ? q1 : nullptr;
        a1.q_out_n = qctr;
        a1.budget = budget1;
        kern<<<(int)blocks, threads, smem, s>>>(a1);
        RefineArgs a2 = args;
        a2.q_in = q1;
        a2.q_in_n = qctr;
        a2.q_in_pos = qctr + 1;
        a2.q_out = q2;
        a2.q_out_n = qctr + 2;
        a2.budget = budget2;
        PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, a2));
        RefineArgs a3 = args;
        a3.q_in = q2;
        a3.q_in_n = qctr + 2;
        a3.q_in_pos = qctr + 3;
        a3.q_out = nullptr;
        a3.q_out_n = nullptr;
        a3.budget = 0;
        PJ_CK(launch_pdl(kern_tasks, (int)blocks, threads, smem, s, a3));
        ctx->launches += 3;
      }
      PJ_CK(cudaGetLastError());
    }
    // the other predicates' last steps: the any-vertex pass over what did
    // not intersect; contains / within combine parity and crossing
    if (pred == PJ_PRED_ANY_VERTEX && Ccap > 0) {
      PJ_CK(cudaMemsetAsync(d_anyv, 0, 8, s));
      RefineArgs av = args;
      av.work = d_anyv;
      av.max_pop = 32;
      PJ_CK(launch_pdl(pick_any_vertex(W), (int)blocks, threads, smem, s, av));
      ++ctx->launches;
    }
    if (split && Ccap > 0) {
      PJ_CK(launch_pdl(k_pred_combine, std::min(blocks_for(Ccap, 256), ctx->num_sms * 8), 256, 0,
                       s, d_flags, (const uint8_t *)d_pflags, (const int64_t *)d_misc));
      ++ctx->launches;
    }
    if (timed) PJ_CK(cudaEventRecord(ev[2], s));
    // 3. compaction: one launch (offsets by look-back), or count, scan and
    // emit in the safe mode
    if (!safe) {
      PJ_CK(cudaMemsetAsync(cmp_lb, 0, 8 * (size_t)(nchunks + 1), s));
      PJ_CK(launch_pdl(k_compact, nchunks, CMP_T, 0, s, (const uint8_t *)d_flags,
                       (const int64_t *)d_misc, (const int32_t *)d_cand,
                       reinterpret_cast<unsigned *>(cmp_lb + nchunks), cmp_lb, d_pairs,
                       d_misc + 1, ctx->d_counters + C_HITS, d_err,
                       o->wait_polls > 0 ? (unsigned)o->wait_polls : (1u << 20)));
      ++ctx->launches;
      PJ_CK(cudaGetLastError());
      return PJ_OK;
    }
    PJ_CK(launch_pdl(k_flag_count, nchunks, CMP_T, 0, s, (const uint8_t *)d_flags,
                     (const int64_t *)d_misc, bcount, ctx->d_counters + C_HITS));
    ++ctx->launches;
    pj_status st2 = scan_i64(ctx, bcount, boff, nchunks, d_misc + 1, s);
    if (st2 != PJ_OK) return st2;
    PJ_CK(launch_pdl(k_flag_emit, nchunks, CMP_T, 0, s, (const uint8_t *)d_flags,
                     (const int64_t *)d_misc, (const int32_t *)d_cand, (const int64_t *)boff,
                     d_pairs));
    ++ctx->launches;
    PJ_CK(cudaGetLastError());
    return PJ_OK;
  };
  char gk[256];
  snprintf(gk, sizeof(gk), "%p|%p|%p|%p|%p|%d|%d|%d|%d|%d|%lld|%d|%d|%d", (void *)A, (void *)B,
           (void *)d_cand, (void *)d_off, (void *)d_cycles, W, key.second, (int)exact, k,
           (int)o->launch_mode, (long long)Ccap, (int)budget1,
           args.max_pop * 1000 + wave_levels * 2 + (stream ? 1 : 0),
           (mbb_in_graph ? 1 + self_join : 0) + 4 * pred);
  snprintf(gk + strlen(gk), sizeof(gk) - strlen(gk), "|%d", (int)o->wait_polls);
  bool replayed = false;
  if (graph) {
    auto it = ctx->graphs.find(gk);
    if (it != ctx->graphs.end()) {
      PJ_CK(cudaGraphLaunch(it->second, s));
      ctx->launches += ctx->graph_kernels[gk];
      replayed = true;
    }
  }
  if (!replayed) {
    if ((st = device_part(true)) != PJ_OK) return st;
    if (graph) {
      // capture the same sequence for the next call with this shape
      cudaGraph_t g = nullptr;
      PJ_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const unsigned long long before = ctx->launches;
      pj_status cst = device_part(false);
      cudaError_t ce = cudaStreamEndCapture(s, &g);
      ctx->graph_kernels[gk] = ctx->launches - before;
      ctx->launches = before;  // captured, not launched
      if (cst != PJ_OK) {
        if (g) cudaGraphDestroy(g);
        return cst;
      }
      PJ_CK(ce);
      cudaGraphExec_t ge = nullptr;
      cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      PJ_CK(ie);
      ctx->graphs[gk] = ge;
    }
  }
  PJ_CK(cudaEventRecord(e1, s));
  PJ_CK(cudaMemcpyAsync(h_misc, d_misc, 16, cudaMemcpyDeviceToHost, s));
  int *herr = reinterpret_cast<int *>(h_misc + 4);  // pinned, beside the counts
  PJ_CK(cudaMemcpyAsync(herr, d_err, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  if (herr[1]) return fail(ctx, PJ_ERR_INVALID_ARG, "a candidate mesh id is out of range");
  if (herr[2]) return fail(ctx, PJ_ERR_INVALID_ARG, "a translated candidate mesh leaves the 2^18 grid");
  if (!safe && (herr[0] == DERR_STACK || herr[0] == DERR_QUEUE || herr[0] == DERR_TIMEOUT)) {
    // batched pops outgrew the stack, a spill queue filled up or a bounded
    // wait gave up: redo the whole join in the safe mode -- every pair in
    // plain depth-first order (whose stack bound holds by construction), in
    // one pass, and the multi-pass box join and compaction
    if (dq) ws_mark_dirty(ctx, "stream_queue");
    pj_join_opts o2 = *o;
    o2.use_graph = 0;
    return run_join(ctx, A, B, cand, cand_off, n_cand, cand_on_device, self_join, &o2, s, out,
                    true);
  }
  if (herr[0]) return fail(ctx, PJ_ERR_INTERNAL, "traversal stack capacity exceeded");
  const int64_t K = h_misc[1];
  if (!count_on_host) C = h_misc[0];  // the device box join's count
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventElapsedTime(&out->mbb_ms, ev[0], ev[1]);
  out->parity_ms = out->front_ms = out->tasks_ms = -1.f;
  out->expand_ms = out->leaf_ms = -1.f;
  if (kev_used && !replayed && stream) {
    cudaEventElapsedTime(&out->expand_ms, kev[0], kev[1]);
    out->leaf_ms = 0.f;
  } else if (kev_used && !replayed) {
    out->expand_ms = out->leaf_ms = 0.f;
    for (int l = 0; l < wave_levels; ++l) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, kev[2 * l], kev[2 * l + 1]);
      cudaEventElapsedTime(&b, kev[2 * l + 1], kev[2 * l + 2]);
      out->expand_ms += a;
      out->leaf_ms += b;
    }
  }
  if (replayed) {
    // one graph launch: refinement and compaction are not separated
    cudaEventElapsedTime(&out->refine_ms, ev[1], ev[3]);
    out->compact_ms = 0.f;
  } else {
    cudaEventElapsedTime(&out->refine_ms, ev[1], ev[2]);
    cudaEventElapsedTime(&out->compact_ms, ev[2], ev[3]);
    if (phases) {
      cudaEventElapsedTime(&out->parity_ms, ev[1], ev[4]);
      cudaEventElapsedTime(&out->front_ms, ev[4], ev[5]);
      cudaEventElapsedTime(&out->tasks_ms, ev[5], ev[2]);
    }
  }

  out->count = K;
  out->n_candidates = C;
  out->device_ms = ms;
  if (cur_exec(ctx)->borrow_out) {
    // serving: the caller reads the result from this slot's workspaces
    // before its next join (the stream is synchronised above)
    out->pairs = d_pairs;
    out->flags = d_flags;
    out->on_device = 1;
    return PJ_OK;
  }
  size_t bytes = sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(K, 1);
  if (o->out_host) {
    cudaError_t pe;
    out->pairs = (int32_t *)hpool_get(ctx, bytes, &pe);
    PJ_CK(pe);
    out->on_device = 0;
    if (K > 0) PJ_CK(cudaMemcpyAsync(out->pairs, d_pairs, sizeof(int32_t) * 2 * K, cudaMemcpyDeviceToHost, s));
  } else {
    cudaError_t pe;
    out->pairs = (int32_t *)pool_get(ctx, bytes, &pe);
    PJ_CK(pe);
    out->on_device = 1;
    if (K > 0) PJ_CK(cudaMemcpyAsync(out->pairs, d_pairs, sizeof(int32_t) * 2 * K, cudaMemcpyDeviceToDevice, s));
  }
  if (o->keep_flags) {
    cudaError_t pe;
    out->flags = (uint8_t *)pool_get(ctx, (size_t)std::max<int64_t>(C, 1), &pe);
    PJ_CK(pe);
    if (C > 0) PJ_CK(cudaMemcpyAsync(out->flags, d_flags, C, cudaMemcpyDeviceToDevice, s));
  }
  if (d_cycles) {
    cudaError_t pe;
    out->cycles = (unsigned int *)pool_get(ctx, sizeof(unsigned int) * (size_t)std::max<int64_t>(C, 1), &pe);
    PJ_CK(pe);
    if (C > 0)
      PJ_CK(cudaMemcpyAsync(out->cycles, d_cycles, sizeof(unsigned int) * C, cudaMemcpyDeviceToDevice, s));
  }
  PJ_CK(cudaStreamSynchronize(s));
  return PJ_OK;
}


// ---------------------------------------------------------------------------
// Join without allocation (pj_join_intersects_noalloc)
//
// For callers that cannot call cudaMalloc: real-time loops that must not
// block on the allocator's implicit device synchronisation, and hosts whose
// device memory is owned by another allocator or budget (a framework's
// caching allocator, a pool sized at start-up).  The caller passes device
// buffers for the candidates, the per-candidate flags, the pairs and the
// count; the little scratch the kernels need (candidate count, work counter,
// error words, per-chunk counts and offsets of the compaction) lives in one
// file-scope device array shared by every call on a device.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocMaxChunks = 4096;
constexpr int64_t kNoAllocMaxCand = kNoAllocMaxChunks * CMP_CHUNK;  // 16,777,216
// int64 words: [0] candidate count, [1] work counter, [2..3] four int error
// words, [4..7] unused, then kNoAllocMaxChunks chunk counts and as many offsets
constexpr size_t kNoAllocScratchWords = 8 + 2 * kNoAllocMaxChunks;
static __device__ __align__(256) int64_t g_noalloc_scratch[kNoAllocScratchWords];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];  // device address of the array, per device

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name is not a device address).
static pj_status noalloc_scratch(Ctx *ctx, int64_t **out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (ctx->device < 0 || ctx->device >= 256)
    return fail(ctx, PJ_ERR_INVALID_ARG, "device ordinal out of range");
  if (!g_noalloc_addr[ctx->device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[ctx->device] = p;
  }
  *out = static_cast<int64_t *>(g_noalloc_addr[ctx->device]);
  return PJ_OK;
}

__global__ void k_noalloc_begin(int64_t *scr, int64_t n) {
  scr[0] = n;  // candidate count
  scr[1] = 0;  // work counter
  scr[2] = 0;  // error words
  scr[3] = 0;
}

// one block of SCAN_T threads: exclusive scan of the chunk counts, then the
// pair count (-1 if a device-side check failed)
__global__ void k_noalloc_scan(const int64_t *counts, int64_t *offs, int64_t nchunks,
                               const int *err, int64_t *out_count) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nchunks; base += SCAN_T) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nchunks ? counts[i] : 0;
    int64_t tot;
    int64_t e = block_excl_scan(v, &tot);
    if (i < nchunks) offs[i] = carry + e;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *out_count = (err[0] || err[1] || err[2]) ? -1 : carry;
}

pj_status run_join_noalloc(Ctx *ctx, Dataset *A, Dataset *B, const int32_t *d_cand,
                           int64_t n, uint8_t *d_flags, int32_t *d_pairs, int64_t *d_count,
                           cudaStream_t s) {
  if (n < 0 || n > kNoAllocMaxCand)
    return fail(ctx, PJ_ERR_INVALID_ARG,
                "n_cand must be in [0, 16777216] for the allocation-free join");
  if (!d_count || (n > 0 && (!d_cand || !d_flags || !d_pairs)))
    return fail(ctx, PJ_ERR_INVALID_ARG, "null device buffer");
  // each dataset's own last-built BVH; the two must have one shape
  if (A->last_bvh != B->last_bvh)
    return fail(ctx, PJ_ERR_INVALID_ARG,
                "the two datasets' last-built BVHs differ in width or leaf size (pj_build_bvh)");
  auto ia = A->bvhs.find(A->last_bvh), ib = B->bvhs.find(B->last_bvh);
  if (ia == A->bvhs.end() || ib == B->bvhs.end())
    return fail(ctx, PJ_ERR_INVALID_ARG, "both datasets need a BVH (pj_build_bvh)");
  Bvh &bA = ia->second, &bB = ib->second;
  const int W = A->last_bvh.first;
  int64_t *scr = nullptr;
  pj_status st = noalloc_scratch(ctx, &scr);
  if (st != PJ_OK) return st;
  int64_t *d_n = scr;
  unsigned long long *work = reinterpret_cast<unsigned long long *>(scr + 1);
  int *err = reinterpret_cast<int *>(scr + 2);
  int64_t *counts = scr + 8, *offs = scr + 8 + kNoAllocMaxChunks;

  // plain depth-first traversal: its stack bound holds by construction, so
  // there is no overflow to recover from
  const int depth = std::max(bA.max_depth, 1) + std::max(bB.max_depth, 1);
  const int stack_cap = 1 + (W * W - 1) * depth + 256;
  const int per_warp = smem_per_warp(W, stack_cap);
  const int threads = 128;
  if (per_warp * 4 > 200 * 1024) return fail(ctx, PJ_ERR_INTERNAL, "BVH too deep for the traversal stack");
  const int smem = per_warp * (threads / 32);
  RefineKernel kern = pick_kernel(W, false);
  int occ = 0;
  PJ_CK(occupancy(ctx->device, (const void *)kern, threads, smem, &occ));
  if (occ < 1) return fail(ctx, PJ_ERR_INTERNAL, "refinement kernel does not fit on an SM");
  RefineArgs args;
  args.A = make_side(A, bA);
  args.B = make_side(B, bB);
  args.cand = d_cand;
  args.cand_off = nullptr;
  args.cycles = nullptr;
  args.q_out = nullptr;
  args.q_out_n = nullptr;
  args.q_cap = 0;
  args.budget = 0;
  args.q_in = nullptr;
  args.q_in_n = nullptr;
  args.q_in_pos = nullptr;
  args.q_in_cap = 0;
  args.q_par = nullptr;
  args.q_par_n = nullptr;
  args.q_par_pos = nullptr;
  args.q_par_cap = 0;
  args.n_cand = d_n;
  args.flags = d_flags;
  args.work = work;
  args.counters = ctx->d_counters;
  args.err = err;
  args.stack_cap = stack_cap;
  args.max_pop = 1;
  args.warps_per_pair = 1;
  args.MA = A->M;
  args.MB = B->M;
  args.single = -1;
  args.predicate = PJ_PRED_INTERSECTS;
  args.pflags = nullptr;

  k_noalloc_begin<<<1, 1, 0, s>>>(scr, n);
  if (n > 0) {
    k_check_cand<<<std::min(blocks_for(n, 256), ctx->num_sms * 8), 256, 0, s>>>(
        d_cand, nullptr, n, A->M, B->M, B->d_aabb, err);
    int64_t blocks = std::min<int64_t>((int64_t)occ * ctx->num_sms, (n * 32 + threads - 1) / threads);
    kern<<<(int)std::max<int64_t>(blocks, 1), threads, smem, s>>>(args);
  }
  const int nchunks = (int)std::max<int64_t>(1, (n + CMP_CHUNK - 1) / CMP_CHUNK);
  k_flag_count<<<nchunks, CMP_T, 0, s>>>(d_flags, d_n, counts, ctx->d_counters + C_HITS);
  k_noalloc_scan<<<1, SCAN_T, 0, s>>>(counts, offs, nchunks, err, d_count);
  k_flag_emit<<<nchunks, CMP_T, 0, s>>>(d_flags, d_n, d_cand, offs, d_pairs);
  PJ_CK(cudaGetLastError());
  return PJ_OK;
}

}  // namespace pj
