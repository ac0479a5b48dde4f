// Dataset-level join: the paper's own formulation (Sec. 3.1-3.5), next to
// the per-pair refinement of the rest of the library.
//
//   * one BVH over all triangles of a dataset (the same LBVH build as the
//     per-mesh trees, run on the dataset as one mesh; each triangle record
//     then carries its owning mesh -- the paper's triangle-to-object map);
//   * Alg. 1 in both directions (Sec. 3.2 "Bidirectional tracing"): every
//     owned edge of one dataset is traced as a bounded segment through the
//     other's BVH (conservative slab test at nodes, the exact strict
//     segment/triangle test at leaves) and every crossing is recorded -- an
//     edge may pierce several objects, so the traversal does not stop at the
//     first hit (the multi-hit loop of Alg. 1);
//   * containment (Sec. 3.3-3.4): each object casts one ray from its
//     lexicographically first vertex through the other dataset's BVH and
//     toggles a parity bit for every object whose triangle it crosses; an
//     odd count records the pair;
//   * materialisation (Sec. 3.5): a hashmap sized by the selectivity
//     estimate (one pass, a relaunch with twice the slots on overflow), the
//     counting two-pass strategy (count, prefix sum, emit, sort, unique), or
//     a hashmap of a fixed size.
//
// Exactness.  The per-pair join's containment test uses, for each pair, the
// first vertex of B_j that is not on A_i's surface.  A parity ray from the
// first vertex decides every pair whose surface does not pass through that
// vertex; pairs whose surface does (checked exactly at the triangles the ray
// meets, which include every triangle holding the vertex), and all pairs of
// a ray that meets more candidate objects than it can track, are handed to
// the per-pair join.  The result therefore equals the per-pair join over the
// bounding-box candidates, which the tests check against the oracle.
#include <cub/cub.cuh>

#include <algorithm>
#include <cstring>
#include <vector>

#include "pj_geom.cuh"
#include "pj_internal.cuh"

namespace pj {

constexpr unsigned long long kHashEmpty = ~0ull;
constexpr int kDsStack = 192;     // traversal stack entries per thread
constexpr int kParList = 48;      // objects a parity ray tracks
constexpr int kHashProbes = 2048;  // probes before a hashmap counts as full

enum { DS_EDGES = 0, DS_NODES, DS_TRIS, DS_HITS, DS_RAYS, DS_OVERFLOW, DS_ERR, DS_NREC,
       DS_NOBJ, DS_NSTAT };

struct DsSide {
  const float *xyz;
  const int32_t *tris;
  const uint8_t *emask;
  const int64_t *toff;
  int64_t M, F;
  const float4 *mrec;    // per mesh: box, first lexicographic vertex
  const float *aabb;     // per mesh: closed box
  const float *nodes;    // dataset BVH
  const float4 *trirec;  // its triangle records, .w of the third = owning mesh
};

// where a pair goes: a hashmap, a per-item count, or a slot of a flat buffer
enum { SINK_HASH = 0, SINK_COUNT = 1, SINK_EMIT = 2 };
struct Sink {
  int mode;
  unsigned long long *table;  // SINK_HASH
  unsigned long long mask;    // slots - 1 (a power of two)
  int64_t *cnt;               // SINK_COUNT: per item
  const int64_t *off;         // SINK_EMIT: per item
  unsigned long long *keys;   // SINK_EMIT
  int64_t base;               // this launch's first item index
};

// pairs handed to the per-pair join, and objects whose rays overflowed
struct Recheck {
  int2 *pairs;
  int32_t *objs;
  unsigned long long cap;
};

// MurmurHash3's 64-bit finaliser (Appleby), to spread pair keys over slots
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ void hash_insert(const Sink &k, unsigned long long key,
                                            unsigned long long *st) {
  unsigned long long h = mix64(key) & k.mask;
  for (int i = 0; i < kHashProbes; ++i) {
    // a plain read first: most records repeat a pair already present
    const unsigned long long cur = __ldcg(k.table + h);
    if (cur == key) return;
    if (cur == kHashEmpty) {
      const unsigned long long prev = atomicCAS(k.table + h, kHashEmpty, key);
      if (prev == kHashEmpty || prev == key) return;
    }
    h = (h + 1) & k.mask;
  }
  atomicExch(st + DS_OVERFLOW, 1ull);  // relaunched with more slots
}

__device__ __forceinline__ int64_t mesh_of(const int64_t *off, int64_t M, int64_t e) {
  int64_t lo = 0, hi = M - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long pair_key(int a, int b, int self_join) {
  if (self_join && a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
}

__device__ __forceinline__ void flush_stats(unsigned long long *st, const unsigned long long *v,
                                            int n) {
  for (int i = 0; i < n; ++i) {
    unsigned long long x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(st + i, x);
  }
}

// Alg. 1, one direction: thread per source triangle, each of its owned edges
// through the target BVH, every strict crossing recorded.  dir 0: source A,
// target B (pairs (source, target)); dir 1 the reverse.
template <int W>
__global__ void __launch_bounds__(128) k_ds_edges(DsSide S, DsSide T, int dir, int self_join,
                                                  Sink sink, unsigned long long *st) {
  uint32_t stk[kDsStack];
  unsigned long long c_edges = 0, c_nodes = 0, c_tris = 0, c_hits = 0;
  const int SW = node_stride_words(W);
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < S.F;
       f += (int64_t)gridDim.x * blockDim.x) {
    const unsigned em = S.emask[f];
    int64_t n_rec = 0;
    if (em) {
      const int os = (int)mesh_of(S.toff, S.M, f);
      const F3 v[3] = {ld3(S.xyz + 3 * (int64_t)S.tris[3 * f]),
                       ld3(S.xyz + 3 * (int64_t)S.tris[3 * f + 1]),
                       ld3(S.xyz + 3 * (int64_t)S.tris[3 * f + 2])};
      for (int k = 0; k < 3; ++k) {
        if (!((em >> k) & 1u)) continue;
        const F3 p = v[k], q = v[k == 2 ? 0 : k + 1];
        const Seg seg = make_seg(p, q);
        c_edges += 1;
        int sp = 0;
        stk[sp++] = 0u;  // the root
        while (sp > 0) {
          const uint32_t node = stk[--sp];
          c_nodes += 1;
          const float4 *slot = reinterpret_cast<const float4 *>(T.nodes + (int64_t)node * SW + 8);
          for (int c = 0; c < W; ++c) {
            const float4 s0 = __ldg(slot + 2 * c), s1 = __ldg(slot + 2 * c + 1);
            const uint32_t ch = __float_as_uint(s1.z);
            if (ch == kEmpty) continue;
            if (!slab_hit(seg, mkf3(s0.x, s0.y, s0.z), mkf3(s0.w, s1.x, s1.y))) continue;
            if (ch & kLeafBit) {
              const int64_t first = (ch >> 3) & 0x0FFFFFFFu;
              const int cnt = (int)(ch & 7u) + 1;
              for (int t = 0; t < cnt; ++t) {
                const float4 r0 = __ldg(T.trirec + 3 * (first + t));
                const float4 r1 = __ldg(T.trirec + 3 * (first + t) + 1);
                const float4 r2 = __ldg(T.trirec + 3 * (first + t) + 2);
                c_tris += 1;
                const int ot = __float_as_int(r2.w);
                if (self_join && ot == os) continue;
                bool ex = false;
                if (!segtri_filtered(p, q, mkf3(r0.x, r0.y, r0.z), mkf3(r0.w, r1.x, r1.y),
                                     mkf3(r1.z, r1.w, r2.x), &ex))
                  continue;
                c_hits += 1;
                const unsigned long long key =
                    dir == 0 ? pair_key(os, ot, self_join) : pair_key(ot, os, self_join);
                if (sink.mode == SINK_HASH) hash_insert(sink, key, st);
                else if (sink.mode == SINK_EMIT) sink.keys[sink.off[sink.base + f] + n_rec] = key;
                ++n_rec;
              }
            } else {
              if (sp >= kDsStack) {
                atomicExch(st + DS_ERR, 1ull);
                sp = 0;
                break;
              }
              stk[sp++] = ch;
            }
          }
        }
      }
    }
    if (sink.mode == SINK_COUNT) sink.cnt[sink.base + f] = n_rec;
  }
  const unsigned long long v[4] = {c_edges, c_nodes, c_tris, c_hits};
  flush_stats(st, v, 4);
}

// Containment rays (Sec. 3.3): thread per object of Q, one ray from its
// first lexicographic vertex through T's BVH along the axis direction that
// leaves T's dataset box soonest (parity is the same in every direction for
// a closed mesh and a point off it).  Only objects whose closed box holds
// the vertex can contain it; up to kParList of them are tracked with a
// parity bit and an on-surface bit.  dir 0: Q = B, T = A; dir 1 the reverse.
template <int W>
__global__ void __launch_bounds__(128) k_ds_parity(DsSide Q, DsSide T, int dir, int self_join,
                                                   Sink sink, Recheck rc, bool first_pass,
                                                   unsigned long long *st) {
  uint32_t stk[kDsStack];
  int lobj[kParList];
  uint8_t lbits[kParList];
  unsigned long long c_rays = 0, c_nodes = 0, c_tris = 0;
  const int SW = node_stride_words(W);
  // T's dataset box: the root's own slot
  const float4 b0 = __ldg(reinterpret_cast<const float4 *>(T.nodes));
  const float4 b1 = __ldg(reinterpret_cast<const float4 *>(T.nodes) + 1);
  const F3 tlo = mkf3(b0.x, b0.y, b0.z), thi = mkf3(b0.w, b1.x, b1.y);
  for (int64_t iq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; iq < Q.M;
       iq += (int64_t)gridDim.x * blockDim.x) {
    int64_t n_rec = 0;
    const float4 q0 = Q.mrec[3 * iq], q1 = Q.mrec[3 * iq + 1], q2 = Q.mrec[3 * iq + 2];
    const F3 vf = mkf3(q0.w, q1.w, q2.x);
    if (vf.x >= tlo.x && vf.x <= thi.x && vf.y >= tlo.y && vf.y <= thi.y && vf.z >= tlo.z &&
        vf.z <= thi.z) {
      c_rays += 1;
      const I3 v = toi(vf);
      int ax, dr;
      ray_axis_choice(vf, tlo, thi, ax, dr);
      int nl = 0;
      bool over = false;
      int sp = 0;
      stk[sp++] = 0u;
      while (sp > 0) {
        const uint32_t node = stk[--sp];
        c_nodes += 1;
        const float4 *slot = reinterpret_cast<const float4 *>(T.nodes + (int64_t)node * SW + 8);
        for (int c = 0; c < W; ++c) {
          const float4 s0 = __ldg(slot + 2 * c), s1 = __ldg(slot + 2 * c + 1);
          const uint32_t ch = __float_as_uint(s1.z);
          if (ch == kEmpty) continue;
          Box bx;
          bx.lo = mkf3(s0.x, s0.y, s0.z);
          bx.hi = mkf3(s0.w, s1.x, s1.y);
          if (!ray_axis_box(vf, bx, ax, dr)) continue;
          if (ch & kLeafBit) {
            const int64_t first = (ch >> 3) & 0x0FFFFFFFu;
            const int cnt = (int)(ch & 7u) + 1;
            for (int t = 0; t < cnt; ++t) {
              const float4 r2 = __ldg(T.trirec + 3 * (first + t) + 2);
              const int ot = __float_as_int(r2.w);
              if (self_join && ot == (int)iq) continue;
              int li = -1;
              for (int j = 0; j < nl; ++j)
                if (lobj[j] == ot) li = j;
              if (li < 0) {
                // an object whose box does not hold the vertex cannot contain it
                const float *ob = T.aabb + 6 * (int64_t)ot;
                if (vf.x < ob[0] || vf.x > ob[3] || vf.y < ob[1] || vf.y > ob[4] || vf.z < ob[2] ||
                    vf.z > ob[5])
                  continue;
                if (nl == kParList) {
                  over = true;
                  continue;
                }
                li = nl++;
                lobj[li] = ot;
                lbits[li] = 0;
              }
              const float4 r0 = __ldg(T.trirec + 3 * (first + t));
              const float4 r1 = __ldg(T.trirec + 3 * (first + t) + 1);
              c_tris += 1;
              const I3 a = toi(mkf3(r0.x, r0.y, r0.z)), b = toi(mkf3(r0.w, r1.x, r1.y));
              const I3 cc = toi(mkf3(r1.z, r1.w, r2.x));
              uint8_t bits = lbits[li];
              if (on_triangle(v, a, b, cc)) bits |= 2;
              if (ray_axis_hit(v, a, b, cc, ax, dr)) bits ^= 1;
              lbits[li] = bits;
            }
          } else {
            if (sp >= kDsStack) {
              atomicExch(st + DS_ERR, 1ull);
              sp = 0;
              break;
            }
            stk[sp++] = ch;
          }
        }
      }
      if (over && first_pass) {
        // every candidate of this object goes to the per-pair join
        const unsigned long long i = atomicAdd(st + DS_NOBJ, 1ull);
        if (i < rc.cap) rc.objs[i] = (int32_t)iq;
        else atomicExch(st + DS_ERR, 2ull);
      }
      for (int j = 0; j < nl; ++j) {
        const int a = dir == 0 ? lobj[j] : (int)iq, b = dir == 0 ? (int)iq : lobj[j];
        if (lbits[j] & 2) {
          // the vertex lies on this object's surface: the pair's own test
          if (first_pass && !over) {
            const unsigned long long i = atomicAdd(st + DS_NREC, 1ull);
            if (i < rc.cap) rc.pairs[i] = make_int2(a, b);
            else atomicExch(st + DS_ERR, 2ull);
          }
        } else if (lbits[j] & 1) {
          const unsigned long long key = pair_key(a, b, self_join);
          if (sink.mode == SINK_HASH) hash_insert(sink, key, st);
          else if (sink.mode == SINK_EMIT) sink.keys[sink.off[sink.base + iq] + n_rec] = key;
          ++n_rec;
        }
      }
    }
    if (sink.mode == SINK_COUNT) sink.cnt[sink.base + iq] = n_rec;
  }
  const unsigned long long v[3] = {c_rays, c_nodes, c_tris};
  unsigned long long w[4] = {0, 0, 0, 0};
  w[0] = v[0];
  flush_stats(st + DS_RAYS, w, 1);
  w[0] = v[1];
  flush_stats(st + DS_NODES, w, 1);
  w[0] = v[2];
  flush_stats(st + DS_TRIS, w, 1);
}

// the occupied slots of a hashmap, in any order
__global__ void k_hash_extract(const unsigned long long *table, int64_t slots,
                               unsigned long long *keys, unsigned long long *n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = table[i];
    const bool has = k != kHashEmpty;
    const unsigned m = __ballot_sync(0xffffffffu, has);
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0 && m) base = atomicAdd(n, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (has) keys[base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = k;
  }
}

__global__ void k_keys_to_pairs(const unsigned long long *keys, const int64_t *n, int32_t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < *n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[2 * i] = (int32_t)(keys[i] >> 32);
    out[2 * i + 1] = (int32_t)(keys[i] & 0xFFFFFFFFull);
  }
}

// the owning mesh of every triangle record of a dataset BVH
__global__ void k_set_owner(float4 *trirec, const int32_t *sorted, const int64_t *toff, int64_t M,
                            int64_t F) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < F;
       s += (int64_t)gridDim.x * blockDim.x)
    trirec[3 * s + 2].w = __int_as_float((int)mesh_of(toff, M, sorted[s]));
}

// The dataset BVH of (W, L): the per-mesh build run on the dataset as a
// single mesh (borrowing its vertex, triangle and edge arrays), then the
// owning meshes written into the triangle records.
static pj_status dataset_bvh(Ctx *ctx, Dataset *ds, int W, int L, cudaStream_t s, Bvh **out) {
  auto it = ds->dbvhs.find({W, L});
  if (it != ds->dbvhs.end()) {
    *out = &it->second;
    return PJ_OK;
  }
  if (ds->F >= (1ll << 28))
    return fail(ctx, PJ_ERR_INVALID_ARG, "dataset too large for the dataset-level BVH (2^28 triangles)");
  Dataset flat;
  flat.M = 1;
  flat.V = ds->V;
  flat.F = ds->F;
  flat.d_xyz = ds->d_xyz;
  flat.d_tris = ds->d_tris;
  flat.d_emask = ds->d_emask;
  flat.h_toff = {0, ds->F};
  flat.h_voff = {0, ds->V};
  float box[6] = {3.4e38f, 3.4e38f, 3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
  for (int64_t m = 0; m < ds->M; ++m)
    for (int d = 0; d < 3; ++d) {
      box[d] = std::min(box[d], ds->h_aabb[6 * m + d]);
      box[3 + d] = std::max(box[3 + d], ds->h_aabb[6 * m + 3 + d]);
    }
  int64_t toff[2] = {0, ds->F};
  PJ_CK(cudaMalloc(&flat.d_toff, sizeof(toff)));
  PJ_CK(cudaMalloc(&flat.d_aabb, sizeof(box)));
  PJ_CK(cudaMemcpyAsync(flat.d_toff, toff, sizeof(toff), cudaMemcpyHostToDevice, s));
  PJ_CK(cudaMemcpyAsync(flat.d_aabb, box, sizeof(box), cudaMemcpyHostToDevice, s));
  pj_status st = build_bvh(ctx, &flat, W, L, s);
  cudaStreamSynchronize(s);
  cudaFree(flat.d_toff);
  cudaFree(flat.d_aabb);
  if (st != PJ_OK) return st;
  Bvh b = flat.bvhs[{W, L}];
  k_set_owner<<<blocks_for(ds->F, 256), 256, 0, s>>>(b.d_trirec, b.d_tri_order, ds->d_toff, ds->M,
                                                     ds->F);
  PJ_CK(cudaGetLastError());
  PJ_CK(cudaStreamSynchronize(s));
  ds->dbvhs[{W, L}] = b;
  *out = &ds->dbvhs[{W, L}];
  return PJ_OK;
}

static DsSide ds_side(Dataset *d, Bvh *b) {
  DsSide x;
  x.xyz = d->d_xyz;
  x.tris = d->d_tris;
  x.emask = d->d_emask;
  x.toff = d->d_toff;
  x.M = d->M;
  x.F = d->F;
  x.mrec = d->d_mrec;
  x.aabb = d->d_aabb;
  x.nodes = b->d_nodes;
  x.trirec = b->d_trirec;
  return x;
}

typedef void (*DsEdgeKernel)(DsSide, DsSide, int, int, Sink, unsigned long long *);
typedef void (*DsParKernel)(DsSide, DsSide, int, int, Sink, Recheck, bool, unsigned long long *);

pj_status run_dataset_join(Ctx *ctx, Dataset *A, Dataset *B, int self_join,
                           const pj_dsjoin_opts *o, pj_pairs *out, pj_dsjoin_stats *stats,
                           cudaStream_t s) {
  const int W = o->width ? o->width : 4, L = o->leaf_size ? o->leaf_size : 2;
  if (!(W == 2 || W == 4 || W == 8) || !(L == 1 || L == 2 || L == 4 || L == 8))
    return fail(ctx, PJ_ERR_INVALID_ARG, "width must be 2, 4 or 8 and leaf size 1, 2, 4 or 8");
  if (o->predicate != PJ_PRED_INTERSECTS && o->predicate != PJ_PRED_OVERLAP)
    return fail(ctx, PJ_ERR_INVALID_ARG, "the dataset-level join evaluates intersects or overlap");
  if (o->materialize < PJ_MAT_ESTIMATED || o->materialize > PJ_MAT_FIXED)
    return fail(ctx, PJ_ERR_INVALID_ARG, "unknown materialisation");
  const bool parity = o->predicate == PJ_PRED_INTERSECTS;
  pj_dsjoin_stats S;
  memset(&S, 0, sizeof(S));
  // events of its own: the estimate and the per-pair join record the
  // context's phase events
  struct Events {
    cudaEvent_t e[6] = {};
    ~Events() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } evs;
  for (auto &x : evs.e) PJ_CK(cudaEventCreate(&x));
  cudaEvent_t *ev = evs.e;
  PJ_CK(cudaEventRecord(ev[0], s));
  // 1. the dataset BVHs (built once per W, L; not part of the timed join)
  Bvh *bA = nullptr, *bB = nullptr;
  pj_status st;
  if ((st = dataset_bvh(ctx, A, W, L, s, &bA)) != PJ_OK) return st;
  if ((st = dataset_bvh(ctx, B, W, L, s, &bB)) != PJ_OK) return st;
  if (1 + (W - 1) * std::max(bA->max_depth, bB->max_depth) > kDsStack)
    return fail(ctx, PJ_ERR_INTERNAL, "dataset BVH too deep for the traversal stack");
  const DsSide sA = ds_side(A, bA), sB = ds_side(B, bB);
  DsEdgeKernel ke = W == 2 ? k_ds_edges<2> : (W == 4 ? k_ds_edges<4> : k_ds_edges<8>);
  DsParKernel kp = W == 2 ? k_ds_parity<2> : (W == 4 ? k_ds_parity<4> : k_ds_parity<8>);
  PJ_CK(cudaEventRecord(ev[1], s));
  // 2. the estimate (sizes the hashmap)
  float ms_est = 0.f;
  int64_t slots = 0;
  if (o->materialize == PJ_MAT_ESTIMATED) {
    pj_estimate e;
    if ((st = run_estimate(ctx, A, B, o->grid, nullptr, &e, s)) != PJ_OK) return st;
    S.estimate = e.e_final;
    ms_est = e.ms;
    slots = (int64_t)std::min(e.slots, 1e12);
  } else if (o->materialize == PJ_MAT_FIXED) {
    slots = o->fixed_slots > 0 ? o->fixed_slots : (int64_t(1) << 26);
  }
  unsigned long long *d_st = (unsigned long long *)ws_get(ctx, "ds_stats", 8 * DS_NSTAT, &st);
  if (!d_st) return st;
  const unsigned long long rc_cap = 1 << 20;
  int2 *rc_pairs = (int2 *)ws_get(ctx, "ds_recheck", sizeof(int2) * rc_cap, &st);
  if (!rc_pairs) return st;
  int32_t *rc_objs = (int32_t *)ws_get(ctx, "ds_recheck_obj", sizeof(int32_t) * rc_cap, &st);
  if (!rc_objs) return st;
  Recheck rc{rc_pairs, rc_objs, rc_cap};
  const int grid = ctx->num_sms * 16;
  // one tracing pass over every item: A's triangles, B's triangles, B's
  // objects, A's objects (count / emit arrays are indexed in this order)
  const int64_t nFA = A->F, nFB = self_join ? 0 : B->F, nMB = parity ? B->M : 0;
  const int64_t nMA = parity && !self_join ? A->M : 0;
  const int64_t items = nFA + nFB + nMB + nMA;
  auto trace = [&](Sink k, bool first_pass) -> pj_status {
    k.base = 0;
    ke<<<grid, 128, 0, s>>>(sA, self_join ? sA : sB, 0, self_join, k, d_st);
    if (!self_join) {
      k.base = nFA;
      ke<<<grid, 128, 0, s>>>(sB, sA, 1, 0, k, d_st);
    }
    if (parity) {
      k.base = nFA + nFB;
      kp<<<grid, 128, 0, s>>>(self_join ? sA : sB, sA, 0, self_join, k, rc, first_pass, d_st);
      if (!self_join) {
        k.base = nFA + nFB + nMB;
        kp<<<grid, 128, 0, s>>>(sA, sB, 1, 0, k, rc, first_pass, d_st);
      }
    }
    ctx->launches += 2 + (self_join ? 0 : 2);
    PJ_CK(cudaGetLastError());
    return PJ_OK;
  };
  unsigned long long h_st[DS_NSTAT];
  unsigned long long *keys = nullptr;
  int64_t n_keys = 0;
  float ms_trace = 0.f;
  if (o->materialize != PJ_MAT_TWO_PASS) {
    // single pass into a hashmap; on overflow twice the slots and again
    // slots rounded up to a power of two (at least 16 for a fixed size,
    // 1,024 for an estimate)
    int64_t cap = o->materialize == PJ_MAT_FIXED ? 16 : 1024;
    while (cap < slots) cap *= 2;
    for (;;) {
      unsigned long long *table =
          (unsigned long long *)ws_get(ctx, "ds_hash", 8 * (size_t)cap, &st);
      if (!table) return st;
      PJ_CK(cudaMemsetAsync(table, 0xff, 8 * (size_t)cap, s));
      PJ_CK(cudaMemsetAsync(d_st, 0, 8 * DS_NSTAT, s));
      PJ_CK(cudaEventRecord(ev[2], s));
      Sink k{SINK_HASH, table, (unsigned long long)(cap - 1), nullptr, nullptr, nullptr, 0};
      if ((st = trace(k, true)) != PJ_OK) return st;
      PJ_CK(cudaEventRecord(ev[4], s));
      PJ_CK(cudaMemcpyAsync(h_st, d_st, sizeof(h_st), cudaMemcpyDeviceToHost, s));
      PJ_CK(cudaStreamSynchronize(s));
      cudaEventElapsedTime(&ms_trace, ev[2], ev[4]);
      if (!h_st[DS_OVERFLOW]) {
        keys = (unsigned long long *)ws_get(ctx, "ds_keys", 8 * (size_t)cap + 8, &st);
        if (!keys) return st;
        unsigned long long *d_n = keys + cap;
        PJ_CK(cudaMemsetAsync(d_n, 0, 8, s));
        k_hash_extract<<<(int)std::min<int64_t>(blocks_for(cap, 256), ctx->num_sms * 16), 256, 0,
                         s>>>(table, cap, keys, d_n);
        ++ctx->launches;
        unsigned long long n = 0;
        PJ_CK(cudaMemcpyAsync(&n, d_n, 8, cudaMemcpyDeviceToHost, s));
        PJ_CK(cudaStreamSynchronize(s));
        n_keys = (int64_t)n;
        S.slots = cap;
        break;
      }
      if (++S.relaunches > 12) return fail(ctx, PJ_ERR_NO_MEMORY, "hashmap overflow after 12 doublings");
      cap *= 2;
    }
  } else {
    // count, prefix sum, emit
    int64_t *cnt = (int64_t *)ws_get(ctx, "ds_count", 8 * (size_t)(items + 1), &st);
    if (!cnt) return st;
    int64_t *off = (int64_t *)ws_get(ctx, "ds_off", 8 * (size_t)(items + 1), &st);
    if (!off) return st;
    PJ_CK(cudaMemsetAsync(d_st, 0, 8 * DS_NSTAT, s));
    PJ_CK(cudaMemsetAsync(cnt + items, 0, 8, s));
    PJ_CK(cudaEventRecord(ev[2], s));
    Sink kc{SINK_COUNT, nullptr, 0, cnt, nullptr, nullptr, 0};
    if ((st = trace(kc, true)) != PJ_OK) return st;
    size_t tb = 0;
    PJ_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, off, (int)(items + 1), s));
    void *tmp = ws_get(ctx, "ds_scan_tmp", tb, &st);
    if (!tmp) return st;
    PJ_CK(cub::DeviceScan::ExclusiveSum(tmp, tb, cnt, off, (int)(items + 1), s));
    int64_t total = 0;
    PJ_CK(cudaMemcpyAsync(&total, off + items, 8, cudaMemcpyDeviceToHost, s));
    PJ_CK(cudaStreamSynchronize(s));
    keys = (unsigned long long *)ws_get(ctx, "ds_keys", 8 * (size_t)std::max<int64_t>(total, 1) + 8, &st);
    if (!keys) return st;
    Sink ke2{SINK_EMIT, nullptr, 0, nullptr, off, keys, 0};
    // the stats count both passes: keep the first pass's
    PJ_CK(cudaMemcpyAsync(h_st, d_st, sizeof(h_st), cudaMemcpyDeviceToHost, s));
    if ((st = trace(ke2, false)) != PJ_OK) return st;
    PJ_CK(cudaEventRecord(ev[4], s));
    PJ_CK(cudaStreamSynchronize(s));
    unsigned long long h2[DS_NSTAT];
    PJ_CK(cudaMemcpyAsync(h2, d_st, sizeof(h2), cudaMemcpyDeviceToHost, s));
    PJ_CK(cudaStreamSynchronize(s));
    h_st[DS_ERR] |= h2[DS_ERR];
    cudaEventElapsedTime(&ms_trace, ev[2], ev[4]);
    n_keys = total;
    S.slots = total;
    ctx->launches += 1;
  }
  if (h_st[DS_ERR] == 1) return fail(ctx, PJ_ERR_INTERNAL, "dataset BVH traversal stack exceeded");
  if (h_st[DS_ERR] == 2) return fail(ctx, PJ_ERR_NO_MEMORY, "too many parity rays to recheck");
  S.edges = (int64_t)h_st[DS_EDGES];
  S.node_visits = (int64_t)h_st[DS_NODES];
  S.tri_tests = (int64_t)h_st[DS_TRIS];
  S.hits = (int64_t)h_st[DS_HITS];
  S.parity_rays = (int64_t)h_st[DS_RAYS];
  // 3. pairs the parity rays left to the per-pair join: candidates of the
  // overflowing objects and the listed pairs, refined by run_join
  std::vector<int32_t> rchk;
  {
    const int64_t np = (int64_t)std::min<unsigned long long>(h_st[DS_NREC], rc_cap);
    const int64_t no = (int64_t)std::min<unsigned long long>(h_st[DS_NOBJ], rc_cap);
    std::vector<int2> hp(np);
    std::vector<int32_t> ho(no);
    if (np) PJ_CK(cudaMemcpyAsync(hp.data(), rc_pairs, sizeof(int2) * np, cudaMemcpyDeviceToHost, s));
    if (no) PJ_CK(cudaMemcpyAsync(ho.data(), rc_objs, sizeof(int32_t) * no, cudaMemcpyDeviceToHost, s));
    PJ_CK(cudaStreamSynchronize(s));
    for (auto &p : hp) {
      int a = p.x, b = p.y;
      if (self_join && a > b) std::swap(a, b);
      rchk.push_back(a);
      rchk.push_back(b);
    }
    // an overflowing object: its bounding-box candidates on the other side.
    // (Object ids from both directions share this list; the kernels of one
    // direction write ids of their own casting side, told apart here by
    // trying both sides' boxes, which only adds candidates.)
    auto meet = [](const float *x, const float *y) {
      return x[0] <= y[3] && y[0] <= x[3] && x[1] <= y[4] && y[1] <= x[4] && x[2] <= y[5] &&
             y[2] <= x[5];
    };
    for (int32_t q : ho) {
      if (q < B->M)
        for (int64_t i = 0; i < A->M; ++i)
          if (meet(&A->h_aabb[6 * i], &B->h_aabb[6 * (int64_t)q])) {
            int a = (int)i, b = q;
            if (self_join && a > b) std::swap(a, b);
            if (!(self_join && a == b)) {
              rchk.push_back(a);
              rchk.push_back(b);
            }
          }
      if (!self_join && q < A->M)
        for (int64_t j = 0; j < B->M; ++j)
          if (meet(&A->h_aabb[6 * (int64_t)q], &B->h_aabb[6 * j])) {
            rchk.push_back(q);
            rchk.push_back((int)j);
          }
    }
  }
  std::vector<unsigned long long> extra;
  S.recheck_pairs = (int64_t)rchk.size() / 2;
  if (!rchk.empty()) {
    pj_join_opts po{};
    po.width = W;
    po.leaf_size = L;
    po.out_host = 1;
    // the per-pair join needs both datasets' per-mesh BVH of this shape
    for (Dataset *D : {A, B})
      if (D->bvhs.find({W, L}) == D->bvhs.end()) {
        if ((st = build_bvh(ctx, D, W, L, s)) != PJ_OK) return st;
      }
    pj_pairs r;
    memset(&r, 0, sizeof(r));
    if ((st = run_join(ctx, A, B, rchk.data(), nullptr, (int64_t)rchk.size() / 2, 0, 0, &po, s,
                       &r)) != PJ_OK)
      return st;
    for (int64_t k = 0; k < r.count; ++k)
      extra.push_back(((unsigned long long)(unsigned)r.pairs[2 * k] << 32) |
                      (unsigned)r.pairs[2 * k + 1]);
    pairs_release(ctx, &r);
  }
  // 4. sort and unique (with the rechecked pairs), then (idA, idB)
  PJ_CK(cudaEventRecord(ev[5], s));
  const int64_t n_all = n_keys + (int64_t)extra.size();
  unsigned long long *k2 = (unsigned long long *)ws_get(ctx, "ds_keys2", 8 * (size_t)std::max<int64_t>(n_all, 1), &st);
  if (!k2) return st;
  unsigned long long *k3 = (unsigned long long *)ws_get(ctx, "ds_keys3", 8 * (size_t)std::max<int64_t>(n_all, 1), &st);
  if (!k3) return st;
  if (!extra.empty()) {
    // the traced keys and the rechecked pairs in one buffer
    unsigned long long *k1 = (unsigned long long *)ws_get(ctx, "ds_keys1", 8 * (size_t)n_all, &st);
    if (!k1) return st;
    if (n_keys > 0)
      PJ_CK(cudaMemcpyAsync(k1, keys, 8 * (size_t)n_keys, cudaMemcpyDeviceToDevice, s));
    PJ_CK(cudaMemcpyAsync(k1 + n_keys, extra.data(), 8 * extra.size(), cudaMemcpyHostToDevice, s));
    PJ_CK(cudaStreamSynchronize(s));  // extra is a host vector
    keys = k1;
  }
  int64_t *d_nu = (int64_t *)ws_get(ctx, "ds_nunique", 8, &st);
  if (!d_nu) return st;
  int64_t K = 0;
  if (n_all > 0) {
    size_t tb = 0, tb2 = 0;
    PJ_CK(cub::DeviceRadixSort::SortKeys(nullptr, tb, keys, k2, (int)n_all, 0, 64, s));
    PJ_CK(cub::DeviceSelect::Unique(nullptr, tb2, k2, k3, d_nu, (int)n_all, s));
    void *tmp = ws_get(ctx, "ds_sort_tmp", std::max(tb, tb2), &st);
    if (!tmp) return st;
    PJ_CK(cub::DeviceRadixSort::SortKeys(tmp, tb, keys, k2, (int)n_all, 0, 64, s));
    PJ_CK(cub::DeviceSelect::Unique(tmp, tb2, k2, k3, d_nu, (int)n_all, s));
    PJ_CK(cudaMemcpyAsync(&K, d_nu, 8, cudaMemcpyDeviceToHost, s));
    PJ_CK(cudaStreamSynchronize(s));
  }
  cudaError_t pe;
  int32_t *d_out = (int32_t *)pool_get(ctx, 8 * (size_t)std::max<int64_t>(K, 1), &pe);
  PJ_CK(pe);
  if (K > 0) {
    k_keys_to_pairs<<<(int)std::min<int64_t>(blocks_for(K, 256), ctx->num_sms * 8), 256, 0, s>>>(
        k3, d_nu, d_out);
    ++ctx->launches;
  }
  PJ_CK(cudaEventRecord(ev[3], s));
  PJ_CK(cudaStreamSynchronize(s));
  memset(out, 0, sizeof(*out));
  out->count = K;
  out->n_candidates = 0;
  if (o->out_host) {
    PJ_CK(cudaMallocHost((void **)&out->pairs, 8 * (size_t)std::max<int64_t>(K, 1)));
    if (K > 0) PJ_CK(cudaMemcpy(out->pairs, d_out, 8 * (size_t)K, cudaMemcpyDeviceToHost));
    pool_put(ctx, d_out);
    out->on_device = 0;
  } else {
    out->pairs = d_out;
    out->on_device = 1;
  }
  float ms_all = 0.f, ms_mat = 0.f;
  cudaEventElapsedTime(&ms_all, ev[1], ev[3]);
  cudaEventElapsedTime(&ms_mat, ev[5], ev[3]);
  out->device_ms = ms_all;
  S.ms_total = ms_all;
  S.ms_estimate = ms_est;
  S.ms_trace = ms_trace;
  S.ms_materialize = ms_mat;
  if (stats) *stats = S;
  return PJ_OK;
}

}  // namespace pj
