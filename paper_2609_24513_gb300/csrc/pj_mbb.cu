// Bounding-box filter join by sort and sweep (Sec. 3.1, the filter step: the
// candidate pairs are the mesh pairs whose closed boxes overlap).
//
// For joins whose all-pairs count is large (tens of thousands of meshes a
// side) testing every pair costs more than the refinement; here the boxes of
// both sides are sorted by their low x, and each box is tested only against
// the boxes after it in that order whose low x does not pass its high x --
// every pair of boxes that overlap on x meets exactly once that way, from
// the one that comes first.  The forward ranges are cut into chunks of 32
// boxes, one per warp step, spread evenly over the warps (a long box's range
// does not serialise on one warp).  A count pass, a scan and an emit pass
// write the pairs; a radix sort puts them in (id A, id B) order, the order of
// the all-pairs join, so that every later step sees the same candidate list.
#include <cub/cub.cuh>

#include "pj_internal.cuh"

namespace pj {

constexpr int SW_T = 256;

// the sort key of a non-negative float is its bit pattern (coordinates lie
// in [0, 2^18), so box bounds are never negative)
__global__ void k_sw_keys(const float *aabbA, int64_t MA, const float *aabbB, int64_t MB,
                          uint32_t *key, int32_t *val) {
  const int64_t n = MA + MB;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float *b = i < MA ? aabbA + 6 * i : aabbB + 6 * (i - MA);
    key[i] = __float_as_uint(b[0]);
    val[i] = (int32_t)i;
  }
}

// sorted boxes, two float4 each: (lo x, lo y, lo z, hi x), (hi y, hi z, id, 0)
// with id < MA for side A and MA + j for mesh j of side B
__global__ void k_sw_gather(const int32_t *val, int64_t n, const float *aabbA, int64_t MA,
                            const float *aabbB, float4 *sb) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = val[p];
    const float *b = v < MA ? aabbA + 6 * (int64_t)v : aabbB + 6 * ((int64_t)v - MA);
    sb[2 * p] = make_float4(b[0], b[1], b[2], b[3]);
    sb[2 * p + 1] = make_float4(b[4], b[5], __int_as_float(v), 0.f);
  }
}

// the end of box p's forward range (the first later box whose low x passes
// p's high x) and its number of 32-box chunks
__global__ void k_sw_range(const float4 *sb, int64_t n, int64_t *ends, int64_t *chunks) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float hx = sb[2 * p].w;
    int64_t lo = p + 1, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (sb[2 * mid].x <= hx) lo = mid + 1;
      else hi = mid;
    }
    ends[p] = lo;
    chunks[p] = (lo - p - 1 + 31) / 32;
  }
}

// Warp w takes chunks [w T / nw, (w + 1) T / nw); chunk t belongs to the box p
// with coff[p] <= t < coff[p + 1] and covers boxes p + 1 + 32 (t - coff[p]) +
// lane.  Without EMIT: the chunk's pair count; with EMIT: the pairs, as keys
// (id A << 32 | id B) at the chunk's offset.
template <bool EMIT>
__global__ void __launch_bounds__(SW_T) k_sw_pairs(const float4 *sb, int64_t n, const int64_t *coff,
                                                   const int64_t *ends, int64_t T, int64_t MA,
                                                   int self_join, int64_t *cnt,
                                                   const int64_t *off, uint64_t *keys) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (SW_T / 32);
  const int64_t w = blockIdx.x * (int64_t)(SW_T / 32) + (threadIdx.x >> 5);
  const int64_t t0 = w * T / nw, t1 = (w + 1) * T / nw;
  if (t0 >= t1) return;
  // the box of chunk t0: the last p with coff[p] <= t0
  int64_t p = 0;
  if (lane == 0) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (coff[mid] <= t0) lo = mid;
      else hi = mid - 1;
    }
    p = lo;
  }
  p = __shfl_sync(0xFFFFFFFFu, p, 0);
  int64_t cb = coff[p], ce = p + 1 < n ? coff[p + 1] : T;
  for (int64_t t = t0; t < t1; ++t) {
    while (t >= ce) {  // boxes with empty ranges have no chunks
      ++p;
      cb = ce;
      ce = p + 1 < n ? coff[p + 1] : T;
    }
    const float4 P0 = sb[2 * p], P1 = sb[2 * p + 1];
    const int64_t q = p + 1 + 32 * (t - cb) + lane;
    bool hit = false;
    int32_t vp = __float_as_int(P1.z), vq = 0;
    if (q < ends[p]) {
      // x overlaps: P0.x <= lo x of q (sorted) <= P0.w (in the range)
      const float4 Q0 = sb[2 * q], Q1 = sb[2 * q + 1];
      vq = __float_as_int(Q1.z);
      const bool sides = self_join ? true : ((vp < MA) != (vq < MA));
      hit = sides && P0.y <= Q1.x && Q0.y <= P1.x && P0.z <= Q1.y && Q0.z <= P1.y;
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, hit);
    if (!EMIT) {
      if (lane == 0) cnt[t] = __popc(m);
    } else if (hit) {
      const int64_t pos = off[t] + __popc(m & ((1u << lane) - 1u));
      uint32_t a, b;
      if (self_join) {
        a = (uint32_t)min(vp, vq);
        b = (uint32_t)max(vp, vq);
      } else {
        a = (uint32_t)(vp < MA ? vp : vq);
        b = (uint32_t)((vp < MA ? vq : vp) - MA);
      }
      keys[pos] = ((uint64_t)a << 32) | b;
    }
  }
}

__global__ void k_sw_unpack(const uint64_t *keys, int64_t n, int32_t *cand) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    cand[2 * i] = (int32_t)(k >> 32);
    cand[2 * i + 1] = (int32_t)(k & 0xFFFFFFFFu);
  }
}

pj_status mbb_sweep(Ctx *ctx, const Dataset *A, const Dataset *B, bool self_join,
                    cudaStream_t s, int64_t *d_count, int32_t **d_cand, int64_t *C) {
  *d_cand = nullptr;
  *C = 0;
  const int64_t MA = A->M, MB = self_join ? 0 : B->M, n = MA + MB;
  pj_status st = PJ_OK;
  int64_t *h = (int64_t *)cur_exec(ctx)->h_pinned;  // pinned: the two totals
  auto get = [&](const char *name, size_t bytes) { return ws_get(ctx, name, bytes, &st); };
  auto cand_ws = [&](int64_t c) -> pj_status {
    *d_cand = (int32_t *)get("cand", sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(c, 1));
    return *d_cand ? PJ_OK : st;
  };
  // no pairs: the device count (read by every later kernel) is zero
  auto none = [&]() -> pj_status {
    PJ_CK(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
    return cand_ws(0);
  };
  if (n < 2) return none();
  const int grid = std::min(blocks_for(n, SW_T), ctx->num_sms * 16);
  uint32_t *k0 = (uint32_t *)get("sw_k0", 4 * (size_t)n);
  uint32_t *k1 = (uint32_t *)get("sw_k1", 4 * (size_t)n);
  int32_t *v0 = (int32_t *)get("sw_v0", 4 * (size_t)n);
  int32_t *v1 = (int32_t *)get("sw_v1", 4 * (size_t)n);
  float4 *sb = (float4 *)get("sw_boxes", 32 * (size_t)n);
  int64_t *ends = (int64_t *)get("sw_ends", 8 * (size_t)n);
  int64_t *chunks = (int64_t *)get("sw_chunks", 8 * (size_t)n);
  int64_t *coff = (int64_t *)get("sw_coff", 8 * (size_t)n);
  int64_t *tot = (int64_t *)get("sw_total", 8);
  if (!k0 || !k1 || !v0 || !v1 || !sb || !ends || !chunks || !coff || !tot) return st;
  k_sw_keys<<<grid, SW_T, 0, s>>>(A->d_aabb, MA, self_join ? nullptr : B->d_aabb, MB, k0, v0);
  size_t tb = 0;
  PJ_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, k0, k1, v0, v1, (int)n, 0, 32, s));
  void *tmp = get("sw_sort", tb);
  if (!tmp) return st;
  PJ_CK(cub::DeviceRadixSort::SortPairs(tmp, tb, k0, k1, v0, v1, (int)n, 0, 32, s));
  k_sw_gather<<<grid, SW_T, 0, s>>>(v1, n, A->d_aabb, MA, self_join ? nullptr : B->d_aabb, sb);
  k_sw_range<<<grid, SW_T, 0, s>>>(sb, n, ends, chunks);
  ctx->launches += 4;
  PJ_CK(cudaGetLastError());
  if ((st = scan_i64(ctx, chunks, coff, n, tot, s)) != PJ_OK) return st;
  PJ_CK(cudaMemcpyAsync(h, tot, 8, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  const int64_t T = h[0];
  if (T == 0) return none();
  int64_t *cnt = (int64_t *)get("sw_cnt", 8 * (size_t)T);
  int64_t *off = (int64_t *)get("sw_off", 8 * (size_t)T);
  if (!cnt || !off) return st;
  const int pgrid = (int)std::min<int64_t>((T + SW_T / 32 - 1) / (SW_T / 32),
                                           (int64_t)ctx->num_sms * 16);
  k_sw_pairs<false><<<pgrid, SW_T, 0, s>>>(sb, n, coff, ends, T, MA, self_join ? 1 : 0, cnt,
                                           nullptr, nullptr);
  ++ctx->launches;
  PJ_CK(cudaGetLastError());
  // the pair count goes to the device count word itself
  if ((st = scan_i64(ctx, cnt, off, T, d_count, s)) != PJ_OK) return st;
  PJ_CK(cudaMemcpyAsync(h + 1, d_count, 8, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  const int64_t c = h[1];
  if (c > INT32_MAX) return fail(ctx, PJ_ERR_NO_MEMORY, "more than 2^31 candidate pairs");
  if ((st = cand_ws(c)) != PJ_OK) return st;
  *C = c;
  if (c == 0) return PJ_OK;
  uint64_t *q0 = (uint64_t *)get("sw_q0", 8 * (size_t)c);
  uint64_t *q1 = (uint64_t *)get("sw_q1", 8 * (size_t)c);
  if (!q0 || !q1) return st;
  k_sw_pairs<true><<<pgrid, SW_T, 0, s>>>(sb, n, coff, ends, T, MA, self_join ? 1 : 0, nullptr,
                                          off, q0);
  size_t tb2 = 0;
  PJ_CK(cub::DeviceRadixSort::SortKeys(nullptr, tb2, q0, q1, (int)c, 0, 63, s));
  void *tmp2 = get("sw_sort", std::max(tb, tb2));
  if (!tmp2) return st;
  PJ_CK(cub::DeviceRadixSort::SortKeys(tmp2, tb2, q0, q1, (int)c, 0, 63, s));
  k_sw_unpack<<<std::min(blocks_for(c, SW_T), ctx->num_sms * 16), SW_T, 0, s>>>(q1, c, *d_cand);
  ctx->launches += 2;
  PJ_CK(cudaGetLastError());
  return PJ_OK;
}

}  // namespace pj
