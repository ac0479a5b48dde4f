// Selectivity estimate of a join on the device (paper Sec. 3.5, "Result
// Materialization"): the expected number of intersecting object pairs, from
// per-cell statistics of a regular grid laid over both datasets.  It sizes
// the deduplicating hashmap of the dataset-level join (pj_dataset_join).
//
// Per cell and dataset k: N_k objects whose closed box touches the cell, S_k
// their mean box side (the three extents averaged), VolRatio_k their mean
// mesh-to-box volume ratio.  Two objects are treated as cubes of the mean
// sides; their centres fall in the interaction volume (S_1 + S_2 + eps)^3
// (the Minkowski sum of the two cubes) with probability P_base = V_int /
// V_cell; the shape factor (sqrt(VolRatio_1 VolRatio_2))^gamma discounts
// boxes that are mostly empty; P = min(P_base F_shape, 1), E_i = N_1 N_2 P,
// E_final = sum of E_i over the cells.
//
// Readings (the paper leaves them open): lengths in units of the grid's full
// extent (coordinates / (2^18 - 1)); the grid spans the box of both datasets
// in G^3 equal cells; "touches" is closed; a mesh's volume is the
// divergence-theorem sum |sum det[a, b, c]| / 6 in float64, after shifting
// the mesh by its first vertex.
#include <algorithm>
#include <cmath>

#include "pj_internal.cuh"

namespace pj {

constexpr double kQ = 262143.0;  // 2^18 - 1

// one warp per mesh: |sum over triangles of (a - p0) . ((b - p0) x (c - p0))| / 6
__global__ void k_mesh_volume(const float *xyz, const int32_t *tris, const int64_t *voff,
                              const int64_t *toff, int64_t M, double *vol) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t m = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); m < M;
       m += warps) {
    const float *p0 = xyz + 3 * voff[m];
    const double ox = p0[0], oy = p0[1], oz = p0[2];
    double s = 0.0;
    for (int64_t f = toff[m] + lane; f < toff[m + 1]; f += 32) {
      const float *a = xyz + 3 * (int64_t)tris[3 * f], *b = xyz + 3 * (int64_t)tris[3 * f + 1];
      const float *c = xyz + 3 * (int64_t)tris[3 * f + 2];
      const double ax = a[0] - ox, ay = a[1] - oy, az = a[2] - oz;
      const double bx = b[0] - ox, by = b[1] - oy, bz = b[2] - oz;
      const double cx = c[0] - ox, cy = c[1] - oy, cz = c[2] - oz;
      s += ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) vol[m] = fabs(s) / 6.0;
  }
}

struct Grid {
  double g0[3], cw[3];
  int G;
};

// one thread per mesh: every cell its closed box touches gets N += 1,
// S += the mean box side, R += the volume ratio
__global__ void k_cell_stats(const float *aabb, const double *vol, int64_t M, Grid g,
                             unsigned long long *N, double *S, double *R) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
       m += (int64_t)gridDim.x * blockDim.x) {
    double lo[3], hi[3], ext[3];
    int i0[3], i1[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = aabb[6 * m + d] / kQ;
      hi[d] = aabb[6 * m + 3 + d] / kQ;
      ext[d] = hi[d] - lo[d];
      i0[d] = (int)fmin(fmax(floor((lo[d] - g.g0[d]) / g.cw[d]), 0.0), (double)(g.G - 1));
      i1[d] = (int)fmin(fmax(floor((hi[d] - g.g0[d]) / g.cw[d]), 0.0), (double)(g.G - 1));
    }
    const double side = (ext[0] + ext[1] + ext[2]) / 3.0;
    const double box = ext[0] * ext[1] * ext[2];
    const double ratio = box > 0.0 ? vol[m] / (kQ * kQ * kQ) / box : 0.0;
    for (int x = i0[0]; x <= i1[0]; ++x)
      for (int y = i0[1]; y <= i1[1]; ++y)
        for (int z = i0[2]; z <= i1[2]; ++z) {
          const int64_t c = ((int64_t)x * g.G + y) * g.G + z;
          atomicAdd(N + c, 1ull);
          atomicAdd(S + c, side);
          atomicAdd(R + c, ratio);
        }
  }
}

// per cell: E_i = N_1 N_2 min(P_base F_shape, 1); their sum and the number of
// cells holding objects of both datasets
__global__ void k_cell_estimate(const unsigned long long *N1, const double *S1, const double *R1,
                                const unsigned long long *N2, const double *S2, const double *R2,
                                int64_t cells, double v_cell, double eps, double gamma,
                                double *E, double *sum, unsigned long long *occupied) {
  double acc = 0.0;
  unsigned long long occ = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    double e = 0.0;
    if (N1[c] > 0 && N2[c] > 0) {
      const double n1 = (double)N1[c], n2 = (double)N2[c];
      const double m1 = S1[c] / n1, m2 = S2[c] / n2, r1 = R1[c] / n1, r2 = R2[c] / n2;
      const double s = m1 + m2 + eps;
      const double p_base = s * s * s / v_cell;
      const double f_shape = pow(sqrt(r1 * r2), gamma);
      e = n1 * n2 * fmin(p_base * f_shape, 1.0);
      occ += 1;
    }
    if (E) E[c] = e;
    acc += e;
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    occ += __shfl_xor_sync(0xffffffffu, occ, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sum, acc);
    atomicAdd(occupied, occ);
  }
}

pj_status run_estimate(Ctx *ctx, Dataset *A, Dataset *B, int G, double *cells_out,
                       pj_estimate *out, cudaStream_t s) {
  if (G <= 0) G = 16;
  if (G > 256) return fail(ctx, PJ_ERR_INVALID_ARG, "grid must be at most 256 cells per axis");
  if (A->M == 0 || B->M == 0) {
    memset(out, 0, sizeof(*out));
    out->grid = G;
    return PJ_OK;
  }
  // the grid over both datasets' boxes (host copies of the mesh boxes)
  Grid g;
  g.G = G;
  for (int d = 0; d < 3; ++d) {
    double lo = 1e300, hi = -1e300;
    for (const Dataset *D : {A, B})
      for (int64_t m = 0; m < D->M; ++m) {
        lo = std::min(lo, D->h_aabb[6 * m + d] / kQ);
        hi = std::max(hi, D->h_aabb[6 * m + 3 + d] / kQ);
      }
    g.g0[d] = lo;
    g.cw[d] = std::max(hi - lo, 1.0 / kQ) / G;
  }
  const int64_t cells = (int64_t)G * G * G;
  pj_status st;
  // one buffer: the two volume arrays, then per dataset N, S, R, then E, sum, occupied
  const size_t bytes = 8 * ((size_t)A->M + (size_t)B->M + 6 * (size_t)cells + 2 * (size_t)cells + 2);
  char *buf = (char *)ws_get(ctx, "estimate", bytes, &st);
  if (!buf) return st;
  double *volA = (double *)buf, *volB = volA + A->M;
  unsigned long long *N1 = (unsigned long long *)(volB + B->M);
  double *S1 = (double *)(N1 + cells), *R1 = S1 + cells;
  unsigned long long *N2 = (unsigned long long *)(R1 + cells);
  double *S2 = (double *)(N2 + cells), *R2 = S2 + cells;
  double *E = R2 + cells, *sum = E + cells;
  unsigned long long *occ = (unsigned long long *)(sum + 1);
  cudaEvent_t *ev = cur_exec(ctx)->ev;
  PJ_CK(cudaEventRecord(ev[0], s));
  PJ_CK(cudaMemsetAsync(N1, 0, 8 * (6 * (size_t)cells + 2 * (size_t)cells + 2), s));
  const int vb = (int)std::min<int64_t>((std::max(A->M, B->M) + 7) / 8, (int64_t)ctx->num_sms * 32);
  k_mesh_volume<<<vb, 256, 0, s>>>(A->d_xyz, A->d_tris, A->d_voff, A->d_toff, A->M, volA);
  k_mesh_volume<<<vb, 256, 0, s>>>(B->d_xyz, B->d_tris, B->d_voff, B->d_toff, B->M, volB);
  k_cell_stats<<<blocks_for(A->M, 128), 128, 0, s>>>(A->d_aabb, volA, A->M, g, N1, S1, R1);
  k_cell_stats<<<blocks_for(B->M, 128), 128, 0, s>>>(B->d_aabb, volB, B->M, g, N2, S2, R2);
  const double v_cell = g.cw[0] * g.cw[1] * g.cw[2];
  k_cell_estimate<<<(int)std::min<int64_t>(blocks_for(cells, 256), ctx->num_sms * 8), 256, 0, s>>>(
      N1, S1, R1, N2, S2, R2, cells, v_cell, 1e-3, 0.8, E, sum, occ);
  ctx->launches += 5;
  PJ_CK(cudaGetLastError());
  PJ_CK(cudaEventRecord(ev[3], s));
  double h[2];
  PJ_CK(cudaMemcpyAsync(h, sum, 16, cudaMemcpyDeviceToHost, s));
  if (cells_out) PJ_CK(cudaMemcpyAsync(cells_out, E, 8 * (size_t)cells, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  memset(out, 0, sizeof(*out));
  out->e_final = h[0];
  out->slots = h[0] / 0.5;
  unsigned long long o;
  memcpy(&o, &h[1], 8);
  out->cells_occupied = (int64_t)o;
  out->grid = G;
  cudaEventElapsedTime(&out->ms, ev[0], ev[3]);
  return PJ_OK;
}

}  // namespace pj
