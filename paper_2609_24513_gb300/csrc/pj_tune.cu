// Autotuner: picks BVH width, leaf size, warps per pair and the depth of the
// breadth-first front end for one dataset pair by timing joins on a seeded
// calibration sample of its candidates (median of a few repeats, CUDA
// events inside the join).  The paper fixes these through OptiX; on GB300
// they trade node-fetch width against traversal depth and lane utilisation,
// and the best point depends on the meshes.
#include <algorithm>
#include <cstring>
#include <random>
#include <set>
#include <vector>

#include "pj_internal.cuh"

namespace pj {

static pj_status candidates_to_host(Ctx *ctx, Dataset *A, Dataset *B, int self_join,
                                    std::vector<int32_t> &out) {
  // the bounding-box candidates, listed on the host from the per-mesh boxes
  // computed at load time (the tuner only draws a sample from them)
  std::vector<float> ha(6 * A->M), hb(6 * B->M);
  cudaError_t e = cudaMemcpy(ha.data(), A->d_aabb, 4 * ha.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hb.data(), B->d_aabb, 4 * hb.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune: mesh boxes");
  out.clear();
  for (int64_t i = 0; i < A->M; ++i) {
    const float *x = &ha[6 * i];
    for (int64_t j = self_join ? i + 1 : 0; j < B->M; ++j) {
      const float *y = &hb[6 * j];
      if (x[0] <= y[3] && y[0] <= x[3] && x[1] <= y[4] && y[1] <= x[4] && x[2] <= y[5] &&
          y[2] <= x[5]) {
        out.push_back((int32_t)i);
        out.push_back((int32_t)j);
      }
    }
  }
  return PJ_OK;
}

pj_status run_autotune(Ctx *ctx, Dataset *A, Dataset *B, const int32_t *cand, int64_t n_cand,
                       int self_join, const pj_tune_space *sp, pj_join_opts *best,
                       pj_tune_entry *table, int table_cap, int *table_n) {
  *table_n = 0;
  auto check_list = [&](const int32_t *v, int n, std::initializer_list<int> ok) -> bool {
    if (n < 1) return false;
    for (int k = 0; k < n; ++k)
      if (std::find(ok.begin(), ok.end(), v[k]) == ok.end()) return false;
    return true;
  };
  if (sp->n_widths > 3 || sp->n_leaf_sizes > 4 || sp->n_warps > 3 || sp->n_wave_levels > 4 ||
      !check_list(sp->widths, sp->n_widths, {2, 4, 8}) ||
      !check_list(sp->leaf_sizes, sp->n_leaf_sizes, {1, 2, 4, 8}) ||
      !check_list(sp->warps, sp->n_warps, {1, 2, 4}) || sp->n_wave_levels < 1)
    return fail(ctx, PJ_ERR_INVALID_ARG, "autotune: bad tuning space");
  // candidate list and calibration sample
  std::vector<int32_t> all;
  if (n_cand >= 0) {
    all.assign(cand, cand + 2 * n_cand);
  } else {
    pj_status st = candidates_to_host(ctx, A, B, self_join, all);
    if (st != PJ_OK) return st;
  }
  const int64_t n = (int64_t)all.size() / 2;
  if (n == 0) return fail(ctx, PJ_ERR_INVALID_ARG, "autotune: no candidates");
  const int permille = sp->sample_permille > 0 ? sp->sample_permille : 20;
  int64_t m = std::max<int64_t>(std::min<int64_t>(n, 1000), n * permille / 1000);
  m = std::min(m, n);
  std::vector<int64_t> idx(n);
  for (int64_t k = 0; k < n; ++k) idx[k] = k;
  std::mt19937_64 rng(sp->seed);
  for (int64_t k = 0; k < m; ++k) {  // partial Fisher-Yates
    std::uniform_int_distribution<int64_t> d(k, n - 1);
    std::swap(idx[k], idx[d(rng)]);
  }
  std::sort(idx.begin(), idx.begin() + m);
  std::vector<int32_t> sample(2 * m);
  for (int64_t k = 0; k < m; ++k) {
    sample[2 * k] = all[2 * idx[k]];
    sample[2 * k + 1] = all[2 * idx[k] + 1];
  }
  const int repeats = sp->repeats > 0 ? sp->repeats : 3;
  // BVH shapes that exist before tuning stay; new losers are freed
  std::set<std::pair<int, int>> had_a, had_b;
  for (auto &kv : A->bvhs) had_a.insert(kv.first);
  for (auto &kv : B->bvhs) had_b.insert(kv.first);
  const std::pair<int, int> last_a = A->last_bvh, last_b = B->last_bvh;
  float best_ms = 3e38f;
  pj_join_opts win{};
  int count = 0;
  pj_status result = PJ_OK;
  for (int wi = 0; wi < sp->n_widths && result == PJ_OK; ++wi) {
    for (int li = 0; li < sp->n_leaf_sizes && result == PJ_OK; ++li) {
      const int W = sp->widths[wi], L = sp->leaf_sizes[li];
      if (!A->bvhs.count({W, L})) result = build_bvh(ctx, A, W, L, ctx->stream);
      if (result == PJ_OK && B != A && !B->bvhs.count({W, L}))
        result = build_bvh(ctx, B, W, L, ctx->stream);
      if (result != PJ_OK) break;
      for (int ki = 0; ki < sp->n_warps && result == PJ_OK; ++ki) {
        for (int vi = 0; vi < sp->n_wave_levels && result == PJ_OK; ++vi) {
          pj_join_opts o{};
          o.width = W;
          o.leaf_size = L;
          o.warps_per_pair = sp->warps[ki];
          o.wave_levels = sp->wave_levels[vi];
          o.use_graph = 0;
          std::vector<float> t;
          for (int r = 0; r <= repeats; ++r) {
            pj_pairs res;
            memset(&res, 0, sizeof(res));
            result = run_join(ctx, A, B, sample.data(), nullptr, m, 0, self_join, &o,
                              ctx->stream, &res);
            if (result != PJ_OK) break;
            if (r > 0) t.push_back(res.device_ms);  // the first run warms up
            pairs_release(ctx, &res);
          }
          if (result != PJ_OK) break;
          std::sort(t.begin(), t.end());
          const float ms = t[t.size() / 2];
          if (count < table_cap) {
            pj_tune_entry &e = table[count];
            e.width = W;
            e.leaf_size = L;
            e.warps_per_pair = o.warps_per_pair;
            e.wave_levels = o.wave_levels;
            e.ms = ms;
            e.reserved = 0.f;
          }
          ++count;
          if (ms < best_ms) {
            best_ms = ms;
            win = o;
          }
        }
      }
    }
  }
  *table_n = std::min(count, table_cap);
  // free the shapes built here that lost; keep the winner as the default
  for (Dataset *D : {A, B}) {
    const auto &had = D == A ? had_a : had_b;
    for (auto it = D->bvhs.begin(); it != D->bvhs.end();) {
      const bool keep = had.count(it->first) ||
                        (result == PJ_OK && it->first == std::make_pair((int)win.width, (int)win.leaf_size));
      if (!keep) {
        free_bvh(it->second);
        it = D->bvhs.erase(it);
      } else {
        ++it;
      }
    }
  }
  for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
  ctx->graphs.clear();
  if (result != PJ_OK) {
    A->last_bvh = last_a;
    B->last_bvh = last_b;
    return result;
  }
  A->last_bvh = B->last_bvh = {win.width, win.leaf_size};
  *best = win;
  return PJ_OK;
}

}  // namespace pj
