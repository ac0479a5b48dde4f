// Out-of-core execution by grid tiling (paper Sec. 3.6, "Out-of-GPU-core
// execution"): the datasets stay in host memory; a coarse grid partitions
// their joint box, every mesh is copied to each cell its closed box touches,
// and the cells are joined one after another with the library's own load,
// BVH build and join.  The paper leaves this to future work and notes that
// only the partitioning and the cell loop are new; that is all this file
// adds.
//
// Each overlapping pair (i, j) is reported in every cell holding both meshes;
// it is kept only in the cell holding its reference point r = the lower
// corner of box(i) and box(j)'s intersection (r lies in both boxes, so both
// meshes were copied to r's cell), which leaves each pair exactly once with
// no global deduplication.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <future>
#include <vector>

#include "pj_internal.cuh"

namespace pj {

namespace {

struct HostSet {
  const pj_host_meshes *m;
  std::vector<float> box;       // 6 per mesh
  std::vector<int64_t> bytes;   // device footprint estimate per mesh
};

// a closed-box grid of G cells per axis over [g0, g0 + G cw]
struct TGrid {
  double g0[3], cw[3];
  int G;
  int idx(double x, int d) const {
    const double c = std::floor((x - g0[d]) / cw[d]);
    return (int)std::min(std::max(c, 0.0), (double)(G - 1));
  }
};

// Device bytes of one mesh once loaded and indexed: vertices, triangles,
// the lexicographic order and per-mesh records, triangle records and sorted
// order, about one W-wide node per L (W - 1) triangles, plus the load and
// build temporaries (sort keys and binary-tree arrays, about 100 B a
// triangle while they live).
int64_t mesh_bytes(int64_t nv, int64_t nf, int W, int L) {
  const int64_t nodes = nf / std::max(1, L * (W - 1)) + 2;
  return nv * 16 + nf * (12 + 1 + 48 + 4 + 100) + nodes * 32 * (W + 1) + 256;
}

pj_status prepare(Ctx *ctx, const pj_host_meshes *m, int W, int L, HostSet &h) {
  if (!m || !m->xyz || !m->tris || !m->mesh_vert_off || !m->mesh_tri_off || m->n_meshes <= 0)
    return fail(ctx, PJ_ERR_INVALID_ARG, "host meshes need coordinates, triangles and offsets");
  h.m = m;
  h.box.assign(6 * (size_t)m->n_meshes, 0.f);
  h.bytes.assign((size_t)m->n_meshes, 0);
  for (int64_t k = 0; k < m->n_meshes; ++k) {
    const int64_t v0 = m->mesh_vert_off[k], v1 = m->mesh_vert_off[k + 1];
    const int64_t t0 = m->mesh_tri_off[k], t1 = m->mesh_tri_off[k + 1];
    if (v1 <= v0 || t1 <= t0) return fail(ctx, PJ_ERR_INVALID_ARG, "empty mesh");
    float *b = &h.box[6 * k];
    for (int d = 0; d < 3; ++d) {
      b[d] = 3.4e38f;
      b[3 + d] = -3.4e38f;
    }
    for (int64_t v = v0; v < v1; ++v)
      for (int d = 0; d < 3; ++d) {
        b[d] = std::min(b[d], m->xyz[3 * v + d]);
        b[3 + d] = std::max(b[3 + d], m->xyz[3 * v + d]);
      }
    h.bytes[k] = mesh_bytes(v1 - v0, t1 - t0, W, L);
  }
  return PJ_OK;
}

void cell_range(const TGrid &g, const float *b, int lo[3], int hi[3]) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = g.idx(b[d], d);
    hi[d] = g.idx(b[3 + d], d);
  }
}

// per cell: the meshes of h whose closed box touches it, in id order
std::vector<std::vector<int32_t>> assign(const TGrid &g, const HostSet &h) {
  std::vector<std::vector<int32_t>> cells((size_t)g.G * g.G * g.G);
  for (int64_t k = 0; k < h.m->n_meshes; ++k) {
    int lo[3], hi[3];
    cell_range(g, &h.box[6 * k], lo, hi);
    for (int x = lo[0]; x <= hi[0]; ++x)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int z = lo[2]; z <= hi[2]; ++z)
          cells[((size_t)x * g.G + y) * g.G + z].push_back((int32_t)k);
  }
  return cells;
}

// one cell's meshes gathered into contiguous host arrays
struct Gathered {
  std::vector<float> xyz;
  std::vector<int32_t> tris;
  std::vector<int64_t> voff{0}, toff{0};
};

void gather(const pj_host_meshes *m, const std::vector<int32_t> &ids, Gathered &out) {
  out.xyz.clear();
  out.tris.clear();
  out.voff.assign(1, 0);
  out.toff.assign(1, 0);
  for (int32_t k : ids) {
    const int64_t v0 = m->mesh_vert_off[k], v1 = m->mesh_vert_off[k + 1];
    const int64_t t0 = m->mesh_tri_off[k], t1 = m->mesh_tri_off[k + 1];
    out.xyz.insert(out.xyz.end(), m->xyz + 3 * v0, m->xyz + 3 * v1);
    out.tris.insert(out.tris.end(), m->tris + 3 * t0, m->tris + 3 * t1);
    out.voff.push_back(out.voff.back() + (v1 - v0));
    out.toff.push_back(out.toff.back() + (t1 - t0));
  }
}

double now() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

pj_status run_join_tiled(Ctx *ctx, const pj_host_meshes *Am, const pj_host_meshes *Bm,
                         int self_join, const pj_tiled_opts *o, pj_pairs *out,
                         pj_tiled_stats *stats) {
  const double t_start = now();
  const int W = o->width ? o->width : 4, L = o->leaf_size ? o->leaf_size : 2;
  if (!(W == 2 || W == 4 || W == 8) || !(L == 1 || L == 2 || L == 4 || L == 8))
    return fail(ctx, PJ_ERR_INVALID_ARG, "width must be 2, 4 or 8 and leaf size 1, 2, 4 or 8");
  if (self_join) Bm = Am;
  HostSet A, B;
  pj_status st;
  if ((st = prepare(ctx, Am, W, L, A)) != PJ_OK) return st;
  if (self_join) B = A;
  else if ((st = prepare(ctx, Bm, W, L, B)) != PJ_OK) return st;
  int64_t budget = o->device_budget;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    PJ_CK(cudaMemGetInfo(&fr, &tot));
    budget = (int64_t)(fr / 4);
  }
  // the grid over both datasets' box
  TGrid g;
  for (int d = 0; d < 3; ++d) {
    double lo = 1e300, hi = -1e300;
    for (const HostSet *H : {&A, &B})
      for (int64_t k = 0; k < H->m->n_meshes; ++k) {
        lo = std::min(lo, (double)H->box[6 * k + d]);
        hi = std::max(hi, (double)H->box[6 * k + 3 + d]);
      }
    g.g0[d] = lo;
    g.cw[d] = std::max(hi - lo, 1.0);
  }
  const double ext[3] = {g.cw[0], g.cw[1], g.cw[2]};
  std::vector<std::vector<int32_t>> ca, cb;
  int64_t max_bytes = 0;
  for (int G = o->grid > 0 ? o->grid : 1;; G *= 2) {
    g.G = G;
    for (int d = 0; d < 3; ++d) g.cw[d] = ext[d] / G;
    ca = assign(g, A);
    cb = self_join ? ca : assign(g, B);
    max_bytes = 0;
    for (size_t c = 0; c < ca.size(); ++c) {
      if (ca[c].empty() || cb[c].empty()) continue;
      int64_t bytes = 0;
      for (int32_t k : ca[c]) bytes += A.bytes[k];
      if (!self_join)
        for (int32_t k : cb[c]) bytes += B.bytes[k];
      max_bytes = std::max(max_bytes, bytes);
    }
    if (o->grid > 0 || max_bytes <= budget || G >= 16) break;
  }
  for (const HostSet *H : {&A, &B})
    for (int64_t b : H->bytes)
      if (b > budget)
        return fail(ctx, PJ_ERR_NO_MEMORY, "a mesh alone exceeds the tiled join's device budget");
  if (max_bytes > budget)
    return fail(ctx, PJ_ERR_NO_MEMORY, "the finest grid's largest cell exceeds the device budget");

  pj_tiled_stats S;
  memset(&S, 0, sizeof(S));
  S.grid = g.G;
  S.max_cell_bytes = max_bytes;
  std::vector<size_t> todo;
  for (size_t c = 0; c < ca.size(); ++c)
    if (!ca[c].empty() && !cb[c].empty()) todo.push_back(c);
  // the next cell is gathered on the host while the current one is on the GPU
  auto gather_cell = [&](size_t c, Gathered *ga, Gathered *gb) {
    const double t0 = now();
    gather(A.m, ca[c], *ga);
    if (!self_join) gather(B.m, cb[c], *gb);
    return now() - t0;
  };
  Gathered buf[2][2];
  std::future<double> next;
  if (!todo.empty()) next = std::async(std::launch::async, gather_cell, todo[0], &buf[0][0], &buf[0][1]);
  std::vector<unsigned long long> keys;
  double t_gather = 0.0, t_device = 0.0;
  pj_join_opts jo = o->join;
  jo.width = W;
  jo.leaf_size = L;
  jo.out_host = 1;
  jo.keep_flags = 0;
  jo.record_cycles = 0;
  // no captured graphs: every cell's datasets are new allocations that are
  // freed before the next cell
  jo.use_graph = 0;
  for (size_t n = 0; n < todo.size(); ++n) {
    const size_t c = todo[n];
    t_gather += next.get();
    Gathered &ga = buf[n & 1][0], &gb = buf[n & 1][1];
    if (n + 1 < todo.size())
      next = std::async(std::launch::async, gather_cell, todo[n + 1], &buf[(n + 1) & 1][0],
                        &buf[(n + 1) & 1][1]);
    const double t0 = now();
    std::unique_ptr<Dataset> da(new Dataset()), db;
    st = load_impl(ctx, ga.xyz.data(), (int64_t)ga.xyz.size() / 3, ga.tris.data(),
                   (int64_t)ga.tris.size() / 3, ga.voff.data(), ga.toff.data(),
                   (int64_t)ga.voff.size() - 1, 0, da.get());
    if (st == PJ_OK && !self_join) {
      db.reset(new Dataset());
      st = load_impl(ctx, gb.xyz.data(), (int64_t)gb.xyz.size() / 3, gb.tris.data(),
                     (int64_t)gb.tris.size() / 3, gb.voff.data(), gb.toff.data(),
                     (int64_t)gb.voff.size() - 1, 0, db.get());
    }
    Dataset *DA = da.get(), *DB = self_join ? da.get() : db.get();
    if (st == PJ_OK) st = build_bvh(ctx, DA, W, L, ctx->stream);
    if (st == PJ_OK && !self_join) st = build_bvh(ctx, DB, W, L, ctx->stream);
    pj_pairs r;
    memset(&r, 0, sizeof(r));
    if (st == PJ_OK) {
      DA->last_bvh = DB->last_bvh = {W, L};
      st = run_join(ctx, DA, DB, nullptr, nullptr, -1, 0, self_join, &jo, ctx->stream, &r);
    }
    cudaStreamSynchronize(ctx->stream);
    free_dataset(DA);
    if (!self_join && db) free_dataset(DB);
    if (st != PJ_OK) {
      pairs_release(ctx, &r);
      if (n + 1 < todo.size()) next.get();
      return st;
    }
    S.cells_joined += 1;
    S.mesh_copies += (int64_t)ca[c].size() + (self_join ? 0 : (int64_t)cb[c].size());
    S.pairs_in_cells += r.count;
    // global ids; keep the pair in its reference point's cell only
    const int cx = (int)(c / ((size_t)g.G * g.G)), cy = (int)((c / g.G) % g.G), cz = (int)(c % g.G);
    for (int64_t k = 0; k < r.count; ++k) {
      const int32_t i = ca[c][r.pairs[2 * k]], j = cb[c][r.pairs[2 * k + 1]];
      const float *bi = &A.box[6 * (int64_t)i], *bj = &B.box[6 * (int64_t)j];
      const int rx = g.idx(std::max(bi[0], bj[0]), 0), ry = g.idx(std::max(bi[1], bj[1]), 1);
      const int rz = g.idx(std::max(bi[2], bj[2]), 2);
      if (rx == cx && ry == cy && rz == cz)
        keys.push_back(((unsigned long long)(unsigned)i << 32) | (unsigned)j);
    }
    pairs_release(ctx, &r);
    t_device += now() - t0;
  }
  std::sort(keys.begin(), keys.end());
  memset(out, 0, sizeof(*out));
  const int64_t K = (int64_t)keys.size();
  out->count = K;
  std::vector<int32_t> flat(2 * (size_t)std::max<int64_t>(K, 1));
  for (int64_t k = 0; k < K; ++k) {
    flat[2 * k] = (int32_t)(keys[k] >> 32);
    flat[2 * k + 1] = (int32_t)(keys[k] & 0xFFFFFFFFull);
  }
  if (o->out_host) {
    PJ_CK(cudaMallocHost((void **)&out->pairs, 8 * (size_t)std::max<int64_t>(K, 1)));
    memcpy(out->pairs, flat.data(), 8 * (size_t)K);
    out->on_device = 0;
  } else {
    cudaError_t pe;
    out->pairs = (int32_t *)pool_get(ctx, 8 * (size_t)std::max<int64_t>(K, 1), &pe);
    PJ_CK(pe);
    if (K > 0) PJ_CK(cudaMemcpy(out->pairs, flat.data(), 8 * (size_t)K, cudaMemcpyHostToDevice));
    out->on_device = 1;
  }
  S.ms_total = (float)((now() - t_start) * 1e3);
  S.ms_gather = (float)(t_gather * 1e3);
  S.ms_device = (float)(t_device * 1e3);
  out->device_ms = S.ms_device;
  if (stats) *stats = S;
  return PJ_OK;
}

}  // namespace pj
