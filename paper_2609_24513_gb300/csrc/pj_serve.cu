// Serving: window join queries submitted from any thread, admitted by a
// device-memory budget and refined in batches on several streams at once.
//
// The paper evaluates one join at a time (Sec. 4); serving adds the request
// loop around the same refinement.  A query selects, on each side, the meshes
// whose closed box meets its window (host side, from the boxes computed at
// load time) and asks for the intersecting pairs among them.
//
// Continuous batching: each serving stream has a worker thread.  A free
// worker takes the oldest pending query and every following pending query on
// the same dataset pair while the admitted device bytes stay within the
// budget, so queries that arrive while other batches run join the next batch
// that a stream frees up for.  A batch runs the bounding-box filter on the
// selected meshes of all its queries (one warp per selected mesh of side A),
// the refinement of the whole candidate list, and a per-query count that
// splits the compacted pairs back into queries.  Batches of different workers
// overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <vector>

#include "pj_internal.cuh"

namespace pj {

static double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Query {
  pj_ticket id = 0;
  Dataset *A = nullptr, *B = nullptr;
  int self_join = 0;
  std::vector<int32_t> selA, selB;
  int64_t est_bytes = 0;
  pj_query_stats st{};
  std::vector<int32_t> pairs;
  pj_status status = PJ_PENDING;
  std::string err;
};

struct Serve {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Query>> pending;
  std::map<pj_ticket, std::shared_ptr<Query>> tickets;
  std::vector<std::thread> workers;
  std::vector<std::unique_ptr<Exec>> execs;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  int64_t budget = 0, inflight = 0;
  pj_ticket next_ticket = 1;
  int next_batch = 0;
  int64_t wait_us = 0;
  std::map<const Dataset *, int64_t> uses;  // unpolled queries per dataset
};

// warp per selected A mesh: count (EMIT = false) or emit (EMIT = true) the
// selected B meshes of the same query whose closed boxes meet it
template <bool EMIT>
__global__ void k_mbb_subset(const float *aabbA, const float *aabbB, const int32_t *selA,
                             const int32_t *selB, const int64_t *offA, const int64_t *offB,
                             int nq, int64_t nA, int self_join, int64_t *counts,
                             const int64_t *offs, int32_t *cand) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t g = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); g < nA;
       g += warps) {
    int lo = 0, hi = nq - 1;  // query of g: largest q with offA[q] <= g
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (offA[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int q = lo;
    const int32_t i = selA[g];
    const float *a = aabbA + 6 * (int64_t)i;
    int64_t cnt = 0, pos = EMIT ? offs[g] : 0;
    for (int64_t k0 = offB[q]; k0 < offB[q + 1]; k0 += 32) {
      const int64_t k = k0 + lane;
      bool ov = false;
      int32_t j = 0;
      if (k < offB[q + 1]) {
        j = selB[k];
        const float *b = aabbB + 6 * (int64_t)j;
        ov = (!self_join || j > i) && a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] &&
             b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
      }
      const unsigned m = __ballot_sync(0xffffffffu, ov);
      if (EMIT && ov) {
        const int64_t p = pos + __popc(m & ((1u << lane) - 1u));
        cand[2 * p] = i;
        cand[2 * p + 1] = j;
      }
      if (EMIT) pos += __popc(m);
      else cnt += __popc(m);
    }
    if (!EMIT && lane == 0) counts[g] = cnt;
  }
}

// per-query number of intersecting candidates
__global__ void k_query_counts(const uint8_t *flags, const int64_t *cand_off, int nq,
                               int64_t *out) {
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    int64_t c = 0;
    for (int64_t k = cand_off[q] + threadIdx.x; k < cand_off[q + 1]; k += blockDim.x)
      c += flags[k] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int64_t ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
      out[q] = t;
    }
    __syncthreads();
  }
}

__global__ void k_gather_i64(const int64_t *src, const int64_t *idx, int n, int64_t *dst) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    dst[k] = src[idx[k]];
}

// Run one batch on the worker's stream and scratch.  Fills each query's
// pairs and counts, or its status on failure.
static pj_status run_batch(Ctx *ctx, Exec *ex, cudaStream_t s,
                           std::vector<std::shared_ptr<Query>> &batch) {
  Dataset *A = batch[0]->A, *B = batch[0]->B;
  const int self_join = batch[0]->self_join;
  const int nq = (int)batch.size();
  std::vector<int64_t> offA(nq + 1, 0), offB(nq + 1, 0);
  for (int q = 0; q < nq; ++q) {
    offA[q + 1] = offA[q] + (int64_t)batch[q]->selA.size();
    offB[q + 1] = offB[q] + (int64_t)batch[q]->selB.size();
  }
  const int64_t nA = offA[nq], nB = offB[nq];
  std::vector<int32_t> selA, selB;
  selA.reserve(nA);
  selB.reserve(nB);
  for (auto &q : batch) {
    selA.insert(selA.end(), q->selA.begin(), q->selA.end());
    selB.insert(selB.end(), q->selB.begin(), q->selB.end());
  }
  pj_status st;
  auto get = [&](const char *name, size_t bytes) { return ws_get(ctx, name, bytes, &st); };
  int32_t *d_selA = (int32_t *)get("srv_sel_a", 4 * (size_t)std::max<int64_t>(nA, 1));
  int32_t *d_selB = (int32_t *)get("srv_sel_b", 4 * (size_t)std::max<int64_t>(nB, 1));
  int64_t *d_offA = (int64_t *)get("srv_off_a", 8 * (size_t)(nq + 1));
  int64_t *d_offB = (int64_t *)get("srv_off_b", 8 * (size_t)(nq + 1));
  int64_t *d_counts = (int64_t *)get("srv_counts", 8 * (size_t)std::max<int64_t>(nA, 1));
  int64_t *d_offs = (int64_t *)get("srv_offs", 8 * (size_t)std::max<int64_t>(nA, 1) + 8);
  int64_t *d_small = (int64_t *)get("srv_small", 8 * (size_t)(3 * (nq + 1) + 8));
  if (!d_selA || !d_selB || !d_offA || !d_offB || !d_counts || !d_offs || !d_small) return st;
  int64_t *d_total = d_small, *d_qcand = d_small + 1, *d_qidx = d_qcand + (nq + 1),
          *d_qcount = d_qidx + (nq + 1);
  PJ_CK(cudaMemcpyAsync(d_selA, selA.data(), 4 * nA, cudaMemcpyHostToDevice, s));
  PJ_CK(cudaMemcpyAsync(d_selB, selB.data(), 4 * nB, cudaMemcpyHostToDevice, s));
  PJ_CK(cudaMemcpyAsync(d_offA, offA.data(), 8 * (nq + 1), cudaMemcpyHostToDevice, s));
  PJ_CK(cudaMemcpyAsync(d_offB, offB.data(), 8 * (nq + 1), cudaMemcpyHostToDevice, s));
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((nA + 7) / 8, (int64_t)ctx->num_sms * 64));
  if (nA > 0)
    k_mbb_subset<false><<<nb, 256, 0, s>>>(A->d_aabb, B->d_aabb, d_selA, d_selB, d_offA, d_offB,
                                           nq, nA, self_join, d_counts, nullptr, nullptr);
  ctx->launches += nA > 0 ? 1 : 0;
  if (nA > 0 && (st = scan_i64(ctx, d_counts, d_offs, nA, d_total, s)) != PJ_OK) return st;
  if (nA == 0) PJ_CK(cudaMemsetAsync(d_total, 0, 8, s));
  int64_t *h = (int64_t *)ex->h_pinned;
  PJ_CK(cudaMemcpyAsync(h, d_total, 8, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  const int64_t C = h[0];
  // candidate offsets of each query: the scan at its first selected A mesh
  std::vector<int64_t> qidx(nq + 1);
  for (int q = 0; q <= nq; ++q) qidx[q] = std::min(offA[q], std::max<int64_t>(nA - 1, 0));
  int32_t *d_cand = (int32_t *)get("srv_cand", 8 * (size_t)std::max<int64_t>(C, 1));
  if (!d_cand) return st;
  if (C > 0)
    k_mbb_subset<true><<<nb, 256, 0, s>>>(A->d_aabb, B->d_aabb, d_selA, d_selB, d_offA, d_offB,
                                          nq, nA, self_join, nullptr, d_offs, d_cand);
  ctx->launches += C > 0 ? 1 : 0;
  std::vector<int64_t> qcand(nq + 1, 0);
  if (nA > 0) {
    PJ_CK(cudaMemcpyAsync(d_qidx, qidx.data(), 8 * (nq + 1), cudaMemcpyHostToDevice, s));
    k_gather_i64<<<1, 256, 0, s>>>(d_offs, d_qidx, nq + 1, d_qcand);
    PJ_CK(cudaMemcpyAsync(qcand.data(), d_qcand, 8 * (nq + 1), cudaMemcpyDeviceToHost, s));
    PJ_CK(cudaStreamSynchronize(s));
    for (int q = 0; q <= nq; ++q)
      if (offA[q] >= nA) qcand[q] = C;  // queries with no selected A mesh at the end
    qcand[nq] = C;
    PJ_CK(cudaMemcpyAsync(d_qcand, qcand.data(), 8 * (nq + 1), cudaMemcpyHostToDevice, s));
  }
  for (auto &q : batch) q->st.t_launch = now_s();
  std::vector<int64_t> qcount(nq, 0);
  std::vector<int32_t> pairs;
  if (C > 0) {
    pj_join_opts o{};
    o.keep_flags = 1;
    pj_pairs res;
    memset(&res, 0, sizeof(res));
    if ((st = run_join(ctx, A, B, d_cand, nullptr, C, 1, self_join, &o, s, &res)) != PJ_OK)
      return st;
    const int64_t K = res.count;
    pairs.resize(2 * (size_t)K);
    k_query_counts<<<std::min(nq, 4096), 256, 0, s>>>(res.flags, d_qcand, nq, d_qcount);
    ctx->launches += 1;
    cudaError_t e = cudaMemcpyAsync(qcount.data(), d_qcount, 8 * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && K > 0)
      e = cudaMemcpyAsync(pairs.data(), res.pairs, 8 * K, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "serving batch results");
  }
  int64_t at = 0;
  for (int q = 0; q < nq; ++q) {
    batch[q]->st.n_candidates = qcand[q + 1] - qcand[q];
    batch[q]->st.n_pairs = qcount[q];
    batch[q]->pairs.assign(pairs.begin() + 2 * at, pairs.begin() + 2 * (at + qcount[q]));
    at += qcount[q];
  }
  return PJ_OK;
}

static void worker(Ctx *ctx, Serve *sv, int w) {
  cudaSetDevice(ctx->device);
  t_exec = sv->execs[w].get();
  t_exec->borrow_out = true;  // join results stay in this thread's workspaces
  cudaStream_t s = sv->streams[w];
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    if (sv->pending.empty() ||
        (sv->inflight > 0 && sv->inflight + sv->pending.front()->est_bytes > sv->budget)) {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // the oldest query and every later one on the same datasets that fits
    std::vector<std::shared_ptr<Query>> batch;
    int64_t bytes = 0;
    const double t = now_s();
    for (auto it = sv->pending.begin(); it != sv->pending.end() && batch.size() < 512;) {
      auto &q = *it;
      const bool same = batch.empty() || (q->A == batch[0]->A && q->B == batch[0]->B &&
                                          q->self_join == batch[0]->self_join);
      if (same && (batch.empty() || sv->inflight + bytes + q->est_bytes <= sv->budget)) {
        bytes += q->est_bytes;
        q->st.t_admit = t;
        batch.push_back(q);
        it = sv->pending.erase(it);
      } else if (!same) {
        ++it;
      } else {
        break;
      }
    }
    const int id = sv->next_batch++;
    for (auto &q : batch) {
      q->st.batch_id = id;
      q->st.batch_queries = (int32_t)batch.size();
      q->st.device_bytes = q->est_bytes;
    }
    sv->inflight += bytes;
    lk.unlock();
    pj_status st;
    {
      std::shared_lock<std::shared_mutex> rl(ctx->ds_rw);
      st = run_batch(ctx, t_exec, s, batch);
    }
    std::string msg;
    if (st != PJ_OK) {
      cudaGetLastError();
      msg = "serving batch failed: " + t_exec->err;
    }
    lk.lock();
    sv->inflight -= bytes;
    const double td = now_s();
    for (auto &q : batch) {
      q->st.t_done = td;
      q->status = st;
      q->err = msg;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

static pj_status serve_start(Ctx *ctx) {
  if (ctx->serve) return PJ_OK;
  cudaSetDevice(ctx->device);
  std::unique_ptr<Serve> sv(new Serve());
  sv->budget = ctx->cfg.budget_bytes > 0 ? ctx->cfg.budget_bytes : (40ll << 30);
  sv->wait_us = ctx->cfg.wait_limit_us > 0 ? ctx->cfg.wait_limit_us : 10000000ll;
  const int n = ctx->cfg.serve_streams > 0 ? std::min(ctx->cfg.serve_streams, 16) : 4;
  for (int w = 0; w < n; ++w) {
    std::unique_ptr<Exec> ex(new Exec());
    pj_status st = exec_init(ctx, ex.get());
    cudaStream_t s = nullptr;
    if (st == PJ_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      st = fail(ctx, PJ_ERR_CUDA, "cudaStreamCreate");
    if (st != PJ_OK) {
      exec_free(ex.get());
      for (auto &e : sv->execs) exec_free(e.get());
      for (auto q : sv->streams) cudaStreamDestroy(q);
      return st;
    }
    sv->execs.push_back(std::move(ex));
    sv->streams.push_back(s);
  }
  ctx->serve = sv.release();
  for (int w = 0; w < n; ++w) ctx->serve->workers.emplace_back(worker, ctx, ctx->serve, w);
  return PJ_OK;
}

bool serve_uses(Ctx *ctx, const Dataset *d) {
  Serve *sv = ctx->serve;
  if (!sv) return false;
  std::lock_guard<std::mutex> lk(sv->mu);
  return sv->uses.count(d) > 0;
}

void serve_stop(Ctx *ctx) {
  Serve *sv = ctx->serve;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto &t : sv->workers) t.join();
  for (auto s : sv->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (auto &e : sv->execs) exec_free(e.get());
  delete sv;
  ctx->serve = nullptr;
}

static void select_meshes(const Dataset *D, const std::vector<float> &box, const int32_t *lo,
                          const int32_t *hi, std::vector<int32_t> &out) {
  out.clear();
  for (int64_t m = 0; m < D->M; ++m) {
    const float *b = &box[6 * m];
    if (b[0] <= hi[0] && lo[0] <= b[3] && b[1] <= hi[1] && lo[1] <= b[4] && b[2] <= hi[2] &&
        lo[2] <= b[5])
      out.push_back((int32_t)m);
  }
}

pj_status serve_submit(Ctx *ctx, Dataset *A, Dataset *B, const pj_query *q, pj_ticket *out) {
  if (A->bvhs.find(A->last_bvh) == A->bvhs.end() || B->bvhs.find(A->last_bvh) == B->bvhs.end())
    return fail(ctx, PJ_ERR_INVALID_ARG, "both datasets need a BVH of the same shape (pj_build_bvh)");
  for (int d = 0; d < 3; ++d)
    if (q->window_lo[d] > q->window_hi[d]) return fail(ctx, PJ_ERR_INVALID_ARG, "empty window");
  pj_status st = serve_start(ctx);
  if (st != PJ_OK) return st;
  auto qq = std::make_shared<Query>();
  qq->st.t_submit = now_s();
  qq->A = A;
  qq->B = B;
  qq->self_join = q->self_join;
  if (A->h_aabb.empty() || B->h_aabb.empty()) return fail(ctx, PJ_ERR_INTERNAL, "no host boxes");
  select_meshes(A, A->h_aabb, q->window_lo, q->window_hi, qq->selA);
  if (A == B && q->self_join) qq->selB = qq->selA;
  else select_meshes(B, B->h_aabb, q->window_lo, q->window_hi, qq->selB);
  qq->st.n_a = (int64_t)qq->selA.size();
  qq->st.n_b = (int64_t)qq->selB.size();
  // device bytes: every selected pair as a candidate (id pair, flag, output
  // pair), the selections, and the scans over them
  qq->est_bytes = qq->st.n_a * qq->st.n_b * 17 + (qq->st.n_a + qq->st.n_b) * 24 + 4096;
  Serve *sv = ctx->serve;
  if (qq->est_bytes > sv->budget)
    return fail(ctx, PJ_ERR_BUSY, "the query needs more device memory than the serving budget");
  std::lock_guard<std::mutex> lk(sv->mu);
  qq->id = sv->next_ticket++;
  sv->tickets[qq->id] = qq;
  ++sv->uses[A];
  ++sv->uses[B];
  sv->pending.push_back(qq);
  sv->cv_work.notify_one();
  *out = qq->id;
  return PJ_OK;
}

pj_status serve_poll(Ctx *ctx, pj_ticket t, int wait, pj_pairs *out, pj_query_stats *stats) {
  Serve *sv = ctx->serve;
  if (!sv) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown ticket");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(t);
  if (it == sv->tickets.end()) return fail(ctx, PJ_ERR_INVALID_ARG, "unknown ticket");
  std::shared_ptr<Query> q = it->second;
  if (q->status == PJ_PENDING) {
    if (!wait) return PJ_PENDING;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(sv->wait_us);
    while (q->status == PJ_PENDING) {
      if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
          q->status == PJ_PENDING)
        return fail(ctx, PJ_ERR_TIMEOUT, "query still pending after the wait limit");
    }
  }
  sv->tickets.erase(it);
  if (--sv->uses[q->A] == 0) sv->uses.erase(q->A);
  if (--sv->uses[q->B] == 0) sv->uses.erase(q->B);
  if (stats) *stats = q->st;
  if (q->status != PJ_OK) return fail(ctx, q->status, q->err);
  memset(out, 0, sizeof(*out));
  out->count = q->st.n_pairs;
  out->n_candidates = q->st.n_candidates;
  out->on_device = 0;
  out->pairs_malloc = 1;
  const size_t bytes = sizeof(int32_t) * 2 * (size_t)std::max<int64_t>(q->st.n_pairs, 1);
  out->pairs = (int32_t *)malloc(bytes);
  if (!out->pairs) return fail(ctx, PJ_ERR_NO_MEMORY, "result buffer");
  if (!q->pairs.empty()) memcpy(out->pairs, q->pairs.data(), 4 * q->pairs.size());
  return PJ_OK;
}

}  // namespace pj
