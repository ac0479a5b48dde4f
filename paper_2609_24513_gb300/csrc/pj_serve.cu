// Serving: window join queries submitted from any thread, admitted by a
// device-memory budget and refined in batches on several streams at once.
//
// The paper evaluates one join at a time (Sec. 4); serving adds the request
// loop around the same refinement.  A query selects, on each side, the meshes
// whose closed box meets its window and asks for the intersecting pairs among
// them.  Admission bounds a query's device bytes in O(1) from a grid of mesh
// counts built at load time; the selection itself runs on the device, per
// batch (one block per query and side, in mesh order).
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
  int32_t lo[3], hi[3];   // window (closed, grid units)
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

// block per (query, side): the ids of the side's meshes whose closed box
// meets the query's window, in id order, to sel[q * M + k], and their number
// to cnt[side * nq + q] (a self join selects one side, read for both)
__global__ void __launch_bounds__(256) k_select(const float *aabbA, int64_t MA, const float *aabbB,
                                                int64_t MB, const int32_t *win, int nq,
                                                int self_join, int32_t *selA, int32_t *selB,
                                                int64_t *cnt) {
  const int q = blockIdx.x, side = blockIdx.y;
  if (side == 1 && self_join) return;
  const int64_t M = side ? MB : MA;
  const float *box = side ? aabbB : aabbA;
  int32_t *sel = (side ? selB : selA) + (int64_t)q * M;
  const int32_t *w = win + 6 * q;
  const float lx = (float)w[0], ly = (float)w[1], lz = (float)w[2];
  const float hx = (float)w[3], hy = (float)w[4], hz = (float)w[5];
  __shared__ int ws[8];
  __shared__ int64_t s_run;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < M; base += 256) {
    const int64_t m = base + threadIdx.x;
    bool in = false;
    if (m < M) {
      const float *b = box + 6 * m;
      in = b[0] <= hx && lx <= b[3] && b[1] <= hy && ly <= b[4] && b[2] <= hz && lz <= b[5];
    }
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    if (lane == 0) ws[wid] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
    for (int k = 0; k < 8; ++k) {
      before += k < wid ? ws[k] : 0;
      tot += ws[k];
    }
    const int64_t run = s_run;
    if (in) sel[run + before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)m;
    __syncthreads();
    if (threadIdx.x == 0) s_run = run + tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) cnt[side * nq + q] = s_run;
}

// one block: offA / offB = exclusive prefixes of the per-query counts
// (nq + 1 entries each; a self join's B side is its A side)
__global__ void k_sel_offsets(const int64_t *cnt, int nq, int self_join, int64_t *offA,
                              int64_t *offB) {
  if (threadIdx.x != 0) return;
  int64_t a = 0, b = 0;
  for (int q = 0; q < nq; ++q) {
    offA[q] = a;
    offB[q] = b;
    a += cnt[q];
    b += cnt[(self_join ? 0 : nq) + q];
  }
  offA[nq] = a;
  offB[nq] = b;
}

// warp per selected A mesh g (over all queries): count (EMIT = false) or
// emit (EMIT = true) the same query's selected B meshes whose closed boxes
// meet it, in B order -- so candidates come out query by query, sorted
template <bool EMIT>
__global__ void k_mbb_subset(const float *aabbA, int64_t MA, const float *aabbB, int64_t MB,
                             const int32_t *selA, const int32_t *selB, const int64_t *offA,
                             const int64_t *cntB, int nq, int self_join, int64_t *counts,
                             const int64_t *offs, int32_t *cand) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t nA = offA[nq];
  for (int64_t g = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); g < nA;
       g += warps) {
    int lo = 0, hi = nq - 1;  // query of g: largest q with offA[q] <= g
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (offA[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const int q = lo;
    const int32_t i = selA[(int64_t)q * MA + (g - offA[q])];
    const float *a = aabbA + 6 * (int64_t)i;
    const int32_t *sb = self_join ? selA + (int64_t)q * MA : selB + (int64_t)q * MB;
    const int64_t nb = cntB[q];
    int64_t cnt = 0, pos = EMIT ? offs[g] : 0;
    for (int64_t k0 = 0; k0 < nb; k0 += 32) {
      const int64_t k = k0 + lane;
      bool ov = false;
      int32_t j = 0;
      if (k < nb) {
        j = sb[k];
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

// per query: the position of its first candidate (the scan at its first
// selected A mesh; past the last one, the total)
__global__ void k_query_starts(const int64_t *offs, const int64_t *offA, int nq, int64_t *qcand) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x)
    qcand[q] = offs[offA[q]];
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

// Run one batch on the worker's stream and scratch: window selection, box
// filter and refinement on the device, with one host synchronisation after
// the candidates are counted and one at the end.  Fills each query's pairs
// and counts, or returns the status of a failure.
static pj_status run_batch(Ctx *ctx, Exec *ex, cudaStream_t s,
                           std::vector<std::shared_ptr<Query>> &batch) {
  Dataset *A = batch[0]->A, *B = batch[0]->B;
  const int self_join = batch[0]->self_join;
  const int nq = (int)batch.size();
  const int64_t MA = A->M, MB = B->M;
  pj_status st;
  auto get = [&](const char *name, size_t bytes) { return ws_get(ctx, name, bytes, &st); };
  // selection slots per query, counts of selected A meshes' candidates
  const int64_t capA = (int64_t)nq * MA;
  int32_t *d_win = (int32_t *)get("srv_win", sizeof(int32_t) * 6 * (size_t)nq);
  int32_t *d_selA = (int32_t *)get("srv_sel_a", 4 * (size_t)std::max<int64_t>(capA, 1));
  int32_t *d_selB = self_join ? d_selA
                              : (int32_t *)get("srv_sel_b", 4 * (size_t)std::max<int64_t>((int64_t)nq * MB, 1));
  int64_t *d_small = (int64_t *)get("srv_small", 8 * (size_t)(6 * (nq + 1) + 8));
  int64_t *d_counts = (int64_t *)get("srv_counts", 8 * (size_t)(capA + 1));
  int64_t *d_offs = (int64_t *)get("srv_offs", 8 * (size_t)(capA + 1));
  if (!d_win || !d_selA || !d_selB || !d_small || !d_counts || !d_offs) return st;
  // per query: selection counts (2 nq), offsets (2 (nq + 1)), first
  // candidate (nq + 1), pair count (nq); then the candidate total
  int64_t *d_cnt = d_small, *d_offA = d_cnt + 2 * nq, *d_offB = d_offA + (nq + 1),
          *d_qcand = d_offB + (nq + 1), *d_qcount = d_qcand + (nq + 1),
          *d_total = d_qcount + nq;
  std::vector<int32_t> win(6 * (size_t)nq);
  for (int q = 0; q < nq; ++q)
    for (int k = 0; k < 3; ++k) {
      win[6 * q + k] = batch[q]->lo[k];
      win[6 * q + 3 + k] = batch[q]->hi[k];
    }
  PJ_CK(cudaMemcpyAsync(d_win, win.data(), sizeof(int32_t) * 6 * nq, cudaMemcpyHostToDevice, s));
  k_select<<<dim3(nq, 2), 256, 0, s>>>(A->d_aabb, MA, B->d_aabb, MB, d_win, nq, self_join, d_selA,
                                       d_selB, d_cnt);
  k_sel_offsets<<<1, 32, 0, s>>>(d_cnt, nq, self_join, d_offA, d_offB);
  PJ_CK(cudaMemsetAsync(d_counts, 0, 8 * (size_t)(capA + 1), s));
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((capA + 7) / 8, (int64_t)ctx->num_sms * 64));
  const int64_t *cntB = d_cnt + (self_join ? 0 : nq);
  k_mbb_subset<false><<<nb, 256, 0, s>>>(A->d_aabb, MA, B->d_aabb, MB, d_selA, d_selB, d_offA,
                                         cntB, nq, self_join, d_counts, nullptr, nullptr);
  if ((st = scan_i64(ctx, d_counts, d_offs, capA + 1, d_total, s)) != PJ_OK) return st;
  k_query_starts<<<1, 256, 0, s>>>(d_offs, d_offA, nq, d_qcand);
  ctx->launches += 4;
  PJ_CK(cudaGetLastError());
  // one round trip: the candidate count, each query's first candidate and
  // selection sizes
  (void)ex;
  std::vector<int64_t> qcand(nq + 1), cnt(2 * (size_t)nq);
  PJ_CK(cudaMemcpyAsync(qcand.data(), d_qcand, 8 * (size_t)(nq + 1), cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaMemcpyAsync(cnt.data(), d_cnt, 8 * 2 * (size_t)nq, cudaMemcpyDeviceToHost, s));
  PJ_CK(cudaStreamSynchronize(s));
  const int64_t C = qcand[nq];
  for (int q = 0; q < nq; ++q) {
    batch[q]->st.n_a = cnt[q];
    batch[q]->st.n_b = cnt[(self_join ? 0 : nq) + q];
  }
  int32_t *d_cand = (int32_t *)get("srv_cand", 8 * (size_t)std::max<int64_t>(C, 1));
  if (!d_cand) return st;
  if (C > 0) {
    k_mbb_subset<true><<<nb, 256, 0, s>>>(A->d_aabb, MA, B->d_aabb, MB, d_selA, d_selB, d_offA,
                                          cntB, nq, self_join, nullptr, d_offs, d_cand);
    ctx->launches += 1;
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
    ex->stream = s;
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
  for (auto s : sv->streams) cudaStreamSynchronize(s);
  for (auto &e : sv->execs) exec_free(e.get());  // on their streams
  for (auto s : sv->streams) cudaStreamDestroy(s);
  delete sv;
  ctx->serve = nullptr;
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
  for (int k = 0; k < 3; ++k) {
    qq->lo[k] = q->window_lo[k];
    qq->hi[k] = q->window_hi[k];
  }
  // admission: an upper bound of each side's selection from the load-time
  // grid of mesh counts (O(1); the exact selection runs on the device)
  const int64_t na = window_mesh_bound(A, q->window_lo, q->window_hi);
  const int64_t nb = (A == B && q->self_join) ? na : window_mesh_bound(B, q->window_lo, q->window_hi);
  // device bytes: every selected pair as a candidate (id pair, flag, output
  // pair), the selections, and the scans over them
  qq->est_bytes = na * nb * 17 + (na + nb) * 24 + 4096;
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
