// Internal data structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pierce.h"

namespace pj {

// ---------------------------------------------------------------------------
// Encodings
// ---------------------------------------------------------------------------
// A wide node of width W is W + 1 slots of 8 32-bit words (32 bytes), so
// that one child is two aligned 16-byte loads:
//   slot 0 (header): lo_x lo_y lo_z hi_x hi_y hi_z 0 0   (the node's own box)
//   slot k + 1:      lo_x lo_y lo_z hi_x hi_y hi_z child 0 (child k)
// A child word is
//   0xFFFFFFFF                 empty slot (its box is inverted: lo > hi)
//   < 2^30                     index of a wide node (global in the dataset)
//   bit 31 | first << 3 | n-1  leaf: n in [1, 8] triangles starting at the
//                              mesh-local sorted position `first` (< 2^28)
// A traversal item is a 32-bit word: an internal wide node index, or
// bit 31 | (node * W + k) for the leaf held in child k of `node`.
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;

__host__ __device__ inline int node_stride_words(int W) { return 8 * (W + 1); }

// Triangle record in BVH-leaf order: three float4
//   r0 = (ax, ay, az, bx)  r1 = (by, bz, cx, cy)  r2 = (cz, owner bits, local id, 0)
// The owner bits (as int) say which of the edges (a,b), (b,c), (c,a) this
// triangle carries in the mesh's unique-edge set.
constexpr int kTriRecF4 = 3;

struct Bvh {
  int W = 0, L = 0;
  int64_t n_nodes = 0;
  int max_depth = 0;
  float *d_nodes = nullptr;        // n_nodes * stride words
  int32_t *d_roots = nullptr;      // per mesh
  int32_t *d_tri_order = nullptr;  // sorted position -> global triangle id
  float4 *d_trirec = nullptr;      // n_tris * 3
  int64_t bytes = 0;
};

struct Dataset {
  int64_t M = 0, V = 0, F = 0, E = 0;
  float *d_xyz = nullptr;       // V * 3
  int32_t *d_tris = nullptr;    // F * 3 global vertex ids
  int64_t *d_voff = nullptr;    // M + 1
  int64_t *d_toff = nullptr;    // M + 1
  std::vector<int64_t> h_voff, h_toff;
  float *d_aabb = nullptr;      // M * 6
  std::vector<float> h_aabb;    // M * 6, host copy (serving window selection)
  int32_t *d_lexorder = nullptr;  // V: global vertex ids, per mesh in (x,y,z) order
  uint8_t *d_emask = nullptr;   // F: owned-edge bits
  // per-mesh record, three float4 (48 B), so that a kernel reaches a mesh's
  // box, first lexicographic vertex and offsets in one aligned fetch:
  //   (lo x y z, v0 x)  (hi x y z, v0 y)  (v0 z, first triangle, first vertex,
  //   vertex count) -- the last three as int bits
  float4 *d_mrec = nullptr;     // M * 3
  std::map<std::pair<int, int>, Bvh> bvhs;
  std::pair<int, int> last_bvh{0, 0};
  // one BVH over all of the dataset's triangles per (W, L), for the
  // dataset-level join; its triangle records carry the owning mesh id
  std::map<std::pair<int, int>, Bvh> dbvhs;
  // serving admission: summed-area table over a kOccG^3 grid of the 2^18
  // cube of the number of meshes whose box touches each cell ((kOccG + 1)^3
  // entries), so that a window's mesh count has an O(1) upper bound
  std::vector<int64_t> occ_sat;
  int64_t bytes = 0;
};

constexpr int kOccG = 32;  // cells per axis of the admission grid (8,192 grid units)
// upper bound on the meshes of d whose closed box meets [lo, hi] (at most M)
int64_t window_mesh_bound(const Dataset *d, const int32_t *lo, const int32_t *hi);

// Counter slots (match pj_counters order)
enum {
  C_PAIRS = 0, C_NODE_PAIRS, C_BOX_TESTS, C_LEAF_PAIRS, C_SLAB_TESTS,
  C_SEGTRI, C_FALLBACK, C_PARITY_RAYS, C_PARITY_NODES, C_PARITY_TRIS,
  C_BYTES, C_HITS, C_SPILLED, C_TASKS, C_BYTES_TASKS,
  C_WARP_NUM = 16,  // the warp-traversal kernels keep these in registers
  C_BYTES_PARITY = 16, C_BYTES_EXPAND, C_BYTES_LEAF, C_PAR_HANDOVER, C_NUM = 20
};

struct Workspace {
  void *ptr = nullptr;
  size_t cap = 0;
  bool zeroed = false;  // ws_get_zeroed: all-zero as of the last use
};

// Scratch of one join in flight: workspaces (grown on demand), the device
// error words and a small pinned host buffer.  The context owns one for its
// API calls; each serving stream has its own.
struct Exec {
  std::map<std::string, Workspace> ws;
  int *d_err = nullptr;      // 4 device error words
  void *h_pinned = nullptr;  // 4 KiB pinned host scratch
  std::string err;           // last failure message of a serving thread
  bool borrow_out = false;   // join results stay in the workspaces (serving)
  cudaEvent_t ev[6] = {};    // a join's phase events, created once
  // a serving slot's stream: its workspaces are released and taken in that
  // stream's order (null: the API calls' scratch, plain cudaMalloc)
  cudaStream_t stream = nullptr;
};

struct Serve;  // serving state (pj_serve.cu)

struct Ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;
  std::mutex err_mu;  // guards err (pj_submit / pj_poll fail outside `mu`)
  std::string err;
  std::map<int, std::unique_ptr<Dataset>> datasets;
  int next_ds = 1;
  unsigned long long *d_counters = nullptr;  // C_NUM
  Exec main;                                 // scratch of the API calls
  pj_config cfg{};
  // captured graphs keyed by a shape string, with their kernel counts
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, unsigned long long> graph_kernels;
  std::atomic<unsigned long long> launches{0};  // kernels launched by joins
  // datasets and their BVHs: serving threads read them under a shared lock,
  // API calls that add or remove one take it exclusively (after `mu`)
  std::shared_mutex ds_rw;
  Serve *serve = nullptr;
  // device buffers of join results (pairs, flags, cycles): pj_free_pairs
  // hands them back here and later joins reuse them, so that neither side
  // pays for cudaMalloc / cudaFree (the latter synchronises the device).
  // pool: free buffers by capacity; cap: capacity of every buffer the pool
  // made, free or lent out.  Guarded by `mu`.
  std::multimap<size_t, void *> pool;
  std::map<void *, size_t> pool_cap;
  size_t pool_bytes = 0;  // capacity of the free buffers
  // the same for host results (pinned memory: cudaMallocHost / cudaFreeHost)
  std::multimap<size_t, void *> hpool;
  std::map<void *, size_t> hpool_cap;
  size_t hpool_bytes = 0;
};

// A device buffer of at least `bytes` from the context's result pool (or a
// new one, its size rounded up to a power of two of at least 4 KiB).
void *pool_get(Ctx *c, size_t bytes, cudaError_t *e);
// Give a buffer back: pooled if the pool made it (and the free buffers stay
// under 1 GiB), else cudaFree.  The caller's work on it must be complete.
void pool_put(Ctx *c, void *p);
void pool_release(Ctx *c);  // free every free pooled buffer (device and host)
// Pinned host buffers for host results, pooled the same way (under 256 MiB
// of free buffers); a pointer the pool did not make is cudaFreeHost'ed.
void *hpool_get(Ctx *c, size_t bytes, cudaError_t *e);
void hpool_put(Ctx *c, void *p);
// Release a result's buffers (pairs, flags, cycles) to where they came from.
void pairs_release(Ctx *c, pj_pairs *r);

// The scratch the calling thread works with: a serving thread's own, else
// the context's.
extern thread_local Exec *t_exec;
inline Exec *cur_exec(Ctx *c) { return t_exec ? t_exec : &c->main; }
pj_status exec_init(Ctx *ctx, Exec *e);
void exec_free(Exec *e);
void serve_stop(Ctx *ctx);
pj_status serve_submit(Ctx *ctx, Dataset *A, Dataset *B, const pj_query *q, pj_ticket *out);
pj_status serve_poll(Ctx *ctx, pj_ticket t, int wait, pj_pairs *out, pj_query_stats *stats);
bool serve_uses(Ctx *ctx, const Dataset *d);  // pending or running queries on d

// set ctx->err and return code
pj_status fail(Ctx *c, pj_status code, const std::string &msg);
pj_status cuda_fail(Ctx *c, cudaError_t e, const char *what);
void clear_err(Ctx *c);
void *ws_get(Ctx *c, const char *name, size_t bytes, pj_status *st);
// A workspace whose users leave it all-zero: cleared on stream s when it is
// (re)allocated or was marked dirty (a launch that used it failed).
void *ws_get_zeroed(Ctx *c, const char *name, size_t bytes, cudaStream_t s, pj_status *st);
void ws_mark_dirty(Ctx *c, const char *name);

#define PJ_CK(call)                                   \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
  } while (0)

// device error codes written by kernels
enum { DERR_NONE = 0, DERR_STACK = 1, DERR_QUEUE = 2, DERR_OFFSET = 3, DERR_TIMEOUT = 4 };

// build.cu
pj_status build_bvh(Ctx *ctx, Dataset *ds, int W, int L, cudaStream_t s);
void free_bvh(Bvh &b);
// tune.cu
pj_status run_autotune(Ctx *ctx, Dataset *A, Dataset *B, const int32_t *cand, int64_t n_cand,
                       int self_join, const pj_tune_space *space, pj_join_opts *best,
                       pj_tune_entry *table, int table_cap, int *table_n);
// join.cu
// safe: plain depth-first refinement and the multi-pass box join and
// compaction (no kernel waits on another block); the join redoes itself this
// way when a bounded wait of the default kernels ran out
pj_status run_join(Ctx *ctx, Dataset *A, Dataset *B, const int32_t *cand,
                   const int32_t *cand_off, int64_t n_cand, int cand_on_device,
                   int self_join, const pj_join_opts *opts, cudaStream_t s,
                   pj_pairs *out, bool safe = false);
pj_status run_estimate(Ctx *ctx, Dataset *A, Dataset *B, int G, double *cells_out,
                       pj_estimate *out, cudaStream_t s);
// load meshes (host or device arrays) into *d, and free a dataset's buffers
pj_status load_impl(Ctx *ctx, const float *xyz, int64_t V, const int32_t *tris, int64_t F,
                    const int64_t *voff, const int64_t *toff, int64_t M, int dev_ptrs,
                    Dataset *d);
void free_dataset(Dataset *d);
pj_status run_join_tiled(Ctx *ctx, const pj_host_meshes *A, const pj_host_meshes *B,
                         int self_join, const pj_tiled_opts *o, pj_pairs *out,
                         pj_tiled_stats *stats);
pj_status run_dataset_join(Ctx *ctx, Dataset *A, Dataset *B, int self_join,
                           const pj_dsjoin_opts *o, pj_pairs *out, pj_dsjoin_stats *stats,
                           cudaStream_t s);
pj_status run_join_noalloc(Ctx *ctx, Dataset *A, Dataset *B, const int32_t *d_cand,
                           int64_t n, uint8_t *d_flags, int32_t *d_pairs, int64_t *d_count,
                           cudaStream_t s);
pj_status run_segtri_batch(Ctx *ctx, const float *pq, const float *abc,
                           int64_t n, int mode, uint8_t *res,
                           int64_t *n_fallback, cudaStream_t s);

// the bounding-box filter join by sort and sweep along x (pj_mbb.cu): the
// candidate pairs in (id A, id B) order in the "cand" workspace, their count
// in *d_count (device) and *C (host)
pj_status mbb_sweep(Ctx *ctx, const Dataset *A, const Dataset *B, bool self_join,
                    cudaStream_t s, int64_t *d_count, int32_t **d_cand, int64_t *C);

// exclusive scan of n int64 values (device), total -> *d_total (device)
pj_status scan_i64(Ctx *ctx, const int64_t *d_in, int64_t *d_out, int64_t n,
                   int64_t *d_total, cudaStream_t s);

inline int blocks_for(int64_t n, int t) {
  int64_t b = (n + t - 1) / t;
  if (b < 1) b = 1;
  if (b > (1 << 30)) b = 1 << 30;
  return (int)b;
}

}  // namespace pj
