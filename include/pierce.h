/*
 * pierce.h -- C ABI of the GB300 (sm_103a) refinement library for the 3-D
 * intersection join of closed triangle meshes.
 *
 * Method (paper "Pierce: GPU Ray Tracing for Spatial Joins over Complex 3D
 * Data"): a pair of closed meshes (A, B) intersects when an edge of one mesh
 * pierces a triangle of the other (Sec. 3.1 observation 1; both directions,
 * Sec. 3.2 "Bidirectional tracing"), or when one mesh lies inside the other
 * by the parity of a +z ray cast from a representative vertex (Alg. 2,
 * Sec. 3.3); the intersection join is the union of the two (Sec. 3.4).
 *
 * Exact semantics fixed by this library (the paper works in FP32):
 *   - coordinates are integers in [0, 2^18) stored as float32, so every
 *     orientation sign is decided exactly (FP32 filter, int64 fallback);
 *   - "pierce" = the open edge segment crosses the open triangle
 *     transversally (tangential contact never counts, Sec. 3.6);
 *   - the representative vertex of B w.r.t. A is B's lexicographically
 *     smallest (x, y, z) vertex that is not on A's closed surface; the +z ray
 *     is perturbed symbolically to (x + e, y + e^2).
 *
 * Conventions for every function:
 *   - the return value is a pj_status; PJ_OK on success.  No C++ exception
 *     crosses this interface.  pj_last_error() gives a message for the last
 *     failure on a context.
 *   - "device" pointers are CUDA device pointers on the context's device;
 *     "host" pointers are ordinary (pageable or pinned) host memory.
 *   - the library copies every input it keeps; the caller keeps ownership of
 *     its buffers and may free them when the call returns.
 *   - calls on one context are serialised by an internal lock, except
 *     pj_poll/pj_submit which may be called from any thread.
 */
#ifndef PIERCE_H
#define PIERCE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pj_status;

enum {
  PJ_OK = 0,
  PJ_ERR_INVALID_ARG = 1,   /* bad pointer, size, handle or option          */
  PJ_ERR_NOT_QUANTIZED = 2, /* a coordinate is not an integer in [0, 2^18)  */
  PJ_ERR_NOT_MANIFOLD = 3,  /* an undirected edge is not used exactly twice,
                               or a triangle repeats a vertex                */
  PJ_ERR_NO_MEMORY = 4,     /* a device or host allocation failed           */
  PJ_ERR_BUSY = 5,          /* serving: the query can never fit the budget  */
  PJ_ERR_TIMEOUT = 6,       /* a bounded wait gave up                       */
  PJ_ERR_CUDA = 7,          /* a CUDA runtime call failed                   */
  PJ_ERR_INTERNAL = 8,      /* a device-side capacity check failed          */
  PJ_PENDING = 9            /* serving: the query has not finished yet      */
};

typedef struct pj_ctx pj_ctx;
typedef int32_t pj_dataset;         /* handle returned by pj_load_meshes */

/* Context configuration.  Zero-initialise and set what you need. */
typedef struct {
  int32_t device;            /* CUDA device ordinal                            */
  int32_t reserved0;
  int64_t budget_bytes;      /* serving admission budget; 0 = 40 GiB           */
  int64_t wait_limit_us;     /* bound on host waits in pj_poll(block); 0 = 10 s */
  int32_t serve_streams;     /* concurrent serving batches; 0 = 4              */
  int32_t reserved1;
} pj_config;

/* BVH shape: width W in {2, 4, 8} children per node, leaf size L in
 * {1, 2, 4, 8} triangles.  Zero fields pick W = 4, L = 4. */
typedef struct {
  int32_t width;
  int32_t leaf_size;
} pj_bvh_params;

enum { PJ_LEAF_FILTERED = 0, PJ_LEAF_EXACT = 1 };
/* pj_segtri_batch only: the FP32 filter with the static bound of the five
 * points' box (the form the streaming kernel uses, with one bound per leaf
 * pair) */
enum { PJ_LEAF_STATIC = 2 };
enum { PJ_LAUNCH_PERSISTENT = 0, PJ_LAUNCH_PER_PAIR = 1 };
enum { PJ_FRONT_NONE = -1, PJ_FRONT_STREAM = -2 };  /* pj_join_opts.wave_levels */
/* pj_join_opts.predicate: the paper's join predicates (Sec. 3.2-3.4).  With
 * cross(A_i, B_j) = an edge of one mesh strictly pierces a triangle of the
 * other (Sec. 3.2, both directions) and inside(X, Y) = X's representative
 * vertex (its lexicographically smallest vertex off Y's surface) has odd
 * ray parity against Y (Sec. 3.3):
 *   PJ_PRED_INTERSECTS  cross OR inside(B_j, A_i) OR inside(A_i, B_j)  (Sec. 3.4)
 *   PJ_PRED_OVERLAP     cross                                           (Sec. 3.2)
 *   PJ_PRED_CONTAINS    A_i contains B_j: no cross AND inside(B_j, A_i) (Alg. 2)
 *   PJ_PRED_WITHIN      A_i within B_j:  no cross AND inside(A_i, B_j)
 *   PJ_PRED_ANY_VERTEX  intersects, or some vertex of either mesh strictly
 *                       inside the other (off its surface, odd parity): a
 *                       completeness mode for meshes whose surfaces cross
 *                       only through edges and vertices, which the strict
 *                       crossing test does not see.  It tests every vertex in
 *                       the other mesh's box, so it costs far more. */
enum { PJ_PRED_INTERSECTS = 0, PJ_PRED_OVERLAP = 1, PJ_PRED_CONTAINS = 2, PJ_PRED_WITHIN = 3,
       PJ_PRED_ANY_VERTEX = 4 };

/* Options of one join.  Zero-initialised = defaults. */
typedef struct {
  int32_t width;            /* which cached BVH to use; 0 = the dataset's last build */
  int32_t leaf_size;
  int32_t warps_per_pair;   /* 1, 2 or 4 warps cooperate on one pair; 0 = 1 */
  int32_t leaf_mode;        /* PJ_LEAF_FILTERED (FP32 filter, int64 fallback)
                               or PJ_LEAF_EXACT (int64 only)                 */
  int32_t launch_mode;      /* PJ_LAUNCH_PERSISTENT: one work-stealing launch;
                               PJ_LAUNCH_PER_PAIR: one launch per candidate  */
  int32_t use_graph;        /* replay the device part as a captured CUDA graph */
  int32_t out_host;         /* 1: result pairs in library-owned host memory   */
  int32_t keep_flags;       /* 1: also return the per-candidate result bytes  */
  int32_t record_cycles;    /* 1: also return each candidate's SM clock cycles
                               (instrumentation of per-pair cost)            */
  int32_t spill_budget;     /* per-warp passes (wave_levels != 0): SM clock
                               cycles a warp spends on one pair in the first
                               pass before handing the rest of it to later
                               passes (0: 40,000; < 0: never); the second
                               pass allows 8 times as many                   */
  int32_t wave_levels;      /* refinement front end.  0 or PJ_FRONT_STREAM:
                               the streaming kernel (one persistent launch;
                               warps keep the tasks of many pairs in shared
                               memory, stage nodes and triangles with
                               asynchronous copies and balance the load
                               through a device task queue).  > 0: this many
                               BVH levels breadth-first, one thread per child
                               test, then the per-warp passes.
                               PJ_FRONT_NONE: the per-warp passes alone      */
  int32_t kernel_times;     /* 1: also time the front end's launches with CUDA
                               events (pj_pairs.expand_ms / leaf_ms; events
                               between launches cost a little overlap)       */
  int32_t wait_polls;       /* bound on the polls of each wait of the
                               streaming kernel (0: 2^19, about half a
                               second) and of the single-pass box join and
                               compaction (0: 2^20); a wait that runs out
                               sets an error word and the join is redone by
                               plain depth-first traversal with the
                               multi-pass box join and compaction (same
                               result, slower)                              */
  int32_t predicate;        /* PJ_PRED_* (0: intersects)                     */
} pj_join_opts;

/* Result of a join.  Owned by the library until pj_free_pairs. */
typedef struct {
  int64_t count;            /* number of intersecting pairs K                 */
  int32_t *pairs;           /* K x 2 (idA, idB), in candidate order: sorted
                               and unique when the candidates are            */
  int32_t on_device;        /* 1 if pairs is a device pointer                 */
  int32_t pairs_malloc;     /* 1 if pairs is plain malloc'd host memory
                               (results of pj_poll); 0 otherwise             */
  int64_t n_candidates;     /* C: candidates refined                          */
  uint8_t *flags;           /* device, C bytes (only with keep_flags)         */
  float device_ms;          /* device time of the join, candidates to
                               compacted pairs (CUDA events on the stream)    */
  float mbb_ms;             /* of which: bounding-box filter join             */
  float refine_ms;          /* of which: refinement (crossing + parity)       */
  float compact_ms;         /* of which: compaction                           */
  float parity_ms;          /* refinement phases (CUDA events; -1 when the
                               join was replayed from a graph): parity rays, */
  float front_ms;           /* front end (the streaming launch, or the
                               breadth-first levels and leaf pairs),         */
  float tasks_ms;           /* and the per-warp passes over what was left     */
  float expand_ms;          /* with pj_join_opts.kernel_times: the streaming
                               launch, or the summed durations of the
                               breadth-first node-pair launches,              */
  float leaf_ms;            /* and of the breadth-first leaf-pair launches
                               (0 with the streaming front end)               */
  float reserved3;
  uint32_t *cycles;         /* device, C values (only with record_cycles):
                               clock64 cycles the refinement spent on each
                               candidate (saturated at 2^32 - 1)              */
  void *impl;
} pj_pairs;

/* Device counters, accumulated over joins until pj_reset_counters. */
typedef struct {
  uint64_t pairs_refined;       /* candidate pairs processed                    */
  uint64_t node_pairs;          /* (node, node) traversal steps                 */
  uint64_t box_tests;           /* child-box overlap tests                      */
  uint64_t leaf_pairs;          /* (leaf, leaf) pairs tested                    */
  uint64_t edge_slab_tests;     /* segment vs leaf-box tests (slab tests; in the
                                   streaming kernel edge-box overlap tests)     */
  uint64_t segtri_tests;        /* strict segment/triangle tests                */
  uint64_t exact_fallbacks;     /* of those, decided by the int64 path          */
  uint64_t parity_rays;         /* +z parity traversals                         */
  uint64_t parity_nodes;        /* nodes visited by parity traversals           */
  uint64_t parity_tri_tests;    /* triangles tested by parity traversals        */
  uint64_t bytes_fetched;       /* algorithmic bytes: nodes, triangles, vertices */
  uint64_t pairs_hit;           /* pairs found intersecting                     */
  uint64_t kernel_launches;     /* kernels launched by joins (host count)       */
  uint64_t tasks_spilled;       /* traversal tasks (streaming: and leaf pairs) handed to another warp or pass */
  uint64_t tasks_resumed;       /* of those, taken up by another warp or pass    */
  uint64_t bytes_tasks;         /* of bytes_fetched: the per-warp passes (with
                                   the streaming front end: the long parity
                                   rays its warps take, also in bytes_parity) */
  uint64_t bytes_parity;        /* of bytes_fetched: the parity rays            */
  uint64_t bytes_expand;        /* of bytes_fetched: breadth-first node pairs   */
  uint64_t bytes_leaf;          /* of bytes_fetched: breadth-first leaf pairs   */
  uint64_t parity_handed_over;  /* parity rays passed from a thread to a warp   */
} pj_counters;

/* Dataset summary. */
typedef struct {
  int64_t n_meshes, n_verts, n_tris, n_edges;
  int64_t bvh_nodes;            /* wide nodes of the last build (0 if none)     */
  int32_t bvh_width, bvh_leaf_size;
  int32_t bvh_max_depth;        /* deepest wide-node level (root = 1)           */
  int32_t reserved;
  int64_t device_bytes;         /* device memory held by the dataset            */
} pj_dataset_info;

/* --------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------ */

/* Create a context on cfg->device (cfg may be NULL: device 0, defaults).
 * *out receives the context; free it with pj_destroy. */
pj_status pj_create(const pj_config *cfg, pj_ctx **out);

/* Destroy a context and free every dataset, BVH and result it owns.  Results
 * not yet freed become invalid. */
pj_status pj_destroy(pj_ctx *ctx);

/* Message of the last failure on ctx (never NULL; "" if none).  The string is
 * owned by the context and valid until the next call on it. */
const char *pj_last_error(pj_ctx *ctx);

/* --------------------------------------------------------------------------
 * Loading (paper Sec. 4.2 "Preprocessing" / "Loading": flat triangles with a
 * triangle-to-object map and per-object unique edges, Sec. 3.1 Step I)
 * ------------------------------------------------------------------------ */

/* Load a dataset of n_meshes closed meshes.
 *   xyz            n_verts x 3 float32 (x, y, z interleaved); every value an
 *                  integer in [0, 2^18)                 -> else PJ_ERR_NOT_QUANTIZED
 *   tris           n_tris x 3 int32, vertex ids local to the mesh
 *   mesh_vert_off  n_meshes + 1 int64, mesh k owns vertices [off[k], off[k+1])
 *   mesh_tri_off   n_meshes + 1 int64, mesh k owns triangles [off[k], off[k+1])
 *   ptr_is_device  0: the four arrays are host pointers; 1: xyz and tris are
 *                  device pointers (the offsets are always host pointers)
 * Each mesh must be a closed 2-manifold: every undirected edge used by
 * exactly two of its triangles, no triangle repeating a vertex
 * (-> PJ_ERR_NOT_MANIFOLD; pj_last_error names the mesh).  Meshes hold at most
 * 2^28 - 2 triangles; a dataset at most 2^31 - 1 triangles and vertices.
 * The library computes per-mesh bounding boxes, the unique edges (each owned
 * by one triangle) and each mesh's vertices in lexicographic order.
 * *out receives the dataset handle.  Synchronous. */
pj_status pj_load_meshes(pj_ctx *ctx, const float *xyz, int64_t n_verts,
                         const int32_t *tris, int64_t n_tris,
                         const int64_t *mesh_vert_off,
                         const int64_t *mesh_tri_off, int64_t n_meshes,
                         int32_t ptr_is_device, pj_dataset *out);

/* Free a dataset and its BVHs. */
pj_status pj_free_dataset(pj_ctx *ctx, pj_dataset ds);

/* Build (or reuse from the cache) the per-mesh BVHs of a dataset: an LBVH
 * over 30-bit Morton codes of triangle centroids (Karras 2012), exact integer
 * boxes, collapsed to W-wide nodes with leaves of at most L triangles.  The
 * BVH stays resident, cached per (W, L); params may be NULL (W = 4, L = 4).
 * Synchronous. */
pj_status pj_build_bvh(pj_ctx *ctx, pj_dataset ds, const pj_bvh_params *params);

pj_status pj_dataset_info_get(pj_ctx *ctx, pj_dataset ds, pj_dataset_info *out);

/* --------------------------------------------------------------------------
 * Join (paper Sec. 3.4 intersection join over candidate pairs)
 * ------------------------------------------------------------------------ */

/* Refine candidate pairs (idA in a, idB in b) with the intersection
 * predicate and return the intersecting ones.
 *   cand_pairs  n_cand x 2 int32 host pointer, or NULL: the candidates are
 *               then produced on the device by the bounding-box filter join
 *               (closed mesh boxes meet), in (idA, idB) lexicographic order
 *   self_join   1: a == b and only pairs with idA < idB are considered
 *   cuda_stream cudaStream_t to order the work on (NULL: the context's stream)
 *   out         filled with the result; free with pj_free_pairs
 * Both datasets need a BVH (pj_build_bvh).  Returns when the result is
 * complete (the stream is synchronised). */
pj_status pj_join_intersects(pj_ctx *ctx, pj_dataset a, pj_dataset b,
                             const int32_t *cand_pairs, int64_t n_cand,
                             int32_t self_join, void *cuda_stream,
                             pj_pairs *out);

/* As pj_join_intersects, with options and per-candidate translations.
 *   cand_offsets  NULL, or n_cand x 3 int32 host pointer: candidate c tests
 *                 A_i against B_j translated by cand_offsets[c] (integer grid
 *                 units; the translated mesh must stay in [0, 2^18)).  Lets
 *                 many placements share one resident mesh and BVH.
 *   cand_on_device 1: cand_pairs / cand_offsets are device pointers.
 *   opts          may be NULL (defaults). */
pj_status pj_join_intersects_ex(pj_ctx *ctx, pj_dataset a, pj_dataset b,
                                const int32_t *cand_pairs,
                                const int32_t *cand_offsets, int64_t n_cand,
                                int32_t cand_on_device, int32_t self_join,
                                const pj_join_opts *opts, void *cuda_stream,
                                pj_pairs *out);

/* Free a join result.  Device buffers (pairs with out_host = 0, flags,
 * cycles) go back to a pool of the context that later joins reuse instead of
 * calling cudaMalloc / cudaFree: any work of the caller that reads them must
 * have completed.  Host pairs of pj_join_intersects[_ex] (out_host = 1) are
 * pinned buffers that go back to a pool of their own the same way
 * (cudaMallocHost / cudaFreeHost are not paid per join); the caller must not
 * touch them afterwards.  pj_destroy frees both pools. */
pj_status pj_free_pairs(pj_ctx *ctx, pj_pairs *res);

/* The join's device part with no allocation at all (the paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- loops that must not stall on the allocator's implicit device
 * synchronisation, or programs whose device memory belongs to another
 * allocator or budget, such as a framework's caching allocator or a pool
 * sized at start-up).  It calls no cudaMalloc, cudaFree or allocating
 * library routine; every buffer is the caller's:
 *   d_cand   device, n_cand x 2 int32 candidates (idA in a, idB in b)
 *   d_flags  device, n_cand bytes: 1 where the candidate intersects
 *   d_pairs  device, room for n_cand x 2 int32: the intersecting candidates
 *            in candidate order
 *   d_count  device, one int64: the number of pairs, or -1 if a device-side
 *            check failed (a candidate id out of range)
 * Uses each dataset's last-built BVH; the two must have the same width and
 * leaf size (else PJ_ERR_INVALID_ARG, nothing queued).  Runs the FP32 filter
 * with int64 fallback, one warp per pair and plain depth-first traversal.
 * A candidate id out of range is skipped (its flag stays 0) and makes
 * *d_count -1; the next call clears that state.  Asynchronous: the work is enqueued on cuda_stream (NULL: the
 * context's stream) and the outputs are valid once it has completed.
 * n_cand above 16,777,216 is rejected with PJ_ERR_INVALID_ARG.
 * Scratch: a 65,600-byte array in device global memory, defined at file
 * scope in the library; every GPU that loads the library holds it until the
 * process exits.  The first call on a device looks up the array's device
 * address (make that first call before any stream capture).  All calls on a
 * device share the array, which keeps the last call's contents (each call
 * clears the parts that must start at zero): calls whose work overlaps on
 * the GPU race, so order them on one stream or synchronise between them.
 * Lifetime: the queued work reads both datasets' BVHs, triangles and vertices
 * until it completes.  pj_free_dataset and pj_destroy wait for the whole
 * device before they free anything, but the caller must not queue such work
 * after freeing a dataset it reads. */
pj_status pj_join_intersects_noalloc(pj_ctx *ctx, pj_dataset a, pj_dataset b,
                                     const int32_t *d_cand, int64_t n_cand,
                                     uint8_t *d_flags, int32_t *d_pairs,
                                     int64_t *d_count, void *cuda_stream);

/* --------------------------------------------------------------------------
 * Out-of-core execution by grid tiling (paper Sec. 3.6, "Out-of-GPU-core
 * execution")
 * ------------------------------------------------------------------------ */

/* Meshes in host memory, in the layout of pj_load_meshes. */
typedef struct {
  const float *xyz;              /* n_verts x 3, integer valued in [0, 2^18)  */
  const int32_t *tris;           /* n_tris x 3, mesh-local vertex ids          */
  const int64_t *mesh_vert_off;  /* n_meshes + 1                               */
  const int64_t *mesh_tri_off;   /* n_meshes + 1                               */
  int64_t n_meshes;
} pj_host_meshes;

typedef struct {
  int64_t device_budget;    /* device bytes one cell's meshes and BVHs may
                               take (0: a quarter of the free memory)        */
  int32_t grid;             /* cells per axis (0: the smallest power of two,
                               at most 16, whose cells fit the budget)       */
  int32_t width;            /* per-cell BVH shape (0: 4)                     */
  int32_t leaf_size;        /* (0: 2)                                        */
  int32_t out_host;         /* 1: pairs in library-owned host memory          */
  pj_join_opts join;        /* each cell's join (predicate, leaf mode, ...)  */
} pj_tiled_opts;

typedef struct {
  int32_t grid;             /* cells per axis used                           */
  int32_t reserved;
  int64_t cells_joined;     /* cells holding meshes of both datasets         */
  int64_t mesh_copies;      /* meshes uploaded, replicas across cells included */
  int64_t max_cell_bytes;   /* largest cell's estimated device footprint     */
  int64_t pairs_in_cells;   /* pairs the cells reported, before each pair is
                               kept in the one cell that holds its reference
                               point                                          */
  float ms_total;           /* wall time of the whole join                   */
  float ms_gather;          /* host time gathering cells (overlapped)        */
  float ms_device;          /* load, BVH build and join of the cells         */
  float reserved2;
} pj_tiled_stats;

/* A join of two datasets that need not fit in device memory: a coarse grid
 * over both datasets' box, each mesh copied to every cell its closed box
 * touches, the cells loaded, indexed and joined one after another with the
 * same kernels as pj_join_intersects_ex (the next cell is gathered on the
 * host while the current one runs).  A pair is kept only in the cell that
 * holds the lower corner of its two boxes' intersection, a point of both
 * boxes, so every pair is reported exactly once.  Global mesh ids, sorted.
 * self_join: b is ignored (a with itself, pairs i < j).  A mesh larger than
 * the budget fails with PJ_ERR_NO_MEMORY.  Synchronous. */
pj_status pj_join_tiled(pj_ctx *ctx, const pj_host_meshes *a, const pj_host_meshes *b,
                        int32_t self_join, const pj_tiled_opts *opts, pj_pairs *out,
                        pj_tiled_stats *stats);

/* --------------------------------------------------------------------------
 * Dataset-level join (the paper's formulation, Sec. 3.1-3.5)
 * ------------------------------------------------------------------------ */

/* How the deduplicated pair set is materialised (Sec. 3.5, Fig. 5). */
enum {
  PJ_MAT_ESTIMATED = 0,   /* one tracing pass inserting pairs into a hashmap
                             of pj_estimate_join's slot count (doubled and
                             rerun if it overflows)                          */
  PJ_MAT_TWO_PASS = 1,    /* a counting pass, a prefix sum, an emitting pass
                             into a flat buffer, then sort and unique        */
  PJ_MAT_FIXED = 2        /* one pass into a hashmap of a fixed slot count   */
};

typedef struct {
  int32_t width;            /* W of the dataset BVHs (0: 4)                  */
  int32_t leaf_size;        /* L (0: 2)                                      */
  int32_t predicate;        /* PJ_PRED_INTERSECTS or PJ_PRED_OVERLAP          */
  int32_t materialize;      /* PJ_MAT_*                                      */
  int64_t fixed_slots;      /* PJ_MAT_FIXED: hashmap slots (0: 2^26)         */
  int32_t grid;             /* estimate grid per axis (0: 16)                */
  int32_t out_host;         /* 1: pairs in library-owned host memory          */
} pj_dsjoin_opts;

typedef struct {
  int64_t edges;            /* owned edges traced (both directions)          */
  int64_t node_visits;      /* BVH nodes visited by edges and parity rays    */
  int64_t tri_tests;        /* strict segment/triangle tests                 */
  int64_t hits;             /* crossings found, repeats included             */
  int64_t parity_rays;      /* one per object with a vertex in the other box */
  int64_t recheck_pairs;    /* pairs the per-pair join decided (a parity
                               vertex on a surface, or a ray that met more
                               candidate objects than it can track)          */
  int64_t slots;            /* hashmap slots, or flat records (two-pass)     */
  int32_t relaunches;       /* hashmap overflows (each doubles the table)    */
  int32_t reserved;
  double estimate;          /* E_final used for sizing (estimated mode)      */
  float ms_total;           /* device time of the join (CUDA events)         */
  float ms_estimate;        /* of which: the estimate                        */
  float ms_trace;           /* tracing passes (edges and parity rays)        */
  float ms_materialize;     /* hashmap extraction or sort, unique, output    */
} pj_dsjoin_stats;

/* The join as the paper formulates it, without candidate pairs: one BVH
 * over all triangles of each dataset (built and cached per W, L on first
 * use); every owned edge of A traced as a bounded segment through B's BVH
 * and every owned edge of B through A's (Alg. 1 both ways, Sec. 3.2), every
 * strict crossing recorded (the multi-hit loop: an edge may pierce several
 * objects) as the pair (idA, idB), duplicates merged by the chosen
 * materialisation (Sec. 3.5).  For PJ_PRED_INTERSECTS each object also casts
 * one parity ray from its lexicographically first vertex against the other
 * dataset's BVH, toggling a parity bit per object it crosses (Sec. 3.3-3.4);
 * odd parity with the vertex off that object's surface records the pair.
 * Where the vertex lies on a surface, or the ray meets more objects whose
 * box holds the vertex than it tracks, those pairs are decided by the
 * per-pair join instead, so the result equals pj_join_intersects over the
 * bounding-box candidates exactly.  self_join: a == b, pairs i < j.
 * out: sorted unique pairs (free with pj_free_pairs); stats may be NULL.
 * Synchronous. */
pj_status pj_dataset_join(pj_ctx *ctx, pj_dataset a, pj_dataset b, int32_t self_join,
                          const pj_dsjoin_opts *opts, pj_pairs *out, pj_dsjoin_stats *stats);

/* --------------------------------------------------------------------------
 * Selectivity estimate (paper Sec. 3.5, "Result Materialization")
 * ------------------------------------------------------------------------ */

typedef struct {
  double e_final;           /* expected intersecting pairs: sum over the grid
                               cells of N_1 N_2 min(P_base F_shape, 1)       */
  double slots;             /* hashmap slots: e_final / 0.5 (load factor)    */
  int64_t cells_occupied;   /* cells touched by objects of both datasets     */
  int32_t grid;             /* G: cells per axis                             */
  float ms;                 /* device time (CUDA events)                     */
} pj_estimate;

/* The paper's estimate of a join's result size, from per-cell statistics of
 * a G x G x G grid over the box of both datasets (Sec. 3.5): per cell and
 * dataset k the number N_k of objects whose closed box touches the cell,
 * their mean box side S_k and mean mesh-to-box volume ratio; P_base =
 * (S_1 + S_2 + 1e-3)^3 / V_cell (the Minkowski sum of two cubes), F_shape =
 * sqrt(VolRatio_1 VolRatio_2)^0.8, E_i = N_1 N_2 min(P_base F_shape, 1).
 * Lengths are in units of the grid extent (coordinates / (2^18 - 1)).
 * grid: G in [1, 256] (0: 16).  cells_out: NULL, or a host array of G^3
 * doubles that receives each cell's E_i (index (x G + y) G + z).  Reads only
 * the datasets' meshes and boxes (no BVH needed).  Synchronous. */
pj_status pj_estimate_join(pj_ctx *ctx, pj_dataset a, pj_dataset b, int32_t grid,
                           double *cells_out, pj_estimate *out);

/* --------------------------------------------------------------------------
 * Autotuning (the paper has no counterpart: its parameters are fixed by
 * OptiX; here BVH width, leaf size, warps per pair and the depth of the
 * breadth-first front end are chosen per dataset pair by measurement)
 * ------------------------------------------------------------------------ */

/* The configurations to try: every combination of the listed values. */
typedef struct {
  int32_t widths[3];        /* subset of {2, 4, 8}                           */
  int32_t n_widths;
  int32_t leaf_sizes[4];    /* subset of {1, 2, 4, 8}                        */
  int32_t n_leaf_sizes;
  int32_t warps[3];         /* subset of {1, 2, 4}                           */
  int32_t n_warps;
  int32_t wave_levels[4];   /* values of pj_join_opts.wave_levels            */
  int32_t n_wave_levels;
  int32_t sample_permille;  /* calibration sample, per mille of the
                               candidates (0: 20, i.e. 2 %; at least 1,000
                               candidates or all of them)                   */
  int32_t repeats;          /* timed joins per configuration (0: 3)          */
  uint64_t seed;            /* sample seed                                   */
} pj_tune_space;

/* One measured configuration. */
typedef struct {
  int32_t width, leaf_size, warps_per_pair, wave_levels;
  float ms;                 /* median device time of the join on the sample  */
  float reserved;
} pj_tune_entry;

/* Measure every configuration of *space on a seeded sample of the
 * candidates (cand: n_cand x 2 host array, or NULL for the bounding-box
 * candidates) and return the fastest as *best (a complete pj_join_opts with
 * that width, leaf size, warps per pair and front-end depth, other fields
 * default).  table (may be NULL) receives up to table_cap entries in the
 * order measured, *table_n (may be NULL) their count.  Builds the BVHs the
 * space needs; the ones it built that did not win are freed again.
 * Synchronous. */
pj_status pj_autotune(pj_ctx *ctx, pj_dataset a, pj_dataset b,
                      const int32_t *cand, int64_t n_cand, int32_t self_join,
                      const pj_tune_space *space, pj_join_opts *best,
                      pj_tune_entry *table, int32_t table_cap, int32_t *table_n);

/* --------------------------------------------------------------------------
 * Serving (the paper has no counterpart: it runs one join at a time, Sec. 4;
 * this is the request loop around the same refinement)
 *
 * A query asks for the intersecting pairs among the meshes of datasets a and
 * b whose closed bounding boxes meet a closed window box.  pj_submit queues
 * it and returns at once; pj_poll collects the answer.  Queued queries are
 * admitted oldest first while the device bytes of the admitted ones stay
 * within pj_config.budget_bytes (0: 40 GiB), and a free serving stream
 * (pj_config.serve_streams, 0: 4) takes every admissible queued query on the
 * same datasets as one batch: the bounding-box filter over the queries'
 * selections, one refinement of all their candidates, and a per-query split
 * of the result.  Batches on different streams run concurrently.  A query's
 * answer does not depend on what it was batched with.
 *
 * Both datasets need a BVH of the same shape (their last pj_build_bvh).  The
 * first pj_submit on a context starts the serving threads and gives each its
 * own stream and scratch (about 0.7 GB of device memory per stream, outside
 * the budget).  pj_free_dataset answers PJ_ERR_BUSY while queries on the
 * dataset have not been polled; pj_build_bvh and pj_autotune wait for the
 * running batches.
 * ------------------------------------------------------------------------ */

typedef int64_t pj_ticket;

typedef struct {
  pj_dataset a, b;
  int32_t self_join;        /* 1: a == b and only pairs idA < idB             */
  int32_t window_lo[3];     /* closed window box, grid units                  */
  int32_t window_hi[3];
  int32_t reserved;
} pj_query;

/* Timings of one query (seconds on the host's steady clock) and its sizes. */
typedef struct {
  double t_submit;          /* pj_submit returned the ticket                  */
  double t_admit;           /* taken into a batch                             */
  double t_launch;          /* the batch's refinement was enqueued            */
  double t_done;            /* the batch's results were on the host           */
  int64_t n_a, n_b;         /* meshes selected by the window on each side     */
  int64_t n_candidates;     /* pairs whose boxes meet                         */
  int64_t n_pairs;          /* intersecting pairs                             */
  int64_t device_bytes;     /* bytes admitted against the budget              */
  int32_t batch_id;         /* batch the query ran in                         */
  int32_t batch_queries;    /* queries in that batch                          */
} pj_query_stats;

/* Queue a query.  *out receives its ticket.  A query that needs more device
 * bytes than the whole budget is refused with PJ_ERR_BUSY.  May be called
 * from any thread. */
pj_status pj_submit(pj_ctx *ctx, const pj_query *q, pj_ticket *out);

/* Collect a query.  wait = 0: returns PJ_PENDING while it is not done;
 * wait = 1: blocks until it is done, at most pj_config.wait_limit_us (0:
 * 10 s; then PJ_ERR_TIMEOUT and the ticket stays valid).  When done, *out
 * receives the pairs (host memory, sorted by (idA, idB); free with
 * pj_free_pairs), stats (may be NULL) the timings, and the ticket is
 * released.  May be called from any thread. */
pj_status pj_poll(pj_ctx *ctx, pj_ticket ticket, int32_t wait, pj_pairs *out,
                  pj_query_stats *stats);

/* --------------------------------------------------------------------------
 * Counters and diagnostics
 * ------------------------------------------------------------------------ */

pj_status pj_get_counters(pj_ctx *ctx, pj_counters *out);
pj_status pj_reset_counters(pj_ctx *ctx);

/* Leaf predicate on explicit segments and triangles (all device pointers,
 * float32 integer-valued coordinates): res[k] = 1 if the open segment
 * (p[k], q[k]) crosses the open triangle (a[k], b[k], c[k]) transversally.
 * pq: n x 6 (p then q), abc: n x 9.  mode: PJ_LEAF_FILTERED (per-test
 * error bound), PJ_LEAF_STATIC (static bound of the points' box) or
 * PJ_LEAF_EXACT.  n_fallback (host, may be NULL) receives how many tests the
 * FP32 filter could not decide. */
pj_status pj_segtri_batch(pj_ctx *ctx, const float *pq, const float *abc,
                          int64_t n, int32_t mode, uint8_t *res,
                          int64_t *n_fallback, void *cuda_stream);

/* Copy a dataset's BVH (built with width W, leaf size L) to host buffers for
 * inspection.  Pass NULL buffers to query the sizes first.
 *   nodes      n_nodes x 8 (W + 1) 32-bit words: W + 1 slots of 8 words; slot
 *              0 = the node's own box (lo x y z, hi x y z, 0, 0), slot k + 1 =
 *              child k (lo x y z, hi x y z as float, child word, 0).  Child
 *              word: -1 empty; < 2^30 wide node; bit 31 set: leaf with first
 *              sorted triangle (bits 3-30) and count - 1 (bits 0-2)
 *   roots      n_meshes int32 root node per mesh
 *   tri_order  n_tris int32: mesh-local triangle id at each sorted position
 * *n_nodes receives the node count. */
pj_status pj_export_bvh(pj_ctx *ctx, pj_dataset ds, int32_t width,
                        int32_t leaf_size, int32_t *nodes, int32_t *roots,
                        int32_t *tri_order, int64_t *n_nodes);

/* Copy per-mesh data computed at load time to host buffers (any may be NULL):
 *   aabb       n_meshes x 6 float (lo x, y, z, hi x, y, z)
 *   lex_first  n_meshes int32: mesh-local id of the lexicographically
 *              smallest vertex
 *   edge_owner n_tris uint8: bit k set if the triangle owns its edge
 *              (v_k, v_(k+1) mod 3) in the unique-edge set */
pj_status pj_export_mesh_data(pj_ctx *ctx, pj_dataset ds, float *aabb,
                              int32_t *lex_first, uint8_t *edge_owner);

#ifdef __cplusplus
}
#endif

#endif /* PIERCE_H */
