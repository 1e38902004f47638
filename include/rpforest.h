/*
 * rpforest.h -- C ABI of the GB300 (sm_103a) rpForests kNN library.
 *
 * Random projection forests kNN search, Yan, Wang, Wang, Wang & Li,
 * "K-nearest Neighbor Search by Random Projection Forests" (arXiv 1812.11689).
 * The library grows T random projection trees on one GPU (Sec. 2,
 * Algorithms 1 and 2), computes exact distances inside every (tree, leaf)
 * block and merges the per-tree candidates into the K nearest neighbours of
 * every point (Algorithm 3).
 *
 * Conventions shared by every entry point:
 *  - Matrices are row-major, contiguous, FP32 (points) / int32 (indices).
 *  - A pointer argument may be device memory or host memory (pageable or
 *    pinned); host buffers are staged through library-owned device memory on
 *    the given stream.  `stream` is a cudaStream_t (NULL = legacy stream).
 *  - Return 0 on success or a negative RPF_E* code.  Nothing is thrown across
 *    the ABI.  On error the output buffers are left in an unspecified state.
 *  - Distances are Euclidean.  Neighbour lists are sorted ascending by the
 *    canonical FP32 squared distance d32(x, y) = fold_k fmaf(x_k - y_k,
 *    x_k - y_k, s) with ties broken by the smaller index; the reported
 *    distance is sqrtf(d32).  Slots without a candidate hold (-1, +inf).
 *  - Every random draw is a pure function of (seed, tree, node key, ...), so
 *    results are deterministic and the first T' trees of a T-tree forest are
 *    exactly the T'-tree forest.
 */
#ifndef RPFOREST_H
#define RPFOREST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RPF_OK 0
#define RPF_EINVAL (-1)    /* bad argument (null pointer, size out of range) */
#define RPF_ENOMEM (-2)    /* a device or host allocation failed */
#define RPF_ECUDA (-3)     /* a CUDA runtime call or kernel failed */
#define RPF_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define RPF_EINTERNAL (-5) /* an internal consistency check failed */

/* Forest handle; owned by the library, read-only after rpf_build. */
typedef struct rpf_forest rpf_forest;

/* Growth and search parameters (Sec. 2 and Sec. 5.2 of the paper). */
typedef struct {
  int32_t n_trees;    /* T >= 1: number of rpTrees (Algorithm 3)                  */
  int32_t leaf_max;   /* L in [1, 1024]: a node with more than L points is split, */
                      /* so no leaf holds more than L (Algorithm 1, n_s = L + 1). */
  int32_t n_try;      /* nTry in [1, 64]: candidate directions per node; the one  */
                      /* with the largest projected dispersion wins (Algorithm 2). */
                      /* 1 = the basic rpTree.                                    */
  int32_t split_rule; /* 0 = c uniform on [min, max] of the projections (Sec. 2);
                         1 = the median (Sec. 2's other usual split point): the
                         floor(m/2) points smallest in (projection, point index)
                         order go left, c = the first right point's projection,
                         so queries go left iff their projection is below c. */
  int32_t form;       /* leaf distances: 0 = plain FP32 SIMT; 1 = BF16 tensor-core */
                      /* Gram (all-kNN) and BF16 rows (queries), each with an     */
                      /* exact FP32 re-rank of a certified shortlist.  Both       */
                      /* return identical lists.                                  */
  int32_t growth;     /* 0 = default (2); 1 = every split decided in FP64 (G-A);  */
                      /* 2 = FP32 projections with a certified error bound and    */
                      /* FP64 recompute of every undecided case (G-B).  1 and 2   */
                      /* grow identical trees.                                    */
  uint64_t seed;      /* seed of every random draw                                */
} rpf_params;

/* Fill `p` with defaults: T=10, L=50, nTry=5, uniform split, plain form,
   growth 0, seed 0. */
void rpf_default_params(rpf_params* p);

/*
 * rpf_build -- grow the forest (Sec. 2, Algorithm 1 per tree, Algorithm 2 per
 * node; Algorithm 3, first loop).
 *   X      : n x d points (device or host).  The library copies X; the caller
 *            may free it when the call returns.
 *   n, d   : 1 <= n, 1 <= d <= 4096, n * n_trees < 2^31.
 *   p      : parameters (copied).
 *   stream : stream for all work; the call synchronises it before returning.
 *   out    : receives the new forest; release with rpf_free.
 * Errors: RPF_EINVAL (null pointer, sizes or parameters out of range),
 * RPF_ENOMEM, RPF_ECUDA.
 */
int rpf_build(const float* X, int64_t n, int32_t d, const rpf_params* p, void* stream,
              rpf_forest** out);

/*
 * rpf_build_shard -- rpf_build for trees tree_first .. tree_first + n_trees - 1
 * of the ensemble.  Every random draw of tree t is keyed by its global index
 * t, so these are exactly the trees a forest of tree_first + n_trees trees
 * holds at those indexes: the trees of Algorithm 3 are independent (Sec. 2,
 * Sec. 5.3), and a forest can be split by tree across processes or GPUs
 * whose per-point lists are then merged (rpf_all_knn_keys, rpf_merge_keys).
 *   tree_first : >= 0, tree_first + n_trees <= 2^20.
 * Other arguments and errors as rpf_build.
 */
int rpf_build_shard(const float* X, int64_t n, int32_t d, const rpf_params* p,
                    int32_t tree_first, void* stream, rpf_forest** out);

/*
 * rpf_all_knn -- K nearest neighbours of every data point among the union of
 * its T leaves, the point itself excluded (Algorithm 3 with Q = U).
 *   K        : 1 <= K <= 128.
 *   idx,dist : n x K outputs (device or host), sorted as described above.
 *   workspace: device scratch of at least rpf_workspace_bytes(f, 0, K, 1)
 *              bytes, or NULL to let the library allocate (stream-ordered).
 *   stream   : work is enqueued on it; the call synchronises it before
 *              returning (host outputs are complete on return).
 * Errors: RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA, RPF_ETIMEOUT (a bounded device
 * wait of this call gave up; the lists are then unspecified).
 */
int rpf_all_knn(rpf_forest* f, int32_t K, int32_t* idx, float* dist, void* workspace,
                size_t ws_bytes, void* stream);

/*
 * rpf_all_knn_trees -- rpf_all_knn over the first n_trees trees only.  Every
 * random draw is keyed by the tree index, so the first T' trees of a forest
 * are exactly the forest that rpf_build grows with T' trees (a nested
 * ensemble): one forest answers the whole sweep over T of the accuracy
 * experiments (Sec. 5.2).  1 <= n_trees <= the forest's trees; the other
 * arguments, the outputs and the errors are those of rpf_all_knn.
 */
int rpf_all_knn_trees(rpf_forest* f, int32_t n_trees, int32_t K, int32_t* idx, float* dist,
                      void* workspace, size_t ws_bytes, void* stream);

/*
 * rpf_all_knn_async -- the lists of rpf_all_knn (Algorithm 3 with Q = U),
 * only enqueued on `stream`: the call allocates nothing, does not
 * synchronise and reads no device memory on the host, so the sequence (a
 * persistent launch over every (tree, leaf) tile per group of trees, then
 * the cross-tree merge) can be recorded into a CUDA graph and replayed.
 *   K        : 1 <= K <= 128.
 *   idx,dist : n x K outputs in DEVICE memory.
 *   workspace: DEVICE scratch of at least rpf_workspace_bytes(f, 0, K, 1)
 *              bytes, owned by the caller; its first word receives the
 *              outcome of the device work.
 * Once the work is done, rpf_query_status(workspace, stream) returns
 * RPF_OK, or RPF_ETIMEOUT if a bounded device wait gave up (the lists are
 * then unspecified).  Calls on one forest share its error word: issue them
 * on one stream.  Errors at enqueue: RPF_EINVAL (host pointer, small
 * workspace), RPF_ECUDA.
 */
int rpf_all_knn_async(rpf_forest* f, int32_t K, int32_t* idx, float* dist, void* workspace,
                      size_t ws_bytes, void* stream);

/*
 * rpf_all_knn_keys -- the lists of rpf_all_knn with the ranking key itself:
 * for every point, its K nearest in the union of its leaves over this
 * forest's trees, as n x K pairs of int32 (bits of the FP32 squared distance
 * d32, index), ascending by (d32, index), empty slots (+inf bits, -1).  These
 * are the lists a group of trees contributes to the union over a larger
 * forest (Algorithm 3): merging the groups' lists per point with
 * rpf_merge_keys gives exactly the larger forest's lists, because a point in
 * the K nearest of the whole union is in the K nearest of every group's
 * union that contains it.
 *   keys      : n x K x 2 int32 (device or host).
 *   workspace : as rpf_all_knn.  Synchronises `stream`.
 * Errors: as rpf_all_knn.
 */
int rpf_all_knn_keys(rpf_forest* f, int32_t K, int32_t* keys, void* workspace, size_t ws_bytes,
                     void* stream);

/*
 * rpf_merge_keys -- merge n_lists key lists per point (rpf_all_knn_keys
 * layout, list-major: lists[(g * n + i) * K + k] is pair k of point i in list
 * g) into the final lists: the K smallest distinct (d32, index) pairs, as
 * indices and Euclidean distances sqrtf(d32), padded with (-1, +inf).
 *   n >= 0, 1 <= K <= 128, n_lists >= 1; pointers device or host.
 * Errors: RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA.
 */
int rpf_merge_keys(int64_t n, int32_t K, int32_t n_lists, const int32_t* lists, int32_t* idx,
                   float* dist, void* stream);

/*
 * rpf_query -- K nearest neighbours of m new points Q among the data, found
 * in the union of the leaves each query falls into (Algorithm 3: each query is
 * dropped through every tree).  Nothing is excluded.  Safe to call concurrently on one
 * forest from several host threads with different streams and workspaces.
 *   Q        : m x d queries (device or host); m >= 0 (m = 0 is a no-op).
 *   K        : 1 <= K <= 128.
 *   idx,dist : m x K outputs (device or host).
 *   workspace: device scratch of rpf_workspace_bytes(f, m, K, 0) bytes, or
 *              NULL to let the library allocate (stream-ordered).
 * Synchronisation: with host outputs, or with workspace NULL, the call
 * synchronises `stream` and its return code covers the device work.  With a
 * caller workspace and device outputs it only enqueues the work; a bounded
 * device wait that gave up is then reported by rpf_query_status(workspace,
 * stream) once the work is done.
 * Errors: RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA, RPF_ETIMEOUT (see above; the
 * lists are then unspecified but every slot is written).
 */
int rpf_query(const rpf_forest* f, const float* Q, int64_t m, int32_t K, int32_t* idx,
              float* dist, void* workspace, size_t ws_bytes, void* stream);

/* Allocation-free query.  The paper has no counterpart to this entry point:
 * it answers the same query as rpf_query, with the same kernels and the same
 * results bit for bit, for callers that must not allocate device memory
 * while they run -- e.g. a serving process whose free HBM is already handed
 * to its own pool, or a latency-critical thread that cannot take the
 * synchronisation a device allocation may imply.  It calls no cudaMalloc,
 * cudaFree or other allocating routine (with launch tracing off, the
 * default).
 *   Q        : m x d queries in DEVICE memory, row-major FP32; m >= 0.
 *   K        : 1 <= K <= 128.
 *   idx,dist : m x K outputs in DEVICE memory, owned by the caller.
 *   stream   : cudaStream_t (NULL = legacy default stream).
 * Scratch: one fixed array of RPF_STATIC_SCRATCH_BYTES per device, inside
 * the library.  A call needs 256 + align256(8 m T) + align256(8 T m K) bytes
 * of it (T = trees of the forest; at T = 32, K = 10 that allows m <= 2978);
 * larger requests return RPF_EINVAL without launching anything -- split
 * them.  Nothing in the scratch has to start at zero: the call clears its
 * error word and every other byte it reads was written earlier in the call.
 * Set-up: the first call on a device (that device current, the forest's
 * device) looks the array up once (cudaGetSymbolAddress) and caches its
 * address.  The cached address does not survive a device reset
 * (cudaDeviceReset).
 * Races: the scratch is shared by every call on the device.  Calls that may
 * overlap in time (different streams, different host threads) race on it and
 * corrupt each other's results: issue them on one stream, or serialise them.
 * The call only enqueues work; rpf_query_status(NULL, stream) reports a
 * bounded device wait of the last call that gave up (RPF_ETIMEOUT).
 * Errors: RPF_EINVAL (bad argument, host pointer, wrong current device,
 * request larger than the scratch), RPF_ECUDA. */
#define RPF_STATIC_SCRATCH_BYTES (8 << 20)
int rpf_query_static(const rpf_forest* f, const float* Q, int64_t m, int32_t K, int32_t* idx,
                     float* dist, void* stream);

/*
 * rpf_query_status -- outcome of the device work of the last rpf_query or
 * rpf_all_knn_async that used `workspace` (or, with workspace NULL, of the
 * last rpf_query_static on the current device): synchronises `stream` (the
 * stream that call ran on), then returns RPF_OK, or RPF_ETIMEOUT if one of
 * its bounded device waits gave up.  Errors: RPF_EINVAL (host pointer),
 * RPF_ECUDA.
 */
int rpf_query_status(const void* workspace, void* stream);

/* Scratch bytes rpf_all_knn / rpf_all_knn_async (for_all_knn = 1, m ignored)
 * or rpf_query needs. */
size_t rpf_workspace_bytes(const rpf_forest* f, int64_t m, int32_t K, int32_t for_all_knn);

/*
 * rpf_autotune -- pick the leaf-tile configuration by timing every candidate
 * on this forest's own tiles (its first trees) with K neighbours; all
 * candidates give identical lists.
 *   plain form  : the tile region R (leaves of a tree starting in one region
 *                 of R positions form a tile; multiples of 32).
 *   chosen form : tile rows (128 or 256, where the leaf bound allows both),
 *                 Gram coordinates per tensor-core chunk, CTAs per SM, and
 *                 the query leaf scan (BF16 rows with the certified re-rank,
 *                 or FP32 rows), timed with the first data points as
 *                 queries; untuned, the chosen form scans BF16 rows.
 * The tile shape is kept for the rest of the process for forests of the same
 * dimension and leaf bound (later builds use it) and this forest's tiles are
 * rebuilt with it; the launch choice is kept per (dimension, tile rows, K
 * bucket).  A chosen-form forest the tensor-core kernel does not cover has
 * nothing to tune (chosen all 0).
 *   chosen : NULL or int32[5] receiving {Gram chunk, CTAs per SM, tile rows,
 *            tile region R, query scan (1 = BF16, 0 = FP32, -1 = not
 *            tuned)} (0 where not tuned).
 * Allocates a scratch list for the first trees; synchronises `stream`; no
 * other call may use the forest meanwhile.
 * Errors: RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA.
 */
int rpf_autotune(rpf_forest* f, int32_t K, void* stream, int32_t* chosen);

/*
 * rpf_add_trees -- grow n_new more trees onto a built forest (an incremental
 * ensemble: Sec. 5.2 studies accuracy as trees are added).  Every random
 * draw is keyed by the tree's index, so the result is exactly the forest
 * rpf_build would grow with T + n_new trees: trees 0..T-1 are untouched and
 * trees T..T+n_new-1 are the ones that build would grow.  The forest's
 * tables are reallocated (stream-ordered on `stream`); no other call may use
 * the forest meanwhile.  Synchronises `stream` before returning.
 * Errors: RPF_EINVAL (n_new < 1, or (T + n_new) n >= 2^31), RPF_ENOMEM,
 * RPF_ECUDA; on an error the forest keeps its first T trees.
 */
int rpf_add_trees(rpf_forest* f, int32_t n_new, void* stream);

/*
 * rpf_set_form -- switch the leaf-distance form of a built forest: 0 = plain
 * FP32, 1 = the chosen form (BF16 tensor-core tiles for all-kNN, BF16 rows
 * for queries, each with a certified exact FP32 re-rank).  Both give the same
 * lists bit for bit; switching to 1 builds the tile packing and the BF16
 * copy of the data if the forest has none.  No other call may use the forest
 * meanwhile; synchronises `stream`.
 * Errors: RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA.
 */
int rpf_set_form(rpf_forest* f, int32_t form, void* stream);

/*
 * rpf_set_query_scan -- which leaf scan rpf_query and rpf_query_static use
 * in the chosen form: -1 = the one rpf_autotune found faster for the
 * forest's (d, leaf bound, K) shape, or BF16 rows where it has not been run
 * (the default); 0 = FP32 rows; 1 = BF16 rows with the certified exact
 * re-rank (where K > 32 or the leaf bound exceeds 128 the FP32 scan runs).
 * All give the same lists bit for bit.  Takes effect on later calls; no
 * device work.  Errors: RPF_EINVAL.
 */
int rpf_set_query_scan(rpf_forest* f, int32_t mode);

/* Release the forest and its device memory.  NULL is a no-op. */
void rpf_free(rpf_forest* f);

/* Static English description of an RPF_E* code. */
const char* rpf_error_string(int code);

/*
 * rpf_brute_knn -- exact kNN by brute force under the same (d32, index) order:
 * for each of the m rows of Q, the K nearest of the n rows of X, skipping
 * index self[i] for row i when self is not NULL (all-kNN ground truth).  This
 * is the ground truth of the missing rate and kNN-distance metrics of Sec. 5.1.
 *   X (n x d), Q (m x d), self (m), idx / dist (m x K): device or host.
 * Errors: RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA.
 */
int rpf_brute_knn(const float* X, int64_t n, int32_t d, const float* Q, int64_t m,
                  const int32_t* self, int32_t K, int32_t* idx, float* dist, void* stream);

/* ---- failure detection --------------------------------------------------- */

/* Time limit of every bounded device wait (the waits on bulk copies and on
   tensor-core commits), in nanoseconds of the GPU's global timer; 0 restores
   the default of 2 s.  A wait that reaches it records RPF_ETIMEOUT, waits
   once more (bounded) for work in flight, frees what it holds and returns,
   so the CUDA context stays usable.  Applies to launches made afterwards. */
void rpf_set_wait_limit(uint64_t limit_ns);

/* Check of the timeout path: one CTA waits, with the given limit, on a
   barrier that nothing completes (no thread arrives on it, no copy is posted
   to it, so nothing is in flight).  Returns RPF_ETIMEOUT when the wait gave
   up as it must, RPF_OK if it ended otherwise, or RPF_ENOMEM / RPF_ECUDA.
   Synchronises `stream`. */
int rpf_wait_selftest(uint64_t limit_ns, void* stream);

/* Allocation-failure injection for tests of the error paths: after `after`
   more device allocations by the library succeed, the next one fails as if
   the device were out of memory (the call in progress returns RPF_ENOMEM);
   later allocations succeed again.  -1 switches it off. */
void rpf_debug_fail_alloc(int64_t after);

/* ---- tracing ---------------------------------------------------------------- */

/* Turn per-kernel timing on (1) or off (0).  When on, every kernel launch of
   the library is bracketed by a CUDA event pair on its launching stream. */
int rpf_trace_enable(int on);

/* Kernels launched by the library since it was loaded (always counted). */
int64_t rpf_launch_count(void);

/* Per-kernel totals of the events recorded since the last read (waits for
   them): up to max_names entries of name (48 bytes each, NUL-terminated),
   timed launches and total milliseconds; n_names receives the number of
   kernel names known.  Clears the recorded events. */
int rpf_trace_read(int32_t max_names, char* names, int64_t* launches, double* ms,
                   int32_t* n_names);

/*
 * rpf_gather_probe -- the row-gather reference of the growth kernels:
 * gathers `rows` rows of X (n x d FP32, device, 16-byte aligned, d a
 * multiple of 4) in a fixed pseudo-random order (seeded by `seed`), d / 4
 * lanes per row (at most 32) reading each row as one coalesced read, and
 * keeps nothing of them (`out`, one device float, is never written in
 * practice).  Only enqueues the kernel on `stream`; the caller times it.
 * rows * d * 4 bytes over the elapsed time is the rate of random whole-row
 * reads that the growth kernels' own row gathers are compared with.
 * Errors: RPF_EINVAL, RPF_ECUDA.
 */
int rpf_gather_probe(const float* X, int64_t n, int32_t d, int64_t rows, int64_t seed, float* out,
                     void* stream);

/* ---- inspection (host outputs; used by tests and tools) ------------------ */

/* Sizes: n, d, T, total node count, leaf count, max depth, and the number of
   nodes whose split needed the FP64 fallback under growth 2.  Any pointer may
   be NULL. */
int rpf_forest_info(const rpf_forest* f, int64_t* n, int32_t* d, int32_t* n_trees,
                    int64_t* n_nodes, int64_t* n_leaves, int32_t* max_depth,
                    int64_t* n_exact_nodes);

/* Counters (host, first n_out of): [0] nodes decided by the FP64 fallback,
   [1] rows the BF16 form rescanned exactly because its certificate failed
   (cumulative over rpf_all_knn calls), [2] level-synchronous growth levels,
   [3] leaf-tile region R, [4] tree groups of rpf_all_knn calls on a
   chosen-form forest that ran the plain form instead (leaf bound above 256,
   K above 32, or rows too wide for the tensor-core tile; cumulative). */
int rpf_forest_counters(const rpf_forest* f, int64_t* out, int32_t n_out);

/* Final permutation of tree t (n int32, host): every leaf is a contiguous
   segment, members in ascending original index. */
int rpf_forest_perm(const rpf_forest* f, int32_t t, int32_t* perm_host);

/* Leaf table (host, n_leaves entries each): tree, begin (offset in the tree's
   permutation), len. */
int rpf_forest_leaves(const rpf_forest* f, int32_t* tree, int32_t* begin, int32_t* len);

/* Node table (host, n_nodes entries each): key (node key of the counter-based
   draws; root 1), tree, begin, len, left child, right child (-1 for leaves),
   chosen try (-1 if none), flags (bit 0: rank split; bit 1: the split was
   decided by the FP64 fallback), split point c. */
int rpf_forest_nodes(const rpf_forest* f, uint64_t* key, int32_t* tree, int32_t* begin,
                     int32_t* len, int32_t* left, int32_t* right, int32_t* jstar,
                     int32_t* flag, double* c);

/* The candidate directions of Algorithm 2 for (tree t, node key, try j),
   d doubles each, for n_keys keys: out[i*d + k].  Device or host output. */
int rpf_directions(uint64_t seed, int32_t t, const uint64_t* keys_host, int32_t n_keys,
                   int32_t j, int32_t d, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RPFOREST_H */
