/*
 * abx.h -- C ABI of the B300 ABX distance / score engine (libabx.so).
 *
 * Implements the hot path of fastabx (arXiv 2505.02692):
 *   features -> angular frame distances -> DTW normalised by path length
 *   (or mean pooling) -> per-cell triplet counts -> collapse to an ABX error.
 *
 * Conventions
 *   - Every call returns ABX_OK (0) or a negative ABX_E_* code; the message
 *     of the last failure on the calling thread is abx_last_error().  No C++
 *     exception crosses this boundary.
 *   - Sizes and offsets are int64_t, label codes int32_t (dense codes >= 0).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls that say "asynchronous" only enqueue work.
 *   - Objects returned through `out` pointers are owned by the caller and
 *     released with the matching *_free call.  Free calls accept NULL.
 *   - One GPU per context; a context is not safe to use from two host
 *     threads at once.
 *   - Item lengths are 1..128 frames; longer items are rejected with
 *     ABX_E_UNSUPPORTED.
 */
#ifndef ABX_H
#define ABX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define ABX_OK 0
#define ABX_E_INVALID (-1)     /* bad argument (NULL pointer, bad size, bad attribute) */
#define ABX_E_ZERO_NORM (-2)   /* a frame with zero L2 norm: its angle is undefined   */
#define ABX_E_OOM (-3)         /* device or pinned host allocation failed             */
#define ABX_E_CUDA (-4)        /* a CUDA runtime call failed                          */
#define ABX_E_UNSUPPORTED (-5) /* valid input outside this build's limits             */
#define ABX_E_STATE (-6)       /* objects from different contexts / wrong order       */
#define ABX_E_CANCELLED (-7)   /* a served job cancelled before it ran                 */

/* Feature storage precision used by the distance kernel.
 *   ABX_FP32_SIMT  FP32 features, FP32 FFMA dot products (CUDA cores).
 *   ABX_FP32       FP32 features, dot products on tcgen05 tensor cores from a
 *                  two-term FP16 split of each (power-of-two scaled) frame,
 *                  v = hi + lo, with FP32 accumulation of hi*hi + hi*lo +
 *                  lo*hi: the stored value carries 22 significant bits and
 *                  the dropped lo*lo term is at most 2^-22 |u||v|.
 *   ABX_BF16       features stored in BF16, tcgen05, FP32 accumulation.
 *   ABX_FP8        features stored in FP8 E4M3 with one scale per item,
 *                  tcgen05, FP32 accumulation.
 * Every precision reports, per item pair, an interval that provably holds the
 * exact distance (see abx_score's recheck). */
#define ABX_FP32_SIMT 0
#define ABX_FP32 1
#define ABX_BF16 2
#define ABX_FP8 3

/* Item distance mode (Sec. 3.2: align with DTW or pool along time). */
#define ABX_DTW 0   /* DTW over angular frame distances, / optimal path length */
#define ABX_MEAN 1  /* angular distance of the mean frames                     */

/* Frame distance (Sec. 3.1: Score takes "angular", "euclidean", etc.). */
#define ABX_DIST_ANGULAR 0   /* arccos(cos) / pi, in [0, 1]                        */
#define ABX_DIST_COSINE 1    /* 1 - cos, in [0, 2]                                 */
#define ABX_DIST_EUCLIDEAN 2 /* |u - v| of the raw frames (from norms and the Gram) */
#define ABX_DIST_KL 3        /* symmetrised Kullback-Leibler divergence of frames
                                read as distributions: (KL(p|q) + KL(q|p)) / 2,
                                p = u / sum(u); components must be > 0        */

/* Where abx_load_items finds the feature matrix. */
#define ABX_MEM_HOST 0          /* host memory; copied to the device             */
#define ABX_MEM_DEVICE_COPY 1   /* device memory; copied into a library buffer    */
#define ABX_MEM_DEVICE_BORROW 2 /* device memory; used in place, caller keeps it
                                   alive and unchanged until abx_items_free       */

typedef struct abx_ctx abx_ctx;
typedef struct abx_items abx_items;
typedef struct abx_cells abx_cells;
typedef struct abx_dist abx_dist;

/* Summary of a task built by abx_build_cells (host-side numbers). */
typedef struct abx_cells_info {
    int64_t n_items;     /* items taking part (all items)                       */
    int64_t n_groups;    /* distinct values of the `by` attributes              */
    int64_t n_blocks;    /* non-empty (group, on, across) item sets             */
    int64_t n_cells;     /* cells with at least one triple                      */
    int64_t n_triplets;  /* sum over cells of |C| (a == x excluded)             */
    int64_t max_group;   /* items in the largest group                          */
} abx_cells_info;

/* Summary of an abx_distances result. */
typedef struct abx_dist_info {
    int64_t n_pairs;       /* unordered item pairs whose distance a triple needs */
    int64_t n_frame_pairs; /* sum over those pairs of Tx * Ty                     */
    int64_t n_tiles;       /* 128 x 128 frame tiles computed                      */
    int64_t n_frames;      /* frames packed for the task                          */
    int32_t mode, precision;
    int32_t distance, reserved;
} abx_dist_info;

/* Counters filled by abx_score. */
typedef struct abx_score_stats {
    int64_t n_cells;          /* cells scored                                       */
    int64_t n_triplets;       /* triples scored                                     */
    int64_t n_undecided;      /* triples whose distance intervals overlapped        */
    int64_t n_recheck_pairs;  /* item pairs of undecided triples, recomputed (recheck
                                 on): with the interval rule in DTW mode first in
                                 TF32 with an interval, otherwise in FP64          */
    int64_t n_flips;          /* undecided triples whose low-precision decision
                                 differed from the exact one (recheck on)           */
    int64_t num2_total;       /* sum over cells of N = 2*wins + ties                */
    int64_t count2_total;     /* sum over cells of 2|C|                             */
    int64_t n_exact_pairs;    /* item pairs recomputed in FP64: those of the triples
                                 the TF32 intervals did not separate (interval rule,
                                 DTW), otherwise all n_recheck_pairs                */
} abx_score_stats;

/* Message of the last failing call on this host thread ("" if none). */
const char *abx_last_error(void);

/* Library version string. */
const char *abx_version(void);

/* Create a context on CUDA device `device`.  Fails with ABX_E_CUDA if the
 * device is absent or is not an sm_103 GPU.  The context keeps up to two
 * device scratch buffers for abx_distances' frame-distance tiles (each the
 * next power of two of a call's need, at most 8 GiB), allocated on first use
 * and reused by later calls in stream order; they are freed when the context
 * and every object made from it are freed. */
int abx_ctx_create(int device, abx_ctx **out);
int abx_ctx_destroy(abx_ctx *ctx);

/*
 * abx_load_items -- register a feature matrix and its item labels
 * (Sec. 3.1 Dataset: labels plus access to the representations).
 *
 *   feats         n_frames x dim FP32, row-major, items stored back to back;
 *                 host or device memory according to `mem`.
 *   item_offsets  host, n_items + 1 int64 CSR offsets into the frames:
 *                 item i owns rows [item_offsets[i], item_offsets[i+1]);
 *                 item_offsets[0] == 0, strictly increasing (no empty item),
 *                 item_offsets[n_items] == n_frames.
 *   labels        host, n_items x n_attr int32, row-major, codes >= 0.
 *   stream        stream for the copies; the items' device data and every
 *                 object derived from them live on this stream (they are
 *                 freed stream-ordered on it).  A host `feats` buffer must stay
 *                 unchanged until the stream has passed this call (the copy
 *                 is asynchronous for pinned host memory).
 * The library copies offsets and labels; feats is copied unless
 * ABX_MEM_DEVICE_BORROW.  Zero-norm frames are detected by abx_distances.
 */
int abx_load_items(abx_ctx *ctx, const float *feats, int64_t n_frames, int32_t dim,
                   const int64_t *item_offsets, int64_t n_items, const int32_t *labels,
                   int32_t n_attr, int32_t mem, void *stream, abx_items **out);
int abx_items_free(abx_items *items);

/*
 * abx_build_cells -- build an ABX task (Sec. 2; Sec. 3.1 Task).
 *
 * A triple (a, b, x) is valid when attribute `on_attr` is equal for a and x
 * and different for b, every attribute of `by` is equal for a, b and x, and
 * `across_attr` (or -1 for none) is equal for a and b and different for x;
 * a != x.  A cell is the set of valid triples sharing (on of a/x, on of b,
 * by values, across of a/b, across of x).
 *   by           host array of n_by distinct attribute indices (n_by may be 0).
 *   across_attr  attribute index or -1; at most one across attribute.
 * Host-side: groups items by the `by` values, sorts each group by
 * (across, on), and counts cells and triples.  Limits: the product of the
 * by-attribute code ranges <= 2^26, groups x on-codes x across-codes <= 2^28.
 */
int abx_build_cells(abx_ctx *ctx, const abx_items *items, int32_t on_attr, const int32_t *by,
                    int32_t n_by, int32_t across_attr, abx_cells **out);
int abx_cells_get_info(const abx_cells *cells, abx_cells_info *info);

/*
 * abx_cells_set_subsampler -- the two subsampling methods of the Subsampler
 * (Sec. 3.1, after Libri-Light), applied by abx_score / abx_score_ex /
 * abx_score_cells to this task:
 *   max_size_group  each of A, B and X of a cell keeps at most this many
 *                   items (0 = all; at most 256);
 *   max_x_across    across tasks: of the cells sharing (by values, on_ax,
 *                   on_b, across_ab), at most this many across_x values are
 *                   kept (0 = all).
 * The draw is seeded and order-free: with h = SplitMix64 hash of (seed,
 * role 0/1/2 for A/B/X, by values, on_ax, on_b, across_ab, across_x), a role
 * keeps the items i (rows of the labels) with the smallest
 * splitmix64(h xor i), ties by i; the across_x values kept are those with the
 * smallest splitmix64(h3 xor v), h3 the hash of (seed, 3, by values, on_ax,
 * on_b, across_ab).  A cell left without a triple drops out.  Distances are
 * still computed for every pair the full task needs; abx_cells_get_info
 * counts the task without subsampling.  Requires level-1 collapse
 * attributes among the by attributes (ABX_E_UNSUPPORTED otherwise).
 */
int abx_cells_set_subsampler(abx_cells *cells, int32_t max_size_group, int32_t max_x_across,
                             uint64_t seed);
int abx_cells_free(abx_cells *cells);

/*
 * abx_distances -- every item-pair distance that some triple of the task
 * compares (Sec. 3.2).  Fully asynchronous on `stream` (it first waits for
 * the task's upload); counts in abx_dist_info become available after a
 * synchronising call.
 *
 *   mode       ABX_DTW: frame distances d(i,j) = arccos(cos)/pi, DTW with
 *              steps (i-1,j), (i,j-1), (i-1,j-1), result = optimal cost /
 *              cells on the optimal path (shorter path on equal cost).
 *              ABX_MEAN: angular distance of the mean raw frames.
 *   precision  ABX_FP32_SIMT, ABX_FP32, ABX_BF16 or ABX_FP8 (see above).
 * The result stays on the device; read it with abx_dist_lookup or score it
 * with abx_score.  ABX_E_ZERO_NORM is reported by the first synchronising
 * call (abx_dist_lookup, abx_score, abx_dist_sync).
 */
int abx_distances(abx_ctx *ctx, const abx_items *items, const abx_cells *cells, int32_t mode,
                  int32_t precision, void *stream, abx_dist **out);
/*
 * abx_distances_ex -- abx_distances with a choice of frame distance
 * (ABX_DIST_*).  Intervals holding the exact distance, and therefore the
 * FP64 recheck of abx_score, exist for ABX_DIST_ANGULAR only (lo = hi = the
 * distance otherwise; abx_score with recheck != 0 then fails with
 * ABX_E_UNSUPPORTED).  ABX_DIST_EUCLIDEAN stores the raw frames in the
 * storage precision (FP8: one scale per item) and takes
 * sqrt(|u|^2 + |v|^2 - 2 <u,v>) from the tile's dot products.  ABX_DIST_KL
 * (precision ABX_FP32 only, else ABX_E_UNSUPPORTED) divides each frame by
 * the sum of its components and stores [p | ln p]; one tile contraction over
 * both halves, A = [p | ln p] against B = [ln p | p], gives
 * <p_i, ln p_j> + <ln p_i, p_j>, and the distance is
 * (h_i + h_j - that) / 2 with h = sum p ln p.  A frame with a component
 * <= 0 makes the deferred error ABX_E_INVALID.
 */
int abx_distances_ex(abx_ctx *ctx, const abx_items *items, const abx_cells *cells,
                     int32_t mode, int32_t distance, int32_t precision, void *stream,
                     abx_dist **out);
/* Summary of the result; waits for the distance work (counts are produced on
 * the device). */
int abx_dist_get_info(abx_dist *dist, abx_dist_info *info);
/* Wait for the distance work and report a deferred error (e.g. zero norm). */
int abx_dist_sync(abx_dist *dist);
/*
 * Read distances of n item pairs (x[k], y[k]), original item indices, host
 * arrays.  Writes the distance, the interval [lo, hi] known to hold the exact
 * value, and the optimal path length (1 in MEAN mode).  Pairs never computed
 * (not needed by the task, or x == y) get NaN and length 0.  Synchronises.
 * Any of d, lo, hi, len may be NULL.
 */
int abx_dist_lookup(abx_dist *dist, int64_t n, const int64_t *x, const int64_t *y, float *d,
                    float *lo, float *hi, int32_t *len);
int abx_dist_free(abx_dist *dist);

/*
 * abx_refine_pairs -- the refined stage of the recheck for chosen pairs: the
 * DTW distance of each item pair (x[k], y[k]) (original item indices, host
 * arrays, n < 2^31) recomputed from the FP32 features with TF32 tensor-core
 * products, as an interval [lo[k], hi[k]] (host outputs) that holds the
 * exact distance (angular frame distance, fastabx Sec. 3.1; DTW normalised
 * by the optimal path's length, Sec. 3.2).  The interval accounts for the
 * TF32 rounding of every feature (the largest angle between a frame and its
 * rounding, per item) and for the FP32 accumulation; pairs of nearly
 * parallel frames (|cos| > 0.999) get [0, 1].  Runs on `stream` and
 * synchronises it.  ABX_E_INVALID for an index out of range.
 */
int abx_refine_pairs(abx_ctx *ctx, const abx_items *items, int64_t n, const int64_t *x,
                     const int64_t *y, float *lo, float *hi, void *stream);

/*
 * abx_score -- cell scores and the collapsed ABX error (Sec. 2).
 *
 * Per cell, N = sum over triples of 2*1[d(x,a) < d(x,b)] + 1[d(x,a) = d(x,b)]
 * (exact integers), D_C = N / (2|C|).
 *   levels    host int32 tokens: attribute indices, -1 between levels, e.g.
 *             {ctx, -1, spk} averages over contexts, then speakers; an across
 *             attribute stands for the pair (across_ab, across_x).  Within a
 *             level, sums run in increasing order of the level's attribute
 *             codes (lexicographic in the listed order); after the last level
 *             the remaining entries are averaged in increasing order of
 *             (on_ax, on_b, remaining by attributes in `by` order, across pair).
 *   weighted  1: error = 1 - sum N / sum 2|C| (cell-size weighting); levels
 *             are then ignored.
 *   recheck   1: triples whose two distance intervals overlap are decided
 *             from recomputed distances, which makes every decision equal to
 *             the exact one.  DTW: both pairs are first recomputed from the
 *             FP32 features (TF32 tensor cores) with a proven interval; the
 *             triples these intervals still do not separate are decided by
 *             FP64 values (the only FP64 step).  Mean mode: FP64 directly.
 *             0: decisions use the stored distances as they are.
 * Writes 1 - D to *error_out (NaN when the task has no cell) and, if stats is
 * not NULL, the counters.  Synchronises `stream`.
 */
int abx_score(abx_ctx *ctx, abx_dist *dist, const abx_cells *cells, const int32_t *levels,
              int32_t n_level_tokens, int32_t weighted, int32_t recheck, void *stream,
              double *error_out, abx_score_stats *stats);

/*
 * abx_score_ex -- abx_score with a choice of recheck rule.
 *   recheck_mode  ABX_RECHECK_OFF       decisions from the stored distances;
 *                 ABX_RECHECK_INTERVAL  triples whose intervals overlap are
 *                                       re-decided exactly (= abx_score with
 *                                       recheck = 1; provably exact);
 *                 ABX_RECHECK_MARGIN    triples whose distance margin
 *                                       |d(x,a) - d(x,b)| is below `margin`
 *                                       are re-decided by recomputing both
 *                                       distances in FP64; exact when
 *                                       every stored distance is within
 *                                       margin / 2 of its exact value (a
 *                                       stated bound, checked empirically).
 * Both recheck modes need ABX_DIST_ANGULAR.
 */
#define ABX_RECHECK_OFF 0
#define ABX_RECHECK_INTERVAL 1
#define ABX_RECHECK_MARGIN 2
int abx_score_ex(abx_ctx *ctx, abx_dist *dist, const abx_cells *cells, const int32_t *levels,
                 int32_t n_level_tokens, int32_t weighted, int32_t recheck_mode, float margin,
                 void *stream, double *error_out, abx_score_stats *stats);

/*
 * abx_score_submit / abx_score_wait -- abx_score_ex in two halves, so that
 * the scoring of several tasks can be enqueued before any of them is waited
 * for (the host then plans the next task while the GPU scores this one).
 *
 * abx_score_submit takes the arguments of abx_score_ex (less the outputs),
 * enqueues the whole scoring on `stream` without synchronising, and returns
 * a job handle in *out.  abx_score_wait blocks until that work is done,
 * writes *error_out and *stats exactly as abx_score_ex would (both may be
 * NULL), reports the deferred errors of the distances (ABX_E_ZERO_NORM, ...)
 * and frees the job, whatever it returns.  Every submitted job must be
 * waited for once.  Until then `dist` and `cells` must stay alive:
 * abx_dist_free and abx_cells_free fail with ABX_E_STATE while a job on
 * them is outstanding.  Results are identical to abx_score_ex.
 */
typedef struct abx_score_job abx_score_job;
int abx_score_submit(abx_ctx *ctx, abx_dist *dist, const abx_cells *cells,
                     const int32_t *levels, int32_t n_level_tokens, int32_t weighted,
                     int32_t recheck_mode, float margin, void *stream, abx_score_job **out);
int abx_score_wait(abx_score_job *job, double *error_out, abx_score_stats *stats);

/*
 * Batched tasks (many independent ABX tasks in shared launches).
 *
 * abx_batch_create takes n_tasks tasks, each its own features, items and
 * labels, all scored with the same on / by / across attributes, mode,
 * precision, collapse levels and recheck rule.  Tasks of equal dimension are
 * joined into one task with a leading task attribute (so that no cell mixes
 * two tasks), and every stage of the path (packing, pair planning, the frame
 * tile kernel, DTW, scoring) runs as one launch per dimension class instead of
 * one per task.  Each task's result is identical to what abx_distances +
 * abx_score give for that task alone.  All buffers are sized at creation, so
 * a run enqueues no host work: the first abx_batch_run captures the whole run
 * into a CUDA graph, later runs replay it (ABX_BATCH_GRAPH=0 disables the
 * graph).  With tune != 0 the kernel variants of each dimension class (tile
 * kernel ring depth, DTW threads and window) are timed once on the batch
 * itself and the fastest kept (tile kernel: ring depth, and one or two tiles
 * of a panel row per work item with 8 or 16 epilogue warps; DTW: threads and
 * window); results are cached in the context per
 * (precision, mode, padded dimension, longest item).
 *
 *   tasks[k].feats       n_frames x dim FP32, row-major; host memory
 *                        (mem = ABX_MEM_HOST) or device memory
 *                        (ABX_MEM_DEVICE_COPY); copied at creation
 *   tasks[k].item_offsets, labels   host arrays as in abx_load_items; every
 *                        task has the same n_attr
 *   levels               collapse levels as in abx_score (attribute ids of the
 *                        tasks; the task attribute is never collapsed)
 * Errors: ABX_E_INVALID (bad arguments), ABX_E_UNSUPPORTED (level-1
 * attributes that are not by attributes), ABX_E_OOM, ABX_E_CUDA.
 * abx_batch_wait synchronises with the last run and writes per task the ABX
 * error (errors[k], NaN for a task without cells) and, if triplets is not
 * NULL, its number of triples; stats (nullable) gets totals over the batch.
 */
typedef struct abx_batch abx_batch;
typedef struct abx_task_input {
    const float *feats;
    int64_t n_frames;
    int32_t dim;
    int32_t mem;
    const int64_t *item_offsets;
    int64_t n_items;
    const int32_t *labels;
} abx_task_input;
typedef struct abx_batch_info {
    int32_t n_tasks;
    int32_t n_classes;          /* dimension classes (shared launch sets)        */
    int64_t graph_kernels;      /* kernel nodes in the captured graph (0: none)  */
    int64_t n_triplets;         /* triples over all tasks                        */
    int64_t n_pairs_cap;        /* upper bound on item pairs over all tasks      */
    int64_t n_pairs;            /* needed item pairs (after a run and a wait)    */
    int64_t n_frame_pairs;      /* their sum of Tx * Ty (after a run and a wait) */
    double flops;               /* sum over classes of 2 * dim * frame pairs     */
    int64_t device_bytes;       /* device memory held by the batch (estimate)    */
    int32_t use_graph;          /* runs replay a CUDA graph                      */
    int32_t tile_variant[8];    /* per class (first 8): chosen kernel variants:  */
    int32_t dtw_variant[8];     /* 0..3 = tile kernel / DTW kernel variant, 4 =  */
                                /* the fused tile + DTW kernel (both fields)     */
    int32_t class_dim[8];
} abx_batch_info;
/* One task spec of a multi-spec batch: attributes as in abx_build_cells,
 * collapse levels as in abx_score (at most 8 by attributes, 16 tokens). */
typedef struct abx_task_spec {
    int32_t on_attr;
    int32_t n_by;
    int32_t by[8];
    int32_t across_attr;
    int32_t n_level_tokens;
    int32_t levels[16];
} abx_task_spec;
/* Several task specs over the same tasks share one device copy of the
 * features; errors and triplets of abx_batch_wait are then indexed
 * [task * n_specs + spec]. */
int abx_batch_create_multi(abx_ctx *ctx, int32_t n_tasks, const abx_task_input *tasks,
                           int32_t n_attr, int32_t n_specs, const abx_task_spec *specs,
                           int32_t mode, int32_t precision, int32_t weighted, int32_t recheck,
                           float margin, int32_t tune, void *stream, abx_batch **out);
int abx_batch_create(abx_ctx *ctx, int32_t n_tasks, const abx_task_input *tasks, int32_t n_attr,
                     int32_t on_attr, const int32_t *by, int32_t n_by, int32_t across_attr,
                     int32_t mode, int32_t precision, const int32_t *levels,
                     int32_t n_level_tokens, int32_t weighted, int32_t recheck, float margin,
                     int32_t tune, void *stream, abx_batch **out);
int abx_batch_run(abx_batch *batch, void *stream);
/* 1 if the last run has completed, 0 if not (no synchronisation). */
int abx_batch_ready(abx_batch *batch);
int abx_batch_wait(abx_batch *batch, double *errors, int64_t *triplets, abx_score_stats *stats);
int abx_batch_get_info(const abx_batch *batch, abx_batch_info *info);
/* Later runs replay the graph (on != 0) or enqueue the kernels directly. */
int abx_batch_set_graph(abx_batch *batch, int32_t on);
int abx_batch_free(abx_batch *batch);

/*
 * Serving (continuous batching of ABX jobs).
 *
 * A server runs n_planners planner threads and max_inflight executor
 * threads, each with its own CUDA stream.  abx_server_submit checks a job (item
 * offsets from 0 to n_frames, every item at least one frame, labels >= 0;
 * ABX_E_INVALID otherwise, and the job is not queued) and queues it (one
 * task's features, offsets and labels; every job is scored on the server's
 * task specs).  A planner takes queued jobs in arrival order while their
 * estimated device memory fits the budget (hbm_budget bytes, default 80% of
 * the device memory free at creation; a job that fits nowhere runs alone once
 * nothing else holds memory), up to max_batch_jobs, and joins them into one
 * batch (abx_batch_create_multi: one feature copy, shared launches for all of
 * them); a free executor launches it and waits for it.  Batching is just in
 * time: while every executor is busy, a planner waits until the earliest
 * one is expected to finish within the time that planning the queued jobs
 * takes (running estimates of host planning and GPU time per item), so jobs
 * that arrive meanwhile join the next batch; with an executor idle it plans
 * at once.  Host planning of one batch runs during the GPU work of the
 * previous ones.  A job's result equals what abx_distances + abx_score give
 * for its task alone.
 *
 * A batch of several jobs that fails (for instance a zero-norm frame found on
 * the GPU, or a failed allocation) is split and its jobs run again one by
 * one, so the error reaches only the job that caused it; stats.retried counts
 * the splits.  abx_server_cancel removes a job that is still queued (its
 * result: status ABX_E_CANCELLED).  cfg.fail_inject is a test hook that makes
 * one batch creation fail on the host as an allocation failure would.
 *
 * The job's feature, offset and label buffers must stay valid and unchanged
 * until the job has completed (abx_server_poll / abx_server_wait returned its
 * result); device features must be complete when submitted (the workers read
 * them on their own streams).  Job times are seconds on the server's clock
 * (steady, from the server's creation): submitted, admitted (its batch
 * formed), launched, and done (its batch complete).  While a server runs,
 * the context belongs to its threads (no other calls on it).
 * abx_server_destroy finishes the batches in flight, fails the queued jobs
 * with ABX_E_STATE and stops the threads.
 */
#define ABX_SERVER_MAX_SPECS 4
typedef struct abx_server abx_server;
typedef struct abx_server_config {
    int32_t n_attr;           /* label columns of every job                           */
    int32_t n_specs;
    abx_task_spec specs[ABX_SERVER_MAX_SPECS];
    int32_t mode, precision, recheck, weighted;
    float margin;
    int32_t max_inflight;     /* executor threads = batches on the GPU at once; 0 = 1  */
    int32_t max_batch_jobs;   /* jobs per batch; 0 = 32                                */
    int64_t hbm_budget;       /* device bytes the server may hold; 0 = 80% of free     */
    int32_t tune;             /* autotune kernel variants per shape key                */
    int32_t fail_inject;      /* test hook: the n-th batch creation fails as if a device
                                 allocation had failed (ABX_E_OOM); 0 = off             */
    int32_t n_planners;       /* planner threads (batches planned at once); 0 = 2      */
} abx_server_config;
typedef struct abx_job_result {
    int32_t status;           /* ABX_OK or the failing call's error code               */
    int32_t n_specs;
    double errors[ABX_SERVER_MAX_SPECS];
    int64_t triplets[ABX_SERVER_MAX_SPECS];
    double t_submit, t_admit, t_launch, t_done;
    int64_t batch_id;         /* jobs with the same id ran in one batch                */
    int32_t batch_jobs;       /* jobs in that batch                                    */
    int32_t reserved;
} abx_job_result;
typedef struct abx_server_stats {
    int64_t submitted, completed, failed, batches;
    int32_t max_inflight_seen, reserved;
    int64_t peak_bytes;       /* largest admitted device memory (estimate)            */
    int64_t cancelled;        /* jobs cancelled while queued                           */
    int64_t retried;          /* failed batches of several jobs split to run alone     */
} abx_server_stats;
int abx_server_create(abx_ctx *ctx, const abx_server_config *cfg, abx_server **out);
int abx_server_submit(abx_server *srv, const abx_task_input *job, int64_t *ticket);
/* Removes a queued job: its result (poll / wait) has status ABX_E_CANCELLED.
 * ABX_E_STATE if the job is already in a batch or done. */
int abx_server_cancel(abx_server *srv, int64_t ticket);
/* 1 and the result if the job is done, 0 if not yet. */
int abx_server_poll(abx_server *srv, int64_t ticket, abx_job_result *out);
int abx_server_wait(abx_server *srv, int64_t ticket, abx_job_result *out);
int abx_server_get_stats(abx_server *srv, abx_server_stats *out);
double abx_server_now(abx_server *srv);
int abx_server_destroy(abx_server *srv);

/*
 * abx_score_cells -- the per-cell integers behind abx_score, for inspection.
 * Writes up to `capacity` cells: keys (row of 4 + n_by int32:
 * on_ax, on_b, across_ab, across_x, by values in `by` order; across codes are
 * 0 without an across attribute), N and |C|.  *n_out receives the total
 * number of cells (call with capacity 0 to size the buffers).  Same recheck
 * semantics as abx_score.  Synchronises `stream`.
 */
int abx_score_cells(abx_ctx *ctx, abx_dist *dist, const abx_cells *cells, int32_t recheck,
                    void *stream, int64_t capacity, int32_t *keys, int64_t *num2,
                    int64_t *count, int64_t *n_out);

/*
 * abx_slice_frames -- frames of a unit spanning [t_on, t_off] (App. A,
 * Eqs. 1-4).  Frame i has time t_i = dt/2 + i*dt and is kept when
 * t_on <= t_i <= t_off:  first = ceil(t_on/dt - 1/2), last = floor(t_off/dt - 1/2),
 * both included.  With libri_light != 0 the last kept frame is dropped
 * (the Libri-Light slicing convention, App. A).  Times are integers in one
 * common unit (microseconds, samples, ...), so the bounds are exact.  An
 * empty slice is reported as *last < *first.  ABX_E_INVALID unless
 * dt > 0 and 0 <= t_on <= t_off.  Host only.
 */
int abx_slice_frames(int64_t t_on, int64_t t_off, int64_t dt, int32_t libri_light,
                     int64_t *first, int64_t *last);
/* The same for n units (host arrays of n entries each). */
int abx_slice_items(int64_t n, const int64_t *t_on, const int64_t *t_off, int64_t dt,
                    int32_t libri_light, int64_t *first, int64_t *last);

/*
 * abx_dtw_pairs_noalloc -- DTW distances of explicit item pairs, allocating
 * nothing.  The paper has no counterpart: this entry point serves callers
 * that cannot allocate device (or pinned host) memory -- code running under a
 * memory pool it does not own, a real-time serving loop where an allocation
 * could stall, an application that gave all device memory to its own
 * allocator.  Same distance as abx_distances with ABX_DTW / ABX_FP32_SIMT:
 * FP32 angular frame distances, DTW with steps (i-1,j), (i,j-1), (i-1,j-1),
 * shorter path on equal cost, cost / optimal path length.
 *
 *   feats         device, n_frames x dim FP32 row-major (items back to back)
 *   item_offsets  host, n_items + 1 CSR frame offsets (0 .. n_frames)
 *   pairs         host, n_pairs x 2 int64 item indices (x rows, y columns)
 *   dist          device, n_pairs FP32 outputs
 *   len           device, n_pairs int32 optimal path lengths, or NULL
 *   stream        stream to run on (asynchronous; outputs valid after it)
 *
 * Work space is one static __device__ array of about 18 MiB that every GPU
 * loading the library holds until process exit.  Limits, rejected with
 * ABX_E_UNSUPPORTED before any GPU work: n_pairs <= 65536, sum over pairs of
 * Tx*Ty <= 2^22, items of 1..128 frames.  Items of a pair must lie inside
 * 0..n_frames (ABX_E_INVALID otherwise).  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current.  The call stages its pair table with a copy from static
 * host memory, which stream capture cannot record: it must not be called
 * while `stream` is capturing and returns ABX_E_UNSUPPORTED if it is.
 * Every call reuses the same array: calls whose GPU work overlaps (different
 * streams, or different host threads) race on it and must be serialised by
 * the caller; the host side of the call is serialised by a mutex.  The
 * caller must size `dist` (and `len`) for n_pairs entries; the library
 * cannot check device buffer sizes.
 *
 * A frame of zero L2 norm has no angular distance: every pair containing it
 * gets dist = NaN (and len 0), and the call sets a status word in the static
 * array (cleared at the start of each call).  abx_dtw_pairs_noalloc_check
 * reads it.
 */
int abx_dtw_pairs_noalloc(const float *feats, int64_t n_frames, int32_t dim,
                          const int64_t *item_offsets, int64_t n_items, const int64_t *pairs,
                          int64_t n_pairs, float *dist, int32_t *len, void *stream);
/* Status of the last abx_dtw_pairs_noalloc call on the current device:
 * synchronises `stream` (the stream that call ran on), then returns
 * ABX_E_ZERO_NORM if one of its frames had zero norm, else ABX_OK.
 * Allocates nothing (the word is read into static host storage). */
int abx_dtw_pairs_noalloc_check(void *stream);

/* ---------------------------------------------------------- diagnostics
 * Not part of the method: launch accounting and per-kernel timing used by the
 * benchmark.  abx_kernel_launches counts every kernel this library has
 * launched in the process.  With abx_prof_enable(1) each launch is bracketed
 * by CUDA events on its own stream; abx_prof_read(i, ...) returns the i-th
 * kernel name (alphabetical), its accumulated milliseconds and launch count
 * (ABX_E_INVALID past the last one), waiting for pending launches first. */
int64_t abx_kernel_launches(void);
/* Bound on |computed - exact| of the cosine of two stored frame vectors that
 * the distance kernels use at `precision` (ABX_FP32_SIMT .. ABX_FP8) for
 * features of dimension `dim` (padded to a multiple of 128): the cosine error
 * behind every distance interval.  Tensor-core precisions assume the
 * accumulation model stated with cosine_error_bound in csrc/abx_host.cu (one
 * MMA instruction of K products commits at most (K + 2) units of 2^-23 of the
 * magnitudes it adds).  Host only; -1 for an invalid argument. */
double abx_cosine_error_bound(int32_t precision, int32_t dim);
int abx_prof_enable(int32_t on);
int abx_prof_reset(void);
int abx_prof_read(int32_t index, char *name, int32_t name_cap, double *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* ABX_H */
