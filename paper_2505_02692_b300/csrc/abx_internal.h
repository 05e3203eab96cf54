// Internal structures and kernel entry points of libabx (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/abx.h"

namespace abx {

constexpr int kPanel = 128;        // frame rows per panel = tile edge
constexpr int kMaxItemLen = 128;   // longest item a panel can hold
constexpr int kMaxDims = 16;       // collapse key digits handled on device
constexpr int kMaxSubCap = 256;    // largest subsampler cap on |A|, |B|, |X|

void set_error(const char *fmt, ...);

// Adds one to the launch counter (no timing, no CUDA calls).
void count_launch();
void count_launches(long long n);  // kernels of a replayed graph

// Counts a kernel launch and, when timing is on, brackets it with CUDA events
// on its stream.  Construct immediately before the launch, in a scope that
// ends right after it.
class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
  private:
    const char *name_;
    cudaStream_t s_;
    void *a_ = nullptr;
};

// Host phase trace (ABX_TRACE=1 prints phase durations to stderr).
struct Trace {
    bool on;
    const char *what;
    std::chrono::steady_clock::time_point t0, last;
    explicit Trace(const char *w) : on(getenv("ABX_TRACE") != nullptr), what(w) {
        t0 = last = std::chrono::steady_clock::now();
    }
    void mark(const char *phase) {
        if (!on) return;
        auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[abx] %s %-16s %8.3f ms\n", what, phase,
                std::chrono::duration<double, std::milli>(now - last).count());
        last = now;
    }
};


// ----------------------------------------------------------------- objects

// Pinned host buffers reused across calls.  A released buffer is handed out
// again only once the event recorded at its release has completed, i.e. once
// the copy that read it is done.
struct PinnedPool {
    struct Buf {
        void *p;
        size_t n;
        cudaEvent_t ev;
        bool busy;
    };
    std::mutex mu;
    std::vector<Buf> bufs;
    void *acquire(size_t n);                // nullptr on failure
    void release(void *p, cudaStream_t s);  // reusable once s passes this point
    ~PinnedPool();
};

struct Ctx {
    int device = 0;
    int n_sm = 0;
    // references: the handle from abx_ctx_create plus one per live object
    // (items, cells, distances, batch, server); freed at zero, so objects may
    // be freed after abx_ctx_destroy
    std::atomic<int64_t> refs{1};
    PinnedPool pinned;
    // autotuner results: key (precision, mode, dim_pad, length class) ->
    // (tile kernel variant, DTW kernel variant)
    std::mutex tune_mu;
    std::map<std::string, std::pair<int32_t, int32_t>> tuned;
    // Device scratch kept between calls (the tile buffer of abx_distances,
    // up to 8 GiB): a few slots that calls borrow in stream order
    // (scratch_acquire / scratch_release), so that a step does not allocate
    // and free it each time (the stream-ordered pool, fragmented by the
    // smaller allocations between, grew by 7 GiB, 7-8 ms of host time, on
    // about every second step).  Freed with the context.
    struct ScratchSlot {
        void *p = nullptr;
        size_t n = 0;
        cudaEvent_t ev = nullptr;   // end of the last use
        cudaStream_t last = nullptr;
        bool busy = false;
    };
    std::mutex scratch_mu;
    std::vector<ScratchSlot> scratch;
    // End of the last host-to-device feature copy abx_load_items enqueued
    // (ABX_MEM_HOST).  The library's small uploads take the copy engine
    // while no such copy is pending, else a kernel that reads the pinned
    // buffer over the bus: a copy engine serves the queued copies of all
    // streams in submission order, so a small copy would wait for the rest
    // of a multi-gigabyte one.
    std::mutex copy_mu;
    cudaEvent_t feat_copy = nullptr;
    ~Ctx();
};
// Borrows at least n bytes of scratch for work enqueued on s (stream s waits
// for the slot's previous use when that ran on another stream); nullptr if
// no slot fits and no more may be made (the caller then allocates).
void *scratch_acquire(Ctx *c, size_t n, cudaStream_t s, int *slot);
// Ends the borrow: the slot is reusable once s passes this point.
void scratch_release(Ctx *c, int slot, cudaStream_t s);

// Flags the pack kernel sets (deferred errors of abx_distances).
constexpr int32_t kPackZeroNorm = 1;     // a frame with zero L2 norm
constexpr int32_t kPackNonPositive = 2;  // KL: a component <= 0

// Packed rows of one sorted item order: the normalised, quantised features
// in that order with per-row norms and quantisation angles and per-item
// angles.  Tasks over one item set often sort the items identically (the
// within- and across-speaker tasks both order by context, speaker, phone),
// so abx_distances keeps the last packing with the items and reuses it when
// the order, mode, distance and precision match.
struct PackedRows {
    int32_t mode = 0, distance = 0, precision = 0, dim_pad = 0;
    std::vector<int32_t> order;        // sorted item order (original indices)
    void *packed = nullptr;
    float *inv_norm = nullptr, *nrm2 = nullptr, *theta = nullptr, *scale = nullptr;
    float *theta_item = nullptr;
    int32_t *err = nullptr;            // the pack kernel's flags (zero-norm frame)
    cudaEvent_t ready = nullptr;       // recorded after the pack kernel
    std::vector<cudaEvent_t> uses;     // recorded after each user's kernels
    int32_t refs = 0;                  // the items' cache + plans using it
};

struct Items {
    Ctx *ctx = nullptr;
    int64_t n_items = 0, n_frames = 0;
    int32_t dim = 0, n_attr = 0;
    std::vector<int64_t> h_offsets;   // n_items + 1
    const float *d_feats = nullptr;   // n_frames x dim
    bool owns_feats = false;
    int64_t *d_offsets = nullptr;     // n_items + 1
    int32_t *d_labels = nullptr;      // n_items x n_attr (same block as d_offsets)
    cudaStream_t stream = nullptr;    // stream the items were loaded on
    cudaEvent_t ready = nullptr;      // the uploads are complete
    int32_t max_len = 1;              // longest item (frames)
    std::vector<int32_t> label_max;   // per attribute: largest code
    mutable std::mutex pack_mu;       // guards pack
    mutable PackedRows *pack = nullptr;  // last packing (abx_distances)
};

// One entry of a group's item-pair matrix: distance, interval holding the
// exact distance, optimal path length (0 = not computed).
struct __align__(16) PairVal {
    float d, lo, hi;
    uint32_t len;
};

// One device-side view of a task, passed by value to kernels.
struct TaskDev {
    int32_t n_items;
    int32_t K_on, K_s;
    int32_t n_groups;
    int32_t across;             // 1 if the task has an across attribute
    const int32_t *item_id;     // sorted index -> original item
    const int32_t *item_g;      // sorted index -> group
    const int32_t *item_p;      // sorted index -> on code
    const int32_t *item_s;      // sorted index -> across code (0 if none)
    const int32_t *group_begin; // n_groups + 1, sorted item ranges
    const int64_t *group_dm;    // n_groups, offset of the group's n_g x n_g matrices
    const int2 *blk;            // [g][s][p] -> (first sorted item, count)
    const int32_t *tot;         // [g][s] -> items of the group with that across code
    const int4 *gmeta;          // [g] -> (first sorted item, n_g, matrix offset lo, hi)
};

__device__ __forceinline__ int blk_count(const TaskDev &t, int g, int p, int s) {
    return t.blk[((int64_t)g * t.K_s + s) * t.K_on + p].y;
}

// Unordered pair {x, y} (same group, x != y) is needed when one of them can
// be the X of a triple in which the other is A or B (symmetric in x, y).
//   no across: same on -> needs some b of another on value in the group;
//              different on -> the X item needs a second item of its on value.
//   across:    across values must differ; same on -> the A item's across
//              value needs some b of another on value; different on -> the
//              B item's across value needs an a with the X item's on value.
__device__ __forceinline__ bool pair_needed(const TaskDev &t, int x, int y) {
    const int g = t.item_g[x];
    const int px = t.item_p[x], py = t.item_p[y];
    if (!t.across) {
        if (px == py) return t.tot[g] - blk_count(t, g, px, 0) > 0;
        return blk_count(t, g, px, 0) >= 2 || blk_count(t, g, py, 0) >= 2;
    }
    const int sx = t.item_s[x], sy = t.item_s[y];
    if (sx == sy) return false;
    if (px == py)
        return t.tot[(int64_t)g * t.K_s + sy] - blk_count(t, g, px, sy) > 0 ||
               t.tot[(int64_t)g * t.K_s + sx] - blk_count(t, g, px, sx) > 0;
    return blk_count(t, g, px, sy) > 0 || blk_count(t, g, py, sx) > 0;
}

struct Cells {
    Ctx *ctx = nullptr;
    const Items *items = nullptr;
    int32_t on = 0, across = -1;
    std::vector<int32_t> by;
    int32_t K_on = 0, K_s = 1;
    std::vector<int32_t> K_by;
    int64_t by_space = 1;           // prod K_by
    int32_t n_groups = 0;
    abx_cells_info info{};
    // host copies
    std::vector<int32_t> item_id, group_begin;
    std::vector<int64_t> group_dm;
    std::vector<int2> blk;          // [g][s][p]
    std::vector<int32_t> tot;
    std::vector<int32_t> item_group;  // original item -> group
    std::vector<int32_t> gtab;      // dense by-code -> group or -1
    std::vector<int4> gmeta;        // per group (first item, n_g, matrix offset)
    int64_t dm_entries = 0;         // sum n_g^2
    int64_t n_cand = 0;             // cells the scorer enumerates (size of its cell arrays)
    std::atomic<int32_t> jobs{0};   // outstanding abx_score_submit jobs
    bool info_done = false;         // n_blocks / n_cells / n_triplets computed
    int32_t sub_cap = 0, sub_xmax = 0;  // subsampler (abx_cells_set_subsampler)
    uint64_t sub_seed = 0;
    // device copies (one block, uploaded on `stream`, complete at `ready`)
    cudaStream_t stream = nullptr;
    cudaEvent_t ready = nullptr;
    uint8_t *d_block = nullptr;
    int32_t *d_item_id = nullptr, *d_item_g = nullptr, *d_item_p = nullptr, *d_item_s = nullptr;
    int32_t *d_group_begin = nullptr;
    int64_t *d_group_dm = nullptr;
    int2 *d_blk = nullptr;
    int32_t *d_tot = nullptr;
    int32_t *d_gtab = nullptr;
    int4 *d_gmeta = nullptr;
    TaskDev dev() const;
    void compute_info();
};

struct Dist {
    Ctx *ctx = nullptr;
    const Items *items = nullptr;
    const Cells *cells = nullptr;
    cudaStream_t stream = nullptr;
    int32_t mode = ABX_DTW, precision = ABX_FP32_SIMT, distance = ABX_DIST_ANGULAR;
    abx_dist_info info{};
    int32_t max_len = 1;
    uint8_t *d_block = nullptr;       // device block holding d_len / d_row
    int64_t pair_cap = 0;             // upper bound on needed pairs (host-known)
    // per sorted item (device): length used by the kernels, first packed row
    int32_t *d_len = nullptr;
    int32_t *d_row = nullptr;
    // group matrices (device, dm_entries each)
    PairVal *d_pv = nullptr;
    // counters (device) and their pinned host mirror, valid after a sync:
    // [0] zero-norm flag, [1] tile pipeline error code; counts: [0] needed
    // pairs, [1] needed frame pairs
    int32_t *d_err = nullptr;
    int64_t *d_count = nullptr;
    void *h_mirror = nullptr;
    int32_t *h_err = nullptr;
    int64_t *h_count = nullptr;
    bool synced = false;
    int64_t n_pairs = 0;
    cudaEvent_t done = nullptr;       // recorded after the last distance kernel
    std::atomic<int32_t> jobs{0};     // outstanding abx_score_submit jobs
};

// Distance plan: everything abx_distances sets up on the host and the device
// (packed-row layout, panels, tiles, chunking, buffers), separated from the
// kernels that run on it so that a plan can be executed repeatedly (and be
// captured in a CUDA graph: execution only enqueues memsets and kernels).
struct DistPlan {
    Ctx *ctx = nullptr;
    const Items *it = nullptr;
    const Cells *c = nullptr;
    int32_t mode = ABX_DTW, distance = ABX_DIST_ANGULAR, precision = ABX_FP32;
    int64_t n = 0, rows = 0, n_tiles = 0, chunk = 1, cap_max = 0, cap_total = 0;
    int32_t dim = 0, dim_pad = 0, max_len = 1;
    size_t elem = 4;
    bool fused = false;
    int32_t fuse_form = 0;  // fused kernel's DTW: 0 thread per pair in place, 1 8-lane wavefronts
    std::vector<int64_t> chunk_cap;
    // kernel variants chosen by the autotuner (0 = default)
    int32_t umma_variant = 0, dtw_variant = 0;
    // device buffers; the first group outlives the plan in a Dist
    uint8_t *keep_block = nullptr;    // d_len, d_row
    int32_t *d_len = nullptr, *d_row = nullptr;
    float *theta_item = nullptr;
    PairVal *pv = nullptr;
    int64_t dm = 1;
    int32_t *d_err = nullptr;
    int64_t *d_count = nullptr;
    // temporaries
    uint8_t *plan_block = nullptr;    // panels, tiles, work items
    int32_t *d_panel_row = nullptr, *d_panel_item = nullptr;
    int2 *d_tiles = nullptr;
    int2 *d_work = nullptr;           // per chunk: pairs of adjacent tiles (wide kernel)
    std::vector<int64_t> work_off;    // per chunk: first work item (n_chunks + 1)
    void *packed = nullptr;
    float *inv_norm = nullptr, *nrm2 = nullptr, *theta = nullptr, *scale = nullptr;
    // share_pack: look up / publish the packing in the items' cache; shared:
    // the entry that owns packed .. theta_item (the plan does not free them)
    bool share_pack = false;
    PackedRows *shared = nullptr;
    bool pack_hit = false;            // shared was found, not packed here
    std::vector<int32_t> h_len, h_row;  // host copies between the build parts
    int32_t *tile_count = nullptr;
    int64_t *tile_base = nullptr, *chunk_total = nullptr;
    float *tilebuf = nullptr;
    int32_t *d_row_item = nullptr;    // packed row -> sorted item (tile buffer strips)
    bool use_scratch = false;         // tile buffer from the context's scratch slots
    int scratch_slot = -1;
    int32_t strips = 0, listed_only = 1;  // tile buffer layout and store rule
    uint64_t *d_xmask = nullptr;      // per tile of a chunk: store map (launch_plan_count)
    uint8_t *d_col_yo = nullptr;
    int4 *pairs = nullptr;
};
// Bound on |computed cosine - exact cosine of the stored vectors|.
float cosine_error_bound(int precision, int dim_pad);
// Host plan, allocations and uploads (stream-ordered on s).  Returns ABX_*.
// In two parts: the packed rows (with p->share_pack, found in or added to the
// items' cache), then panels, tiles, chunks and work items.
int dist_plan_build(Ctx *ctx, const Items *it, const Cells *c, int32_t mode, int32_t distance,
                    int32_t precision, cudaStream_t s, DistPlan *p);
int dist_plan_build_rows(Ctx *ctx, const Items *it, const Cells *c, int32_t mode,
                         int32_t distance, int32_t precision, cudaStream_t s, DistPlan *p);
int dist_plan_build_tiles(cudaStream_t s, DistPlan *p);
// Memsets and kernels only.  Returns ABX_*.  Also in two parts: the pack
// (or, for a cache hit, a wait for it), then planning, tiles and DTW.
int dist_plan_exec(const DistPlan &p, cudaStream_t s);
int dist_plan_exec_pack(const DistPlan &p, cudaStream_t s);
int dist_plan_exec_tiles(const DistPlan &p, cudaStream_t s);
// Drops one reference to a packing of the items; the last frees its buffers
// on stream s after every recorded use.
void packed_rows_release(const Items *it, PackedRows *pr, cudaStream_t s);
cudaStream_t build_stream(int device);  // per (thread, device), for cell building
void ctx_retain(Ctx *c);
void ctx_release(Ctx *c);  // deletes the context at zero references

// Device bytes the plan holds (buffers of dist_plan_build).
int64_t dist_plan_bytes(const DistPlan &p);
// Frees the temporaries (and, if all, the persistent buffers too).
void dist_plan_free(DistPlan *p, cudaStream_t s, bool all);

// Score plan of a group-structured task (many tasks joined by a leading
// group attribute): buffers sized on the host, execution without host
// synchronisation (capturable), per-group errors.
struct ScorePlanB;
int score_plan_b_build(Ctx *ctx, const Cells *c, const Items *it, const DistPlan &dp,
                       const int32_t *levels, int32_t n_tok, int32_t weighted, int32_t recheck,
                       float margin, cudaStream_t s, ScorePlanB **out);
int score_plan_b_exec(ScorePlanB *b, cudaStream_t s);
int score_plan_b_read(const ScorePlanB *b, double *errors, int64_t *triplets,
                      abx_score_stats *stats);
void score_plan_b_free(ScorePlanB *b, cudaStream_t s);

// ------------------------------------------------------------ kernel hosts
// Every launcher enqueues on `s` and returns a cudaError_t.

struct PackArgs {
    const float *feats;       // raw features, original order
    const int64_t *offsets;   // original item offsets
    const int32_t *item_id;   // sorted -> original
    const int32_t *row;       // sorted -> first packed row
    const int32_t *len;       // sorted -> packed rows of the item
    int32_t n_items, dim, dim_pad, mode, precision, distance;
    int64_t n_rows;
    void *packed;             // packed storage (precision-dependent layout)
    float *inv_norm;          // per packed row: 1 / |stored vector| (angular, cosine) or
                              // the factor that turns stored values into raw ones (Euclidean)
    float *nrm2;              // per packed row: |raw vector|^2 as stored (Euclidean)
    float *theta;             // per packed row: angle stored vs exact
    float *theta_item;        // per sorted item: max theta
    float *item_scale;        // per sorted item: FP8 scale (scratch)
    int32_t *err;
};
cudaError_t launch_pack(const PackArgs &a, cudaStream_t s);

// Per sorted item: group (through the dense by-code table), on and across codes.
struct ItemAttrArgs {
    const int32_t *item_id, *labels, *gtab;
    int32_t n_items, n_attr, on, across, n_by;
    int32_t by[8], K_by[8];
    int32_t *item_g, *item_p, *item_s;
};
cudaError_t launch_item_attrs(const ItemAttrArgs &a, cudaStream_t s);

struct TileList {
    const int2 *tiles;        // (panel i, panel j)
    const int32_t *panel_row; // first packed row of each panel
    const int32_t *panel_item;// first sorted item of each panel (n_panels + 1 entries)
    int64_t n_tiles;
};

// Counts needed pairs per tile and adds their Tx * Ty to *frame_pairs.
// Count pass; also writes, per tile of the list, the store map of the tile
// kernels' epilogue (nullable; row_item: packed row -> sorted item, n_rows
// packed rows): col_yo[t * 128 + c] = index of the column panel's item
// holding tile column c (255 past its last item), and, when the column panel
// has at most 64 items, xmask[t * 128 + xo] = bit yo set iff the pair (row
// item xo, column item yo) is listed (needed, and y > x on a diagonal tile).
cudaError_t launch_plan_count(const TaskDev &t, const TileList &tl, const int32_t *len,
                              const int32_t *row, int32_t *tile_count, int64_t *frame_pairs,
                              uint64_t *xmask, uint8_t *col_yo, const int32_t *row_item,
                              int64_t n_rows, cudaStream_t s);
cudaError_t launch_plan_write(const TaskDev &t, const TileList &tl, const int32_t *len,
                              const int32_t *row, const int64_t *tile_base, int4 *pairs,
                              cudaStream_t s);
// Exclusive scan; writes the total to *total and adds it to *accum.
cudaError_t launch_scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total,
                                   int64_t *accum, cudaStream_t s);

// Cell building on the device (csrc/abx_cells.cu).
struct CellBuildArgs {
    const int32_t *labels;       // n x n_attr
    int64_t n;
    int32_t n_attr, on, across, n_by;
    int32_t by[8], K_by[8];
    int32_t K_on, K_s;
    int64_t by_space, nkeys;
    // scratch
    int32_t *flags;              // by_space: group present
    int64_t *gpos;               // by_space + 1: group numbers (scan of flags)
    int32_t *counts;             // nkeys_max: items per key
    int64_t *pos;                // nkeys_max + 1: first item of each key
    int64_t *cursor;             // nkeys_max: scatter positions
    int64_t *key;                // n: key of each item
    int32_t *ng2;                // g_max: items per group
    int32_t *nz_s;               // g_max * K_s: non-empty blocks per (group, across)
    // results
    int64_t *n_groups;           // 1
    int64_t *dm_total;           // 1: sum of n_g^2
    int32_t *gtab;               // by_space: by code -> group or -1
    int32_t *item_group;         // n: group of each item (original order)
    int32_t *item_id;            // n: sorted position -> item
    int2 *blk;                   // g_max * K_s * K_on
    int32_t *tot;                // g_max * K_s
    int32_t *group_begin;        // g_max + 1
    int64_t *group_dm;           // g_max
    int4 *gmeta;                 // g_max
    int64_t *n_cand;             // 1: score candidates (cells the scorer enumerates)
};
cudaError_t launch_cell_build(const CellBuildArgs &a, int64_t nkeys_max, int64_t g_max,
                              int64_t *scratch, cudaStream_t s);

struct TileGemmArgs {
    const void *packed;
    const float *inv_norm;
    int64_t n_rows;
    int32_t dim_pad;
    const int2 *tiles;
    const int32_t *panel_row;
    const int32_t *tile_count;   // tiles with zero needed pairs are skipped
    int64_t n_tiles;
    float *tilebuf;              // n_tiles x 128 x 128 frame distances
    int32_t distance;            // ABX_DIST_*
    const float *nrm2;           // per packed row |raw|^2 (Euclidean), sum p ln p (KL)
    int32_t *err;                // set to a nonzero code if a bounded wait expires
    int32_t b_rot = 0;           // B operand's k offset (elements, mod dim_pad): KL
    // fused tile + DTW (tcgen05 path, items of at most umma_fuse_max_len() frames):
    // 0 off, 1 a thread per pair in place on the shared d tile, 2 8-lane wavefronts
    int32_t fused;
    const int4 *pairs;           // the chunk's needed pairs, in tile order
    const int64_t *tile_base;    // per tile of the chunk: first pair (n_tiles + 1)
    const int32_t *len;
    const float *theta_item;
    float eps_c;
    int32_t intervals;
    const int32_t *item_g;
    const int4 *gmeta;
    PairVal *pv;
    int32_t variant = 0;         // kernel variant (autotuner)
    // work items of the wide tile kernel: (tile, next tile of the same panel
    // row or -1), tile indices relative to the chunk
    const int2 *work = nullptr;
    int64_t n_work = 0;
    // tile buffer in strips (tile_strip_offset): packed row -> sorted item,
    // sorted item -> first packed row, panel -> first item (+ sentinel), and
    // the per-tile map of the blocks the tcgen05 kernels store (the listed
    // pairs' blocks)
    const int32_t *row_item = nullptr;
    const int32_t *row = nullptr;
    const int32_t *panel_item = nullptr;
    const uint64_t *xmask = nullptr;   // launch_plan_count's store map
    const uint8_t *col_yo = nullptr;
    int32_t strips = 0;                // tile buffer layout: 1 strips, 0 column-major
    int32_t listed_only = 1;           // narrow / pair kernels: store only the listed blocks
};
cudaError_t launch_tile_simt(const TileGemmArgs &a, cudaStream_t s);
cudaError_t launch_tile_umma(const TileGemmArgs &a, int precision, int n_sm, cudaStream_t s);
bool umma_supported(int precision);
int umma_fuse_max_len();
// True when launch_tile_umma runs the wide kernel, which writes column-major
// tiles with every entry (TileGemmArgs::strips and listed_only do not apply).
bool umma_wide(int precision, int variant);

// Tile buffer layout.  In the tile of panel pair (pi, pj) the rows of each
// item x of panel pi (tile rows rx .. rx + Tx - 1) form a strip of Tx x 128
// entries stored column by column: entry (i, c) at rx * 128 + c * Tx +
// (i - rx).  The block of an item pair (x, y), tile columns cy .. cy + Ty - 1,
// is then Tx * Ty consecutive floats, column by column, which the DTW reads
// front to back.  Rows past the panel's last item belong to no strip.
__host__ __device__ __forceinline__ int64_t tile_strip_offset(int rx, int Tx, int i, int c) {
    return (int64_t)rx * kPanel + (int64_t)c * Tx + (i - rx);
}
cudaError_t launch_row_items(const int32_t *len, const int32_t *row, int64_t n_items,
                             int32_t *row_item, cudaStream_t s);

struct DtwArgs {
    TaskDev t;
    const int4 *pairs;
    const int64_t *n_pairs;      // device count
    int64_t pair_cap;            // host upper bound (grid sizing)
    const float *tilebuf;
    int32_t strips = 0;          // tile buffer layout (TileGemmArgs::strips)
    const int32_t *len;
    const float *theta_item;
    float eps_c;                 // bound on the cosine error of the kernel
    int32_t intervals;           // 1: angular distance, emit exact-value intervals
    int32_t max_len;
    PairVal *pv;
    int32_t variant = 0;         // kernel variant (autotuner)
};
cudaError_t launch_dtw(const DtwArgs &a, cudaStream_t s);


// ------------------------------------------------------------ scoring

// Unsigned 32-bit division by an invariant divisor d >= 1 as a multiply-high
// and two shifts (Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994, Sec. 4): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, the quotient of n is
// (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = high word of m * n.
struct FastDiv {
    uint32_t m = 1, s1 = 0, s2 = 0;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv &f) {
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
#endif

struct CollapseDigit {
    int32_t comp;     // 0 = P, 1 = Q, 2.. = by position + 2, 2 + n_by = across pair
    int32_t radix;
    FastDiv fd;       // division by radix
};

struct ScoreArgs {
    TaskDev t;
    const PairVal *pv;
    int32_t recheck;             // 0 off, 1 intervals, 2 stated margin
    float margin;                // recheck 2: undecided when |d_xa - d_xb| < margin
    int32_t pass;                // 0 mark, 1 score, 2 count cells, 3 emit cells
    int32_t stage;               // recheck stage: 0 mark undecided pairs, 1 decide from
                                 // the refined intervals (mark the rest for FP64),
                                 // 2 refined intervals, then FP64 values
    int32_t gate;                // run only if acc[gate] != 0 (0: always)
    int32_t dirty_slot;          // acc entry counting cells that met a deferred triple
    const int32_t *gtab;
    int32_t n_by;
    int32_t by_radix[kMaxDims];
    int32_t n_seg_digits, n_loop_digits;
    CollapseDigit seg[kMaxDims], loop[kMaxDims];
    int64_t n_seg;
    int64_t loop_len;
    // presence bitsets over level-1 values (when the level-1 attributes are
    // by attributes only): row ((p * K_s + s) * rest_radix + rest) holds bit l
    // set iff the block (group(l, rest), p, s) is non-empty
    const uint32_t *bits;
    int32_t bits_words;
    int32_t n_rest;
    int32_t rest_by[kMaxDims];   // by positions outside level 1, in by order
    int64_t rest_radix;
    // recheck state
    int32_t *rc_idx;             // canonical pair entry -> slot, -1 (not flagged), -2
                                 // (flagged, slot not yet assigned)
    int64_t rc_dm;               // entries of rc_idx
    int32_t *rc_block_n;         // compaction scratch (compact_blocks(rc_dm) entries)
    int2 *rc_list;               // exact slot -> (x, y) sorted indices
    int32_t *rc_count;
    int32_t rc_capacity;
    const double *rc_exact;      // exact distances per slot
    const float2 *rc_iv;         // refined interval per slot (NULL: no refined stage)
    int32_t *rc_state;           // per slot: 1 once listed for FP64
    int32_t *rc64_list;          // slots listed for FP64
    int32_t *rc64_count;
    // outputs
    double *res;                 // per segment: mean of D_C over the loop
    int32_t *res_n;              // per segment: cells averaged
    unsigned long long *acc;     // [0]=sum N, [1]=sum 2|C|, [2]=cells, [3]=triplets,
                                 // [4]=undecided, [5]=flips, [6]=overflow flag,
                                 // [7]=cells that met a triple not yet rechecked,
                                 // [8]=the same after the refined stage (kAccN entries)
    int64_t *cell_count;         // pass 2: cells per segment; pass 3: base offsets
    int32_t *cell_keys;          // pass 3
    int64_t *cell_num2, *cell_cnt;
    int32_t key_width;
    // materialised cells (bitset path): per segment the candidate count and
    // base, per cell (segment, level-1 value)
    int32_t *seg_n;
    int64_t *seg_base;
    int2 *cell_id;
    const int64_t *n_cells_dev;  // total candidates (device)
    int64_t cell_cap;            // host upper bound
    int64_t *big;                // cells evaluated one warp each (capacity cell_cap)
    int64_t *big_count;
    // subsampler: caps on |A|, |B|, |X| per cell and on the across_x values
    // per (by, on_ax, on_b, across_ab); 0 = off
    int32_t sub_cap, sub_xmax;
    uint64_t sub_seed;
    FastDiv ks_div;              // division by K_s (across pair code -> s_ab, s_x)
};
cudaError_t launch_score(const ScoreArgs &a, cudaStream_t s);

// Presence bitsets: bit l of row ((p * K_s + s) * rest_radix + rest) is set
// iff the group with level-1 value l (mixed radix of the by attributes
// loop_by) and other by values rest has a non-empty (p, s) block.
struct BitsArgs {
    const int2 *blk;           // [g][s][p] -> (first, count)
    const int32_t *gtab;       // by code -> group or -1
    int64_t by_space;
    int32_t n_by;
    int32_t by_radix[kMaxDims];
    int32_t K_on, K_s;
    int32_t n_loop, loop_by[kMaxDims];   // by positions of the level-1 digits
    int32_t n_rest, rest_by[kMaxDims];   // the other by positions, in by order
    int32_t words;
    uint32_t *bits;
};
cudaError_t launch_bits(const BitsArgs &b, cudaStream_t s);
// Bitset path: candidate counts per segment; enumeration; evaluation of
// every cell; ordered per-segment means.
cudaError_t launch_seg_count(const ScoreArgs &a, cudaStream_t s);
cudaError_t launch_cell_enum(const ScoreArgs &a, cudaStream_t s);
cudaError_t launch_cell_eval(const ScoreArgs &a, cudaStream_t s);
cudaError_t launch_seg_reduce(const ScoreArgs &a, cudaStream_t s);
cudaError_t launch_cell_emit(const ScoreArgs &a, cudaStream_t s);

cudaError_t launch_collapse_level(const double *in, const int32_t *in_n, int64_t n_out,
                                  int64_t radix, double *out, int32_t *out_n, cudaStream_t s);
cudaError_t launch_final_mean(const double *in, const int32_t *in_n, int64_t n,
                              double *out, int64_t *out_n, cudaStream_t s);
// Zeroes acc[0..5] when acc[gate] != 0 (before a pass that scores again).
cudaError_t launch_reset_if_dirty(unsigned long long *acc, int gate, cudaStream_t s);
// Per-group final means: the collapsed array is indexed
// (outer * n_group + g) * inner + r; group g's mean runs over outer, then r,
// in increasing order (the order of the single-task final mean).
cudaError_t launch_final_group(const double *in, const int32_t *in_n, int64_t n_outer,
                               int32_t n_group, int64_t inner, double *out, int64_t *out_n,
                               cudaStream_t s);
// Per-group sums of N and |C| over the materialised cells; the group is the
// segment digit (seg / seg_div) % n_group.
cudaError_t launch_cell_group_sums(const ScoreArgs &a, int64_t seg_div, int32_t n_group,
                                   unsigned long long *num2, unsigned long long *cnt,
                                   cudaStream_t s);

struct RecheckArgs {
    const float *feats;          // raw features, original order
    const int64_t *offsets;
    const int32_t *item_id;
    int32_t dim, mode, max_len;
    const int2 *list;
    const int32_t *count;
    int32_t capacity;
    double *exact;
    const int32_t *slots;        // non-NULL: recompute list[slots[k]], k < *count
};
cudaError_t launch_recheck(const RecheckArgs &a, int32_t capacity, cudaStream_t s);

// Slots for the pairs flagged (-2) in rc_idx, assigned in entry order:
// rc_idx[e] = slot, rc_list[slot] = the pair's sorted item indices,
// *rc_count = the number flagged (acc[6] set if above capacity).  Runs only
// if acc[gate] != 0; block_n holds one int32 per 4096 entries.
struct CompactArgs {
    TaskDev t;
    int32_t *rc_idx;
    int64_t dm;
    int2 *rc_list;
    int32_t *rc_count;
    int32_t capacity;
    int32_t *block_n;
    unsigned long long *acc;
    int32_t gate;
};
cudaError_t launch_recheck_compact(const CompactArgs &c, cudaStream_t s);
inline int64_t compact_blocks(int64_t dm) { return (dm + 4095) / 4096; }

// Refined stage of the recheck (DTW, angular distance): every listed pair
// recomputed from the raw FP32 features on the CUDA cores, with an interval
// that holds the exact distance.
struct RefineArgs {
    const float *feats;
    const int64_t *offsets;
    const int32_t *item_id;
    int32_t dim, max_len;
    const int2 *list;
    const int32_t *count;
    int32_t capacity;
    float2 *iv;                  // per slot: [lo, hi]
    const float *inv_q;          // per frame (original order): 1 / |tf32(x)|
    const float *theta_frame;    // per frame (original order): TF32 rounding angle
    float eps_c;                 // cosine error bound of this kernel (refine_cosine_bound)
    int32_t group;               // pairs per warp and round (set by launch_refine)
    // two-kernel form (used when fd is set and rows are 16-byte aligned):
    float *fd;                   // frame distances of the listed pairs, fd_cap floats
    int64_t fd_cap;
    int64_t *fd_off;             // per slot: offset in fd, or -1 (did not fit)
    float *dev;                  // per slot: largest |d - 1/2|
    unsigned long long *fd_used; // allocation counter (zeroed by launch_refine)
};
cudaError_t launch_refine(const RefineArgs &a, int32_t capacity, cudaStream_t s);
struct RefinePrepArgs {
    const float *feats;
    const int64_t *offsets;
    int64_t n_items, n_frames;
    int32_t dim;
    float *inv_q;                // n_frames
    float *theta_frame;          // n_frames
    const unsigned long long *acc;  // runs only if acc[gate] != 0 (NULL: always)
    int32_t gate;
};
cudaError_t launch_refine_prep(const RefinePrepArgs &a, cudaStream_t s);
float refine_cosine_bound(int dim);
constexpr int kAccN = 10;        // entries of ScoreArgs::acc

// Gather group-matrix entries (entry < 0 or not computed gives NaN / 0).
cudaError_t launch_gather(const PairVal *pv, const int64_t *entries, int64_t n, float *oD,
                          float *olo, float *ohi, int32_t *oL, cudaStream_t s);

}  // namespace abx
