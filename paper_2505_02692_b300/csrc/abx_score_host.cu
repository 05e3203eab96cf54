// Host side of abx_score / abx_score_cells: builds the collapse plan from the
// level list (fastabx Sec. 2 weighting; Sec. 3.1 Score.collapse), runs the
// optional FP64 recheck, the level-1 scoring kernel, the further levels and
// the final mean.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "abx_internal.h"

using namespace abx;

#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                      __FILE__, __LINE__);                                         \
            return e_ == cudaErrorMemoryAllocation ? ABX_E_OOM : ABX_E_CUDA;       \
        }                                                                          \
    } while (0)

#define REQUIRE(cond, code, ...)      \
    do {                              \
        if (!(cond)) {                \
            set_error(__VA_ARGS__);   \
            return (code);            \
        }                             \
    } while (0)

namespace {

struct Plan {
    std::vector<std::vector<int>> levels;  // component ids per level
    std::vector<int> leftover;             // components not collapsed by a level
    std::vector<CollapseDigit> seg, loop;  // level-1 kernel digits
    std::vector<int64_t> level_radix;      // radix of each level >= 2 (innermost)
    int64_t n_seg = 1, loop_len = 1;
    // presence bitsets over the level-1 values (level 1 = by attributes
    // only), built on the device (launch_bits): bits_words x bits_rows words
    bool has_bits = false;
    int64_t bits_rows = 0;
    std::vector<int> rest_by;
    int64_t rest_radix = 1;
    int32_t words = 0;
};

// Bit l of row ((p * K_s + s) * rest_radix + rest) is set iff the group with
// level-1 value l and other by values `rest` has a non-empty (p, s) block.
// Available only when every level-1 digit is a by attribute; the rows are
// filled on the device from the block table (launch_bits).
void make_bits(const Cells *c, Plan *pl) {
    const int n_by = (int)c->by.size();
    for (auto &d : pl->loop)
        if (d.comp >= 2 + n_by) return;  // the across pair varies in the loop
    std::vector<bool> in_l1(n_by, false);
    for (auto &d : pl->loop) in_l1[d.comp - 2] = true;
    pl->rest_by.clear();
    pl->rest_radix = 1;
    for (int b = 0; b < n_by; ++b)
        if (!in_l1[b]) {
            pl->rest_by.push_back(b);
            pl->rest_radix *= c->K_by[b];
        }
    const int64_t W = (pl->loop_len + 31) / 32;
    const int64_t rows = (int64_t)c->K_on * c->K_s * pl->rest_radix;
    if (W * rows > (1LL << 24) || (int)pl->rest_by.size() > kMaxDims) return;
    pl->words = (int32_t)W;
    pl->bits_rows = rows;
    pl->has_bits = true;
}

// Device bitsets of the plan (stream-ordered; zeroed, then filled).
int upload_bits(const Cells *c, const Plan &pl, cudaStream_t s, uint32_t **out) {
    const size_t words = (size_t)pl.words * pl.bits_rows;
    CU(cudaMallocAsync((void **)out, std::max<size_t>(words, 1) * sizeof(uint32_t), s));
    CU(cudaMemsetAsync(*out, 0, words * sizeof(uint32_t), s));
    BitsArgs b;
    memset(&b, 0, sizeof(b));
    b.blk = c->d_blk;
    b.gtab = c->d_gtab;
    b.by_space = c->by_space;
    b.n_by = (int32_t)c->by.size();
    for (int i = 0; i < b.n_by; ++i) b.by_radix[i] = c->K_by[i];
    b.K_on = c->K_on;
    b.K_s = c->K_s;
    b.n_loop = (int32_t)pl.loop.size();
    for (size_t i = 0; i < pl.loop.size(); ++i) b.loop_by[i] = pl.loop[i].comp - 2;
    b.n_rest = (int32_t)pl.rest_by.size();
    for (size_t i = 0; i < pl.rest_by.size(); ++i) b.rest_by[i] = pl.rest_by[i];
    b.words = pl.words;
    b.bits = *out;
    CU(launch_bits(b, s));
    return ABX_OK;
}

int comp_radix(const Cells *c, int comp) {
    const int n_by = (int)c->by.size();
    if (comp < 2) return c->K_on;
    if (comp < 2 + n_by) return c->K_by[comp - 2];
    return c->K_s * c->K_s;
}

int make_plan(const Cells *c, const int32_t *tok, int32_t ntok, Plan *pl) {
    const int n_by = (int)c->by.size();
    std::vector<int> cur;
    std::vector<bool> used(2 + n_by + 1, false);
    auto flush = [&]() -> int {
        if (!cur.empty()) pl->levels.push_back(cur);
        cur.clear();
        return ABX_OK;
    };
    for (int i = 0; i < ntok; ++i) {
        if (tok[i] < 0) {
            flush();
            continue;
        }
        int comp = -1;
        for (int b = 0; b < n_by; ++b)
            if (c->by[b] == tok[i]) comp = 2 + b;
        if (c->across >= 0 && tok[i] == c->across) comp = 2 + n_by;
        REQUIRE(comp >= 0, ABX_E_INVALID, "level attribute %d is neither by nor across", tok[i]);
        REQUIRE(!used[comp], ABX_E_INVALID, "level attribute %d collapsed twice", tok[i]);
        used[comp] = true;
        cur.push_back(comp);
    }
    flush();
    const int ncomp = 2 + n_by + (c->across >= 0 ? 1 : 0);
    for (int comp = 2; comp < ncomp; ++comp)
        if (!used[comp]) pl->leftover.push_back(comp);
    auto add = [&](std::vector<CollapseDigit> &v, int comp) {
        const int32_t r = comp_radix(c, comp);
        v.push_back(CollapseDigit{comp, r, make_fastdiv((uint32_t)r)});
    };
    add(pl->seg, 0);
    add(pl->seg, 1);
    for (int comp : pl->leftover) add(pl->seg, comp);
    const int L = (int)pl->levels.size();
    for (int lv = L - 1; lv >= 1; --lv)
        for (int comp : pl->levels[lv]) add(pl->seg, comp);
    if (L >= 1)
        for (int comp : pl->levels[0]) add(pl->loop, comp);
    for (int lv = 1; lv < L; ++lv) {
        int64_t r = 1;
        for (int comp : pl->levels[lv]) r *= comp_radix(c, comp);
        pl->level_radix.push_back(r);
    }
    REQUIRE((int)pl->seg.size() <= kMaxDims && (int)pl->loop.size() <= kMaxDims,
            ABX_E_UNSUPPORTED, "too many collapse attributes");
    for (auto &d : pl->seg) {
        pl->n_seg *= d.radix;
        REQUIRE(pl->n_seg <= (1LL << 28), ABX_E_UNSUPPORTED,
                "collapse key space exceeds 2^28 entries");
    }
    for (auto &d : pl->loop) {
        pl->loop_len *= d.radix;
        REQUIRE(pl->loop_len <= (1LL << 32), ABX_E_UNSUPPORTED, "level-1 loop too long");
    }
    make_bits(c, pl);
    return ABX_OK;
}

struct ScoreRun {
    uint8_t *bits = nullptr;
    int32_t *seg_n = nullptr;
    int64_t *seg_base = nullptr, *n_cells = nullptr, *cell_num2 = nullptr, *cell_cnt = nullptr;
    int2 *cell_id = nullptr;
    int64_t *big = nullptr, *big_count = nullptr;
    double *res = nullptr;
    int32_t *res_n = nullptr;
    unsigned long long *acc = nullptr;
    int32_t *rc_idx = nullptr, *rc_count = nullptr;
    int2 *rc_list = nullptr;
    double *rc_exact = nullptr;
    float2 *rc_iv = nullptr;
    int32_t *rc_state = nullptr, *rc64_list = nullptr, *rc64_count = nullptr;
    int32_t *rc_block_n = nullptr;
    float *rc_invq = nullptr, *rc_theta = nullptr;
    float *rc_fd = nullptr, *rc_dev = nullptr;
    int64_t *rc_fdoff = nullptr;
    unsigned long long *rc_fdused = nullptr;
    int64_t rc_fdcap = 0;
    const Items *items = nullptr;
    cudaStream_t s = nullptr;
    void release() {
        for (void *p : {(void *)bits, (void *)res, (void *)res_n, (void *)acc, (void *)rc_idx,
                        (void *)rc_count, (void *)rc_list, (void *)rc_exact, (void *)seg_n,
                        (void *)seg_base, (void *)n_cells, (void *)cell_num2, (void *)cell_cnt,
                        (void *)cell_id, (void *)big, (void *)big_count, (void *)rc_iv,
                        (void *)rc_state, (void *)rc64_list, (void *)rc64_count,
                        (void *)rc_block_n, (void *)rc_invq, (void *)rc_theta, (void *)rc_fd,
                        (void *)rc_dev, (void *)rc_fdoff, (void *)rc_fdused})
            if (p) cudaFreeAsync(p, s);
        rc_invq = rc_theta = rc_fd = rc_dev = nullptr;
        rc_fdoff = nullptr;
        rc_fdused = nullptr;
        rc_iv = nullptr;
        rc_state = rc64_list = rc64_count = rc_block_n = nullptr;
        seg_n = nullptr;
        seg_base = n_cells = cell_num2 = cell_cnt = nullptr;
        cell_id = nullptr;
        big = big_count = nullptr;
        bits = nullptr;
        res = nullptr;
        res_n = nullptr;
        acc = nullptr;
        rc_idx = rc_count = nullptr;
        rc_list = nullptr;
        rc_exact = nullptr;
    }
    ~ScoreRun() { release(); }
};

ScoreArgs base_args(const PairVal *pv, const Cells *c, const Plan &pl, int recheck) {
    ScoreArgs a;
    memset(&a, 0, sizeof(a));
    a.t = c->dev();
    a.pv = pv;
    a.recheck = recheck;
    a.dirty_slot = 7;
    a.gtab = c->d_gtab;
    a.n_by = (int)c->by.size();
    for (int b = 0; b < a.n_by; ++b) a.by_radix[b] = c->K_by[b];
    a.n_seg_digits = (int)pl.seg.size();
    a.n_loop_digits = (int)pl.loop.size();
    for (size_t i = 0; i < pl.seg.size(); ++i) a.seg[i] = pl.seg[i];
    for (size_t i = 0; i < pl.loop.size(); ++i) a.loop[i] = pl.loop[i];
    a.n_seg = pl.n_seg;
    a.loop_len = pl.loop_len;
    a.key_width = 4 + a.n_by;
    a.sub_cap = c->sub_cap;
    a.sub_xmax = c->sub_xmax;
    a.sub_seed = c->sub_seed;
    a.ks_div = make_fastdiv((uint32_t)std::max(c->K_s, 1));
    return a;
}

int alloc_recheck(ScoreRun &run, ScoreArgs &a, int64_t dm, int64_t cap, int32_t mode,
                  const Items *it, cudaStream_t s);
int reset_recheck(ScoreRun &run, int64_t dm, int32_t cap, cudaStream_t s);

// Shared prefix of abx_score / abx_score_cells: bitsets, counters and (with
// recheck) the exact-value bookkeeping.
int prepare(Dist *d, const Cells *c, const Plan &pl, int recheck, cudaStream_t s, ScoreRun &run,
            ScoreArgs &a) {
    run.s = s;
    a = base_args(d->d_pv, c, pl, recheck);
    CU(cudaStreamWaitEvent(s, d->done, 0));
    if (pl.has_bits) {
        int rc = upload_bits(c, pl, s, (uint32_t **)&run.bits);
        if (rc) return rc;
        a.bits = reinterpret_cast<const uint32_t *>(run.bits);
        a.bits_words = pl.words;
        a.n_rest = (int32_t)pl.rest_by.size();
        for (size_t i = 0; i < pl.rest_by.size(); ++i) a.rest_by[i] = pl.rest_by[i];
        a.rest_radix = pl.rest_radix;
    }
    CU(cudaMallocAsync((void **)&run.acc, kAccN * sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(run.acc, 0, kAccN * sizeof(unsigned long long), s));
    a.acc = run.acc;
    if (recheck) {
        const int64_t dm = std::max<int64_t>(c->dm_entries, 1);
        const int64_t cap = std::max<int64_t>(d->pair_cap, 1);
        int rc = alloc_recheck(run, a, dm, cap, d->mode, d->items, s);
        if (rc) return rc;
        rc = reset_recheck(run, dm, a.rc_capacity, s);
        if (rc) return rc;
    }
    return ABX_OK;
}

// Recheck state of one scoring run: the pair -> slot index, the slot list and
// its FP64 values, and (DTW, interval rule) the refined intervals and the
// FP64 sub-list.  a.recheck must be set.
int alloc_recheck(ScoreRun &run, ScoreArgs &a, int64_t dm, int64_t cap, int32_t mode,
                  const Items *it, cudaStream_t s) {
    REQUIRE(cap < (1LL << 31), ABX_E_UNSUPPORTED, "too many pairs for the recheck list");
    CU(cudaMallocAsync((void **)&run.rc_idx, dm * sizeof(int32_t), s));
    CU(cudaMallocAsync((void **)&run.rc_block_n, compact_blocks(dm) * sizeof(int32_t), s));
    CU(cudaMallocAsync((void **)&run.rc_count, sizeof(int32_t), s));
    CU(cudaMallocAsync((void **)&run.rc_list, cap * sizeof(int2), s));
    CU(cudaMallocAsync((void **)&run.rc_exact, cap * sizeof(double), s));
    a.rc_idx = run.rc_idx;
    a.rc_dm = dm;
    a.rc_block_n = run.rc_block_n;
    a.rc_count = run.rc_count;
    a.rc_list = run.rc_list;
    a.rc_capacity = (int32_t)cap;
    a.rc_exact = run.rc_exact;
    // the refined stage serves the interval rule in DTW mode; the stated
    // margin rule re-decides its triples from FP64 values directly
    if (mode == ABX_DTW && a.recheck == ABX_RECHECK_INTERVAL) {
        CU(cudaMallocAsync((void **)&run.rc_iv, cap * sizeof(float2), s));
        CU(cudaMallocAsync((void **)&run.rc_state, cap * sizeof(int32_t), s));
        CU(cudaMallocAsync((void **)&run.rc64_list, cap * sizeof(int32_t), s));
        CU(cudaMallocAsync((void **)&run.rc64_count, sizeof(int32_t), s));
        a.rc_iv = run.rc_iv;
        a.rc_state = run.rc_state;
        a.rc64_list = run.rc64_list;
        a.rc64_count = run.rc64_count;
        CU(cudaMallocAsync((void **)&run.rc_invq,
                           std::max<int64_t>(it->n_frames, 1) * sizeof(float), s));
        CU(cudaMallocAsync((void **)&run.rc_theta,
                           std::max<int64_t>(it->n_frames, 1) * sizeof(float), s));
        // frame distances of the refined pairs: at most 2^28 floats; pairs
        // past the end are left to the FP64 stage (ABX_REFINE_FD_KB caps the
        // buffer further, so that tests can reach that path)
        const int64_t ml = it->max_len;
        run.rc_fdcap = std::min<int64_t>(1LL << 28, cap * ml * ml);
        if (const char *e = getenv("ABX_REFINE_FD_KB"))
            run.rc_fdcap = std::max<int64_t>(
                1, std::min<int64_t>(run.rc_fdcap, atoll(e) * 1024 / (int64_t)sizeof(float)));
        CU(cudaMallocAsync((void **)&run.rc_fd, run.rc_fdcap * sizeof(float), s));
        CU(cudaMallocAsync((void **)&run.rc_fdoff, cap * sizeof(int64_t), s));
        CU(cudaMallocAsync((void **)&run.rc_dev, cap * sizeof(float), s));
        CU(cudaMallocAsync((void **)&run.rc_fdused, sizeof(unsigned long long), s));
        run.items = it;
    }
    return ABX_OK;
}

int reset_recheck(ScoreRun &run, int64_t dm, int32_t cap, cudaStream_t s) {
    CU(cudaMemsetAsync(run.rc_idx, 0xFF, dm * sizeof(int32_t), s));
    CU(cudaMemsetAsync(run.rc_count, 0, sizeof(int32_t), s));
    if (run.rc_state) {
        CU(cudaMemsetAsync(run.rc_state, 0, (size_t)cap * sizeof(int32_t), s));
        CU(cudaMemsetAsync(run.rc64_count, 0, sizeof(int32_t), s));
    }
    return ABX_OK;
}

// The recheck between a stage-0 evaluation (which marked both pairs of
// every triple the stored values left undecided) and the final one.  DTW
// with the interval rule: the marked pairs are recomputed (TF32 tensor
// cores) with intervals, a stage-1 evaluation lists the pairs of the
// triples those intervals do not separate, and only these are recomputed in
// FP64.  Mean mode and the stated margin rule: every marked pair in FP64.  With `scoring`, each evaluation after the first runs only if the
// previous one met deferred triples (acc[7], then acc[8]) and starts from
// cleared sums; eval(a) runs one evaluation.  On return `a` is set up for
// the final evaluation (stage 2), which the caller runs.
template <class Eval>
int recheck_stages(const RecheckArgs &ra0, const ScoreRun &run, ScoreArgs &a, bool scoring,
                   Eval eval, cudaStream_t s) {
    RecheckArgs ra = ra0;
    int gate = 7;
    {
        CompactArgs ca;
        ca.t = a.t;
        ca.rc_idx = a.rc_idx;
        ca.dm = a.rc_dm;
        ca.rc_list = a.rc_list;
        ca.rc_count = a.rc_count;
        ca.capacity = a.rc_capacity;
        ca.block_n = a.rc_block_n;
        ca.acc = a.acc;
        ca.gate = 7;
        CU(launch_recheck_compact(ca, s));
    }
    if (a.rc_iv) {
        RefinePrepArgs pa;
        pa.feats = ra0.feats;
        pa.offsets = ra0.offsets;
        pa.n_items = run.items->n_items;
        pa.n_frames = run.items->n_frames;
        pa.dim = ra0.dim;
        pa.inv_q = run.rc_invq;
        pa.theta_frame = run.rc_theta;
        pa.acc = a.acc;
        pa.gate = 7;
        CU(launch_refine_prep(pa, s));
        RefineArgs rf;
        memset(&rf, 0, sizeof(rf));
        rf.fd = run.rc_fd;
        rf.fd_cap = run.rc_fdcap;
        rf.fd_off = run.rc_fdoff;
        rf.dev = run.rc_dev;
        rf.fd_used = run.rc_fdused;
        rf.feats = ra0.feats;
        rf.offsets = ra0.offsets;
        rf.item_id = ra0.item_id;
        rf.dim = ra0.dim;
        rf.max_len = ra0.max_len;
        rf.list = ra0.list;
        rf.count = ra0.count;
        rf.capacity = ra0.capacity;
        rf.iv = run.rc_iv;
        rf.inv_q = run.rc_invq;
        rf.theta_frame = run.rc_theta;
        rf.eps_c = refine_cosine_bound(ra0.dim);
        CU(launch_refine(rf, a.rc_capacity, s));
        if (scoring) CU(launch_reset_if_dirty(run.acc, 7, s));
        a.stage = 1;
        a.gate = scoring ? 7 : 0;
        a.dirty_slot = 8;
        int rc = eval(a);
        if (rc) return rc;
        ra.slots = run.rc64_list;
        ra.count = run.rc64_count;
        gate = 8;
    }
    CU(launch_recheck(ra, a.rc_capacity, s));
    if (scoring) CU(launch_reset_if_dirty(run.acc, gate, s));
    a.stage = 2;
    a.gate = scoring ? gate : 0;
    a.dirty_slot = 9;  // nothing is deferred at stage 2
    return ABX_OK;
}

RecheckArgs recheck_args(const Dist *d, const Cells *c, const ScoreRun &run, int32_t cap) {
    RecheckArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.feats = d->items->d_feats;
    ra.offsets = d->items->d_offsets;
    ra.item_id = c->d_item_id;
    ra.dim = d->items->dim;
    ra.mode = d->mode;
    ra.max_len = d->items->max_len;
    ra.list = run.rc_list;
    ra.count = run.rc_count;
    ra.capacity = cap;
    ra.exact = run.rc_exact;
    ra.slots = nullptr;
    return ra;
}

// Bitset path: count candidates per segment, scan, enumerate and evaluate
// every cell; with recheck, further evaluations run only if some triple was
// undecidable from the intervals (recheck_stages).
template <class Eval>
int recheck_stages(const RecheckArgs &ra0, const ScoreRun &run, ScoreArgs &a, bool scoring,
                   Eval eval, cudaStream_t s);
RecheckArgs recheck_args(const Dist *d, const Cells *c, const ScoreRun &run, int32_t cap);

int eval_cells(Dist *d, const Cells *c, const Plan &pl, int recheck, cudaStream_t s,
               ScoreRun &run, ScoreArgs &a) {
    CU(cudaMallocAsync((void **)&run.seg_n, pl.n_seg * sizeof(int32_t), s));
    CU(cudaMallocAsync((void **)&run.seg_base, (pl.n_seg + 1) * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.n_cells, 2 * sizeof(int64_t), s));
    CU(cudaMemsetAsync(run.n_cells, 0, 2 * sizeof(int64_t), s));
    a.seg_n = run.seg_n;
    a.seg_base = run.seg_base;
    a.n_cells_dev = run.n_cells;
    CU(launch_seg_count(a, s));
    CU(launch_scan_i32_to_i64(run.seg_n, run.seg_base, pl.n_seg, run.n_cells, run.n_cells + 1, s));
    // the cell arrays are sized by the candidate count of abx_build_cells (no
    // read-back); the enumeration stores only within it, and the device total
    // is checked against it with the results
    const int64_t cap = std::max<int64_t>(c->n_cand, 1);
    CU(cudaMallocAsync((void **)&run.cell_id, cap * sizeof(int2), s));
    CU(cudaMallocAsync((void **)&run.cell_num2, cap * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.cell_cnt, cap * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.big, cap * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.big_count, sizeof(int64_t), s));
    a.big = run.big;
    a.big_count = run.big_count;
    a.cell_id = run.cell_id;
    a.cell_cap = c->n_cand;
    a.cell_num2 = run.cell_num2;
    a.cell_cnt = run.cell_cnt;
    CU(launch_cell_enum(a, s));
    a.stage = 0;
    a.gate = 0;
    a.dirty_slot = 7;
    CU(launch_cell_eval(a, s));
    if (recheck) {
        // device-driven: the recheck kernels read how many pairs were marked
        // (none: they return at once); the later evaluations run only if some
        // triple was deferred
        auto eval = [&](ScoreArgs &x) -> int {
            CU(launch_cell_eval(x, s));
            return ABX_OK;
        };
        int rc = recheck_stages(recheck_args(d, c, run, a.rc_capacity), run, a, true, eval, s);
        if (rc) return rc;
        CU(launch_cell_eval(a, s));
        a.gate = 0;
    }
    return ABX_OK;
}

}  // namespace

namespace abx {

// Score plan for a group-structured task (a batch of tasks joined by a
// leading group attribute): every buffer sized on the host, execution
// without host synchronisation, per-group results.
struct ScorePlanB {
    Plan pl;
    ScoreRun run;
    ScoreArgs a;
    RecheckArgs ra;
    int recheck = 0, weighted = 0;
    int64_t cells = 0, n_outer = 0, inner = 1, seg_div = 1, dm = 1;
    int32_t n_group = 0;
    std::vector<std::pair<double *, int32_t *>> lv;  // level outputs
    std::vector<int64_t> lv_n;
    double *gmean = nullptr;
    int64_t *gn = nullptr;
    unsigned long long *gnum2 = nullptr, *gcnt = nullptr;
    // pinned result mirror
    void *mirror = nullptr;
    Ctx *ctx = nullptr;
    cudaStream_t s = nullptr;
};

int score_plan_b_build(Ctx *ctx, const Cells *c, const Items *it, const DistPlan &dp,
                       const int32_t *levels, int32_t n_tok, int32_t weighted, int32_t recheck,
                       float margin, cudaStream_t s, ScorePlanB **out) {
    *out = nullptr;
    REQUIRE(recheck >= ABX_RECHECK_OFF && recheck <= ABX_RECHECK_MARGIN, ABX_E_INVALID,
            "bad recheck mode %d", recheck);
    REQUIRE(!c->by.empty(), ABX_E_INVALID, "group attribute missing");
    std::unique_ptr<ScorePlanB> P(new (std::nothrow) ScorePlanB);
    REQUIRE(P, ABX_E_OOM, "host allocation failed");
    ScorePlanB &b = *P;
    b.ctx = ctx;
    b.s = s;
    b.recheck = recheck;
    b.weighted = weighted;
    int rc = make_plan(c, levels, n_tok, &b.pl);
    if (rc) return rc;
    const Plan &pl = b.pl;
    REQUIRE(pl.has_bits, ABX_E_UNSUPPORTED,
            "batched scoring needs level-1 attributes among the by attributes");
    REQUIRE(!pl.leftover.empty() && pl.leftover[0] == 2 && pl.seg.size() >= 3 &&
                pl.seg[2].comp == 2,
            ABX_E_INVALID, "the group attribute must be the first by attribute, not collapsed");
    b.n_group = c->K_by[0];
    for (size_t d = 3; d < pl.seg.size(); ++d) b.seg_div *= pl.seg[d].radix;
    b.n_outer = (int64_t)c->K_on * c->K_on;
    for (size_t i = 1; i < pl.leftover.size(); ++i) b.inner *= comp_radix(c, pl.leftover[i]);

    // buffers (stream-ordered)
    ScoreRun &run = b.run;
    run.s = s;
    ScoreArgs &a = b.a;
    a = base_args(dp.pv, c, pl, recheck);
    a.margin = margin;
    {
        if ((rc = upload_bits(c, pl, s, (uint32_t **)&run.bits))) return rc;
        a.bits = reinterpret_cast<const uint32_t *>(run.bits);
        a.bits_words = pl.words;
        a.n_rest = (int32_t)pl.rest_by.size();
        for (size_t i = 0; i < pl.rest_by.size(); ++i) a.rest_by[i] = pl.rest_by[i];
        a.rest_radix = pl.rest_radix;
    }
    CU(cudaMallocAsync((void **)&run.acc, kAccN * sizeof(unsigned long long), s));
    a.acc = run.acc;
    if (recheck) {
        const int64_t dm = std::max<int64_t>(c->dm_entries, 1);
        b.dm = dm;
        const int64_t cap = std::max<int64_t>(dp.cap_total, 1);
        if ((rc = alloc_recheck(run, a, dm, cap, dp.mode, it, s))) return rc;
        RecheckArgs &r = b.ra;
        memset(&r, 0, sizeof(r));
        r.feats = it->d_feats;
        r.offsets = it->d_offsets;
        r.item_id = c->d_item_id;
        r.dim = it->dim;
        r.mode = dp.mode;
        r.max_len = it->max_len;
        r.list = run.rc_list;
        r.count = run.rc_count;
        r.capacity = a.rc_capacity;
        r.exact = run.rc_exact;
    }
    CU(cudaMallocAsync((void **)&run.res, pl.n_seg * sizeof(double), s));
    CU(cudaMallocAsync((void **)&run.res_n, pl.n_seg * sizeof(int32_t), s));
    a.res = run.res;
    a.res_n = run.res_n;
    CU(cudaMallocAsync((void **)&run.seg_n, pl.n_seg * sizeof(int32_t), s));
    CU(cudaMallocAsync((void **)&run.seg_base, (pl.n_seg + 1) * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.n_cells, 2 * sizeof(int64_t), s));
    a.seg_n = run.seg_n;
    a.seg_base = run.seg_base;
    a.n_cells_dev = run.n_cells;
    // number of materialised cells: the candidate count of abx_build_cells
    // (each run counts again on the device and the read-back compares)
    b.cells = c->n_cand;
    const int64_t cap = std::max<int64_t>(b.cells, 1);
    CU(cudaMallocAsync((void **)&run.cell_id, cap * sizeof(int2), s));
    CU(cudaMallocAsync((void **)&run.cell_num2, cap * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.cell_cnt, cap * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.big, cap * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&run.big_count, sizeof(int64_t), s));
    a.big = run.big;
    a.big_count = run.big_count;
    a.cell_id = run.cell_id;
    a.cell_cap = b.cells;
    a.cell_num2 = run.cell_num2;
    a.cell_cnt = run.cell_cnt;
    int64_t n_cur = pl.n_seg;
    for (int64_t radix : pl.level_radix) {
        const int64_t n_out = n_cur / radix;
        double *o = nullptr;
        int32_t *on = nullptr;
        CU(cudaMallocAsync((void **)&o, std::max<int64_t>(n_out, 1) * sizeof(double), s));
        CU(cudaMallocAsync((void **)&on, std::max<int64_t>(n_out, 1) * sizeof(int32_t), s));
        b.lv.push_back({o, on});
        b.lv_n.push_back(n_out);
        n_cur = n_out;
    }
    REQUIRE(n_cur == b.n_outer * b.n_group * b.inner, ABX_E_STATE, "collapse layout mismatch");
    const int32_t G = std::max(b.n_group, 1);
    CU(cudaMallocAsync((void **)&b.gmean, G * sizeof(double), s));
    CU(cudaMallocAsync((void **)&b.gn, G * sizeof(int64_t), s));
    CU(cudaMallocAsync((void **)&b.gnum2, G * sizeof(unsigned long long), s));
    CU(cudaMallocAsync((void **)&b.gcnt, G * sizeof(unsigned long long), s));
    b.mirror = ctx->pinned.acquire(64 + (size_t)G * 32 + 16);
    REQUIRE(b.mirror, ABX_E_OOM, "pinned host allocation failed");
    *out = P.release();
    return ABX_OK;
}

int score_plan_b_exec(ScorePlanB *pb, cudaStream_t s) {
    ScorePlanB &b = *pb;
    ScoreArgs a = b.a;
    ScoreRun &run = b.run;
    const Plan &pl = b.pl;
    const int32_t G = std::max(b.n_group, 1);
    CU(cudaMemsetAsync(run.acc, 0, kAccN * sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(run.n_cells, 0, 2 * sizeof(int64_t), s));
    CU(cudaMemsetAsync(b.gnum2, 0, G * sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(b.gcnt, 0, G * sizeof(unsigned long long), s));
    if (b.recheck) {
        int rc = reset_recheck(run, b.dm, a.rc_capacity, s);
        if (rc) return rc;
    }
    // materialised cells: counts, offsets, enumeration (capacity known)
    CU(launch_seg_count(a, s));
    CU(launch_scan_i32_to_i64(run.seg_n, run.seg_base, pl.n_seg, run.n_cells, run.n_cells + 1, s));
    CU(launch_cell_enum(a, s));
    a.stage = 0;
    a.gate = 0;
    a.dirty_slot = 7;
    CU(launch_cell_eval(a, s));
    if (b.recheck) {
        auto eval = [&](ScoreArgs &x) -> int {
            CU(launch_cell_eval(x, s));
            return ABX_OK;
        };
        int rc = recheck_stages(b.ra, run, a, true, eval, s);
        if (rc) return rc;
        CU(launch_cell_eval(a, s));
        a.gate = 0;
    }
    CU(launch_seg_reduce(a, s));
    const double *cur = run.res;
    const int32_t *cur_n = run.res_n;
    for (size_t i = 0; i < b.lv.size(); ++i) {
        CU(launch_collapse_level(cur, cur_n, b.lv_n[i], pl.level_radix[i], b.lv[i].first,
                                 b.lv[i].second, s));
        cur = b.lv[i].first;
        cur_n = b.lv[i].second;
    }
    CU(launch_final_group(cur, cur_n, b.n_outer, b.n_group, b.inner, b.gmean, b.gn, s));
    CU(launch_cell_group_sums(a, b.seg_div, b.n_group, b.gnum2, b.gcnt, s));
    // results to the pinned mirror: acc[0..7], n_cells, rc_count, rc64_count,
    // then per group
    uint8_t *m = (uint8_t *)b.mirror;
    CU(cudaMemcpyAsync(m, run.acc, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(m + 64, run.n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (b.recheck) {
        CU(cudaMemcpyAsync(m + 72, run.rc_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(m + 76, run.rc64_count ? run.rc64_count : run.rc_count,
                           sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    uint8_t *g = m + 80;
    CU(cudaMemcpyAsync(g, b.gmean, G * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(g + G * 8, b.gn, G * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(g + G * 16, b.gnum2, G * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(g + G * 24, b.gcnt, G * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    return ABX_OK;
}

// After the stream has passed score_plan_b_exec: per-group errors (NaN for a
// group without cells) and triple counts; totals into stats.
int score_plan_b_read(const ScorePlanB *pb, double *errors, int64_t *triplets,
                      abx_score_stats *stats) {
    const ScorePlanB &b = *pb;
    const int32_t G = std::max(b.n_group, 1);
    const uint8_t *m = (const uint8_t *)b.mirror;
    const unsigned long long *acc = (const unsigned long long *)m;
    const int64_t n_cells = *(const int64_t *)(m + 64);
    const int32_t rc = b.recheck ? *(const int32_t *)(m + 72) : 0;
    const int32_t rc64 = b.recheck ? *(const int32_t *)(m + 76) : 0;
    REQUIRE(n_cells == b.cells, ABX_E_STATE, "cell count %lld differs from the plan's %lld",
            (long long)n_cells, (long long)b.cells);
    REQUIRE(acc[6] == 0, ABX_E_INVALID, "recheck list overflow");
    const uint8_t *g = m + 80;
    const double *gmean = (const double *)g;
    const int64_t *gn = (const int64_t *)(g + G * 8);
    const unsigned long long *gnum2 = (const unsigned long long *)(g + G * 16);
    const unsigned long long *gcnt = (const unsigned long long *)(g + G * 24);
    for (int32_t k = 0; k < b.n_group; ++k) {
        if (b.weighted)
            errors[k] = gcnt[k] ? 1.0 - (double)gnum2[k] / (2.0 * (double)gcnt[k]) : std::nan("");
        else
            errors[k] = gn[k] ? 1.0 - gmean[k] : std::nan("");
        if (triplets) triplets[k] = (int64_t)gcnt[k];
    }
    if (stats) {
        stats->n_cells = (int64_t)acc[2];
        stats->n_triplets = (int64_t)acc[3];
        stats->n_undecided = (int64_t)acc[4];
        stats->n_recheck_pairs = rc;
        stats->n_flips = (int64_t)acc[5];
        stats->num2_total = (int64_t)acc[0];
        stats->count2_total = (int64_t)acc[1];
        stats->n_exact_pairs = rc64;
    }
    return ABX_OK;
}

void score_plan_b_free(ScorePlanB *pb, cudaStream_t s) {
    if (!pb) return;
    pb->run.s = s;
    pb->run.release();
    for (auto &l : pb->lv) {
        cudaFreeAsync(l.first, s);
        cudaFreeAsync(l.second, s);
    }
    for (void *p : {(void *)pb->gmean, (void *)pb->gn, (void *)pb->gnum2, (void *)pb->gcnt})
        if (p) cudaFreeAsync(p, s);
    if (pb->mirror) pb->ctx->pinned.release(pb->mirror, s);
    delete pb;
}

}  // namespace abx

namespace {

// An enqueued abx_score: the pinned result mirror and the event after the
// last copy into it.  The mirror layout: [0] final mean (double), [8] entries
// averaged (int64), [16] counters acc[0..7], [80] rechecked pairs (int32),
// [84] pairs recomputed in FP64 (int32), [88] device cell total (int64).
struct ScoreJob {
    static constexpr size_t kMirror = 96;
    Ctx *ctx = nullptr;
    Dist *d = nullptr;
    const Cells *c = nullptr;
    cudaStream_t s = nullptr;
    int32_t weighted = 0;
    bool materialised = false;  // cells enumerated; their count is checked
    int64_t n_cand = 0;
    void *mirror = nullptr;
    cudaEvent_t done = nullptr;
    ~ScoreJob() {
        if (done) cudaEventDestroy(done);
        if (mirror) ctx->pinned.release(mirror, s);
    }
};

}  // namespace

extern "C" {

int abx_score(abx_ctx *ctx_, abx_dist *dist_, const abx_cells *cells_, const int32_t *levels,
              int32_t n_level_tokens, int32_t weighted, int32_t recheck, void *stream,
              double *error_out, abx_score_stats *stats) {
    return abx_score_ex(ctx_, dist_, cells_, levels, n_level_tokens, weighted,
                        recheck ? ABX_RECHECK_INTERVAL : ABX_RECHECK_OFF, 0.0f, stream,
                        error_out, stats);
}

int abx_score_ex(abx_ctx *ctx_, abx_dist *dist_, const abx_cells *cells_, const int32_t *levels,
                 int32_t n_level_tokens, int32_t weighted, int32_t recheck, float margin,
                 void *stream, double *error_out, abx_score_stats *stats) {
    REQUIRE(error_out, ABX_E_INVALID, "NULL argument");
    abx_score_job *job = nullptr;
    int rc = abx_score_submit(ctx_, dist_, cells_, levels, n_level_tokens, weighted, recheck,
                              margin, stream, &job);
    if (rc) return rc;
    return abx_score_wait(job, error_out, stats);
}

int abx_score_submit(abx_ctx *ctx_, abx_dist *dist_, const abx_cells *cells_,
                     const int32_t *levels, int32_t n_level_tokens, int32_t weighted,
                     int32_t recheck, float margin, void *stream, abx_score_job **out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    Dist *d = reinterpret_cast<Dist *>(dist_);
    const Cells *c = reinterpret_cast<const Cells *>(cells_);
    REQUIRE(ctx && d && c && out, ABX_E_INVALID, "NULL argument");
    *out = nullptr;
    REQUIRE(d->ctx == ctx && c->ctx == ctx && d->cells == c, ABX_E_STATE,
            "distances were computed for another task");
    REQUIRE(n_level_tokens >= 0 && (n_level_tokens == 0 || levels), ABX_E_INVALID, "bad levels");
    REQUIRE(recheck >= ABX_RECHECK_OFF && recheck <= ABX_RECHECK_MARGIN, ABX_E_INVALID,
            "bad recheck mode %d", recheck);
    REQUIRE(recheck != ABX_RECHECK_MARGIN || margin >= 0.0f, ABX_E_INVALID, "negative margin");
    REQUIRE(!recheck || d->distance == ABX_DIST_ANGULAR, ABX_E_UNSUPPORTED,
            "the FP64 recheck is defined for the angular distance only");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    Trace tr("score");
    Plan pl;
    int rc = make_plan(c, levels, n_level_tokens, &pl);
    if (rc) return rc;
    tr.mark("plan+bits");
    std::unique_ptr<ScoreJob> job(new (std::nothrow) ScoreJob);
    REQUIRE(job, ABX_E_OOM, "host allocation failed");
    job->ctx = ctx;
    job->d = d;
    job->c = c;
    job->s = s;
    job->weighted = weighted;
    job->n_cand = c->n_cand;
    ScoreRun run;
    ScoreArgs a;
    if ((rc = prepare(d, c, pl, recheck, s, run, a))) return rc;
    tr.mark("prepare");
    a.margin = margin;
    CU(cudaMallocAsync((void **)&run.res, pl.n_seg * sizeof(double), s));
    CU(cudaMallocAsync((void **)&run.res_n, pl.n_seg * sizeof(int32_t), s));
    a.res = run.res;
    a.res_n = run.res_n;
    REQUIRE(a.bits || (c->sub_cap == 0 && c->sub_xmax == 0), ABX_E_UNSUPPORTED,
            "the subsampler needs level-1 attributes among the by attributes");
    if (a.bits) {
        if ((rc = eval_cells(d, c, pl, recheck, s, run, a))) return rc;
        job->materialised = true;
        CU(launch_seg_reduce(a, s));
    } else {
        a.pass = 1;
        a.stage = 0;
        a.gate = 0;
        a.dirty_slot = 7;
        CU(launch_score(a, s));
        if (recheck) {
            // later passes run only if some triple was not decidable from
            // the stored values; those pairs are now marked (device-driven)
            auto eval = [&](ScoreArgs &x) -> int {
                CU(launch_score(x, s));
                return ABX_OK;
            };
            if ((rc = recheck_stages(recheck_args(d, c, run, a.rc_capacity), run, a, true, eval,
                                     s)))
                return rc;
            CU(launch_score(a, s));
            a.gate = 0;
        }
    }
    tr.mark("cells enqueued");
    // further levels: each folds its own digits, innermost first
    double *cur = run.res;
    int32_t *cur_n = run.res_n;
    int64_t n_cur = pl.n_seg;
    std::vector<void *> tmp;
    for (int64_t radix : pl.level_radix) {
        int64_t n_out = n_cur / radix;
        double *o = nullptr;
        int32_t *on = nullptr;
        CU(cudaMallocAsync((void **)&o, std::max<int64_t>(n_out, 1) * sizeof(double), s));
        CU(cudaMallocAsync((void **)&on, std::max<int64_t>(n_out, 1) * sizeof(int32_t), s));
        tmp.push_back(o);
        tmp.push_back(on);
        CU(launch_collapse_level(cur, cur_n, n_out, radix, o, on, s));
        cur = o;
        cur_n = on;
        n_cur = n_out;
    }
    double *fin = nullptr;
    int64_t *fin_n = nullptr;
    CU(cudaMallocAsync((void **)&fin, sizeof(double), s));
    CU(cudaMallocAsync((void **)&fin_n, sizeof(int64_t), s));
    tmp.push_back(fin);
    tmp.push_back(fin_n);
    CU(launch_final_mean(cur, cur_n, n_cur, fin, fin_n, s));
    // results into a pinned mirror (ScoreJob::kMirror), read by abx_score_wait
    uint8_t *m = (uint8_t *)ctx->pinned.acquire(ScoreJob::kMirror);
    REQUIRE(m, ABX_E_OOM, "pinned host allocation failed");
    job->mirror = m;
    memset(m, 0, ScoreJob::kMirror);
    CU(cudaMemcpyAsync(m, fin, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(m + 8, fin_n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(m + 16, run.acc, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    if (recheck) {
        CU(cudaMemcpyAsync(m + 80, run.rc_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(m + 84, run.rc64_count ? run.rc64_count : run.rc_count,
                           sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    if (job->materialised)
        CU(cudaMemcpyAsync(m + 88, run.n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    for (void *p : tmp) cudaFreeAsync(p, s);
    run.release();
    CU(cudaEventCreateWithFlags(&job->done, cudaEventDisableTiming));
    CU(cudaEventRecord(job->done, s));
    tr.mark("levels enqueued");
    ++d->jobs;
    ++const_cast<Cells *>(c)->jobs;
    *out = reinterpret_cast<abx_score_job *>(job.release());
    return ABX_OK;
}

int abx_score_wait(abx_score_job *job_, double *error_out, abx_score_stats *stats) {
    ScoreJob *job = reinterpret_cast<ScoreJob *>(job_);
    REQUIRE(job, ABX_E_INVALID, "NULL argument");
    // the job is freed on every return path below
    std::unique_ptr<ScoreJob> own(job);
    Dist *d = job->d;
    --d->jobs;
    --const_cast<Cells *>(job->c)->jobs;
    CU(cudaSetDevice(job->ctx->device));
    Trace tr("score");
    CU(cudaEventSynchronize(job->done));
    tr.mark("final sync");
    const uint8_t *m = (const uint8_t *)job->mirror;
    const double h_fin = *(const double *)m;
    const int64_t h_fin_n = *(const int64_t *)(m + 8);
    const unsigned long long *h_acc = (const unsigned long long *)(m + 16);
    const int32_t h_rc = *(const int32_t *)(m + 80);
    const int32_t h_rc64 = *(const int32_t *)(m + 84);
    const int64_t h_cells = *(const int64_t *)(m + 88);
    if (!d->synced) {  // the distance counters arrived before d->done
        d->synced = true;
        d->n_pairs = d->h_count[0];
        d->info.n_pairs = d->h_count[0];
        d->info.n_frame_pairs = d->h_count[1];
    }
    REQUIRE(!(d->h_err[0] & kPackNonPositive), ABX_E_INVALID,
            "the KL distance needs every frame component > 0");
    REQUIRE(!(d->h_err[0] & kPackZeroNorm), ABX_E_ZERO_NORM,
            "a frame has zero L2 norm (angle undefined)");
    REQUIRE(d->h_err[1] == 0, ABX_E_CUDA, "tile kernel pipeline wait expired (code %d)",
            d->h_err[1]);
    REQUIRE(!job->materialised || h_cells == job->n_cand, ABX_E_STATE,
            "cell count %lld differs from the candidate count %lld", (long long)h_cells,
            (long long)job->n_cand);
    REQUIRE(h_acc[6] == 0, ABX_E_INVALID, "recheck list overflow");
    if (!error_out) return ABX_OK;
    if (job->weighted)
        *error_out = h_acc[1] ? 1.0 - (double)h_acc[0] / (double)h_acc[1] : std::nan("");
    else
        *error_out = h_fin_n ? 1.0 - h_fin : std::nan("");
    if (stats) {
        stats->n_cells = (int64_t)h_acc[2];
        stats->n_triplets = (int64_t)h_acc[3];
        stats->n_undecided = (int64_t)h_acc[4];
        stats->n_recheck_pairs = h_rc;
        stats->n_flips = (int64_t)h_acc[5];
        stats->num2_total = (int64_t)h_acc[0];
        stats->count2_total = (int64_t)h_acc[1];
        stats->n_exact_pairs = h_rc64;
    }
    return ABX_OK;
}

int abx_score_cells(abx_ctx *ctx_, abx_dist *dist_, const abx_cells *cells_, int32_t recheck,
                    void *stream, int64_t capacity, int32_t *keys, int64_t *num2, int64_t *count,
                    int64_t *n_out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    Dist *d = reinterpret_cast<Dist *>(dist_);
    const Cells *c = reinterpret_cast<const Cells *>(cells_);
    REQUIRE(ctx && d && c && n_out, ABX_E_INVALID, "NULL argument");
    REQUIRE(capacity == 0 || (keys && num2 && count), ABX_E_INVALID, "NULL output buffer");
    REQUIRE(d->ctx == ctx && c->ctx == ctx && d->cells == c, ABX_E_STATE,
            "distances were computed for another task");
    REQUIRE(!recheck || d->distance == ABX_DIST_ANGULAR, ABX_E_UNSUPPORTED,
            "the FP64 recheck is defined for the angular distance only");
    recheck = recheck ? ABX_RECHECK_INTERVAL : ABX_RECHECK_OFF;
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    // one thread per (on_ax, on_b, across pair), looping over all by values
    Plan pl;
    std::vector<int32_t> tok(c->by.begin(), c->by.end());
    int rc = make_plan(c, tok.data(), (int32_t)tok.size(), &pl);
    if (rc) return rc;
    ScoreRun run;
    ScoreArgs a;
    if ((rc = prepare(d, c, pl, recheck, s, run, a))) return rc;
    if (a.bits) {
        if ((rc = eval_cells(d, c, pl, recheck, s, run, a))) return rc;
        const int kw = 4 + (int)c->by.size();
        int64_t total = 0;
        CU(cudaMemcpyAsync(&total, run.n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        int32_t *dk = nullptr;
        CU(cudaMallocAsync((void **)&dk, std::max<int64_t>(a.cell_cap, 1) * kw * sizeof(int32_t), s));
        a.cell_keys = dk;
        a.key_width = kw;
        CU(launch_cell_emit(a, s));
        CU(cudaStreamSynchronize(s));
        REQUIRE(total == c->n_cand, ABX_E_STATE,
                "cell count %lld differs from the candidate count %lld", (long long)total,
                (long long)c->n_cand);
        REQUIRE(!(d->h_err[0] & kPackNonPositive), ABX_E_INVALID,
                "the KL distance needs every frame component > 0");
        REQUIRE(!(d->h_err[0] & kPackZeroNorm), ABX_E_ZERO_NORM,
                "a frame has zero L2 norm (angle undefined)");
        std::vector<int32_t> hk((size_t)std::max<int64_t>(total, 1) * kw);
        std::vector<int64_t> hn(std::max<int64_t>(total, 1)), hc(std::max<int64_t>(total, 1));
        if (total) {
            CU(cudaMemcpy(hk.data(), dk, total * kw * sizeof(int32_t), cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(hn.data(), run.cell_num2, total * sizeof(int64_t), cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(hc.data(), run.cell_cnt, total * sizeof(int64_t), cudaMemcpyDeviceToHost));
        }
        cudaFreeAsync(dk, s);
        int64_t m = 0;
        for (int64_t i = 0; i < total; ++i) {
            if (!hc[i]) continue;
            if (m < capacity) {
                memcpy(keys + m * kw, &hk[i * kw], kw * sizeof(int32_t));
                num2[m] = hn[i];
                count[m] = hc[i];
            }
            ++m;
        }
        *n_out = m;
        REQUIRE(capacity == 0 || capacity >= m, ABX_E_INVALID, "capacity %lld < %lld cells",
                (long long)capacity, (long long)m);
        return ABX_OK;
    }
    if (recheck) {
        a.pass = 0;
        a.stage = 0;
        a.gate = 0;
        a.dirty_slot = 7;
        CU(launch_score(a, s));
        auto eval = [&](ScoreArgs &x) -> int {
            CU(launch_score(x, s));
            return ABX_OK;
        };
        if ((rc = recheck_stages(recheck_args(d, c, run, a.rc_capacity), run, a, false, eval, s)))
            return rc;
    }
    int64_t *cc = nullptr;
    CU(cudaMallocAsync((void **)&cc, pl.n_seg * sizeof(int64_t), s));
    a.cell_count = cc;
    a.pass = 2;
    CU(launch_score(a, s));
    std::vector<int64_t> h(pl.n_seg);
    CU(cudaMemcpyAsync(h.data(), cc, pl.n_seg * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    REQUIRE(!(d->h_err[0] & kPackNonPositive), ABX_E_INVALID,
            "the KL distance needs every frame component > 0");
    REQUIRE(!(d->h_err[0] & kPackZeroNorm), ABX_E_ZERO_NORM,
            "a frame has zero L2 norm (angle undefined)");
    int64_t total = 0;
    for (auto &v : h) {
        int64_t t = v;
        v = total;
        total += t;
    }
    *n_out = total;
    if (capacity >= total && total > 0) {
        const int kw = 4 + (int)c->by.size();
        int32_t *dk = nullptr;
        int64_t *dn = nullptr, *dc = nullptr;
        CU(cudaMemcpyAsync(cc, h.data(), pl.n_seg * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        CU(cudaMallocAsync((void **)&dk, total * kw * sizeof(int32_t), s));
        CU(cudaMallocAsync((void **)&dn, total * sizeof(int64_t), s));
        CU(cudaMallocAsync((void **)&dc, total * sizeof(int64_t), s));
        a.cell_keys = dk;
        a.cell_num2 = dn;
        a.cell_cnt = dc;
        a.pass = 3;
        CU(launch_score(a, s));
        CU(cudaMemcpyAsync(keys, dk, total * kw * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(num2, dn, total * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(count, dc, total * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        cudaFreeAsync(dk, s);
        cudaFreeAsync(dn, s);
        cudaFreeAsync(dc, s);
        CU(cudaStreamSynchronize(s));
    } else if (capacity > 0 && capacity < total) {
        cudaFreeAsync(cc, s);
        set_error("capacity %lld < %lld cells", (long long)capacity, (long long)total);
        return ABX_E_INVALID;
    }
    cudaFreeAsync(cc, s);
    return ABX_OK;
}

}  // extern "C"
