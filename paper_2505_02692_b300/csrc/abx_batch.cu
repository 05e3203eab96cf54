// Batched tasks: many independent ABX tasks (Sec. 3.1 Task / Score per task)
// run in shared launches.
//
// Tasks of one feature dimension are joined into one task whose items carry
// a leading task attribute; the attribute is the first `by` attribute, so
// every group, and hence every cell and every needed item pair, belongs to
// one task, and the collapse keeps it apart (it is never a collapse level;
// the final mean runs per task value in the single-task order).  Each stage
// of the path then runs once per dimension class for all its tasks: packing,
// pair planning, the frame tile kernel over the tiles of every task, one DTW
// launch over every pair, and the scoring kernels.  All buffers are sized at
// creation; a run is memsets and kernels only, captured once into a CUDA graph
// and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "abx_internal.h"

namespace abx {
namespace {

// One task spec (on / by / across / levels) over a class's items.
struct BatchSpec {
    abx_cells *cells = nullptr;
    DistPlan dp;
    ScorePlanB *sp = nullptr;
};

struct BatchClass {
    int32_t dim = 0;
    std::vector<int32_t> tasks;   // batch task indices, in order
    float *feats = nullptr;       // owned: the class's frames, task after task
    abx_items *items = nullptr;
    std::vector<BatchSpec> specs;
};

struct Batch {
    Ctx *ctx = nullptr;
    int32_t n_tasks = 0, n_specs = 1;
    int32_t mode = ABX_DTW, precision = ABX_FP32, recheck = 1, weighted = 0;
    std::vector<BatchClass> cls;
    std::vector<int32_t> task_class, task_pos;
    cudaStream_t s = nullptr;        // creation stream
    cudaStream_t last = nullptr;     // stream of the last run
    bool use_graph = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_kernels = 0;
    void *err_mirror = nullptr;      // pinned, 32 B per (class, spec): 4 int32 flags, 2 int64 counts
    int64_t runs = 0;
};

}  // namespace
}  // namespace abx

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

#define RC(call)               \
    do {                       \
        int rc_ = (call);      \
        if (rc_) return rc_;   \
    } while (0)

namespace {

// One run of a class: distances, then scores, then the error flags.
int exec_class(Batch &b, size_t k, cudaStream_t s) {
    BatchClass &c = b.cls[k];
    for (size_t j = 0; j < c.specs.size(); ++j) {
        BatchSpec &sp = c.specs[j];
        RC(dist_plan_exec(sp.dp, s));
        RC(score_plan_b_exec(sp.sp, s));
        uint8_t *m = (uint8_t *)b.err_mirror + 32 * (k * b.n_specs + j);
        CU(cudaMemcpyAsync(m, sp.dp.d_err, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(m + 16, sp.dp.d_count, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                           s));
    }
    return ABX_OK;
}

// Time the class's distance stage with the given variants (best of 2 after
// one warm-up run), in ms.
int time_variant(Batch &b, DistPlan &dp, int32_t uv, int32_t dv, float *ms) {
    dp.umma_variant = uv;
    dp.dtw_variant = dv;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        CU(cudaEventRecord(e0, b.s));
        RC(dist_plan_exec(dp, b.s));
        CU(cudaEventRecord(e1, b.s));
        CU(cudaEventSynchronize(e1));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, e0, e1));
        if (r > 0) best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return ABX_OK;
}

// Autotuner of the unfused path (items longer than the fused kernel takes):
// DTW variant first (tile kernel at its default), then the tile kernel
// variant with the chosen DTW variant.  Cached per key in the context.
int tune_plan(Batch &b, DistPlan &dp) {
    if (dp.fused) return ABX_OK;  // one fused kernel: nothing to choose
    char key[128];
    // length class rather than the exact longest item: the variants differ in
    // whether 256 DTW row buffers fit, not in the exact length, and jobs of
    // one workload would otherwise each re-run the timings
    const int lclass = dp.max_len <= 32 ? 32 : dp.max_len <= 64 ? 64 : 128;
    snprintf(key, sizeof key, "p%d m%d k%d L%d", dp.precision, dp.mode, dp.dim_pad, lclass);
    {
        std::lock_guard<std::mutex> lk(b.ctx->tune_mu);
        auto it = b.ctx->tuned.find(key);
        if (it != b.ctx->tuned.end()) {
            dp.umma_variant = it->second.first;
            dp.dtw_variant = it->second.second;
            return ABX_OK;
        }
    }
    int32_t best_d = dp.dtw_variant, best_u = dp.umma_variant;
    float best = 1e30f, t = 0.f;
    if (dp.mode == ABX_DTW) {
        for (int32_t dv = 0; dv < 4; ++dv) {
            RC(time_variant(b, dp, best_u, dv, &t));
            if (t < best) {
                best = t;
                best_d = dv;
            }
        }
    }
    if (dp.precision != ABX_FP32_SIMT) {
        best = 1e30f;
        for (int32_t uv = 0; uv < 4; ++uv) {
            RC(time_variant(b, dp, uv, best_d, &t));
            if (t < best) {
                best = t;
                best_u = uv;
            }
        }
    }
    dp.umma_variant = best_u;
    dp.dtw_variant = best_d;
    std::lock_guard<std::mutex> lk(b.ctx->tune_mu);
    b.ctx->tuned[key] = {best_u, best_d};
    return ABX_OK;
}

void free_batch(Batch *b) {
    if (!b) return;
    cudaStream_t s = b->last ? b->last : b->s;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &c : b->cls) {
        for (auto &sp : c.specs) {
            if (sp.sp) score_plan_b_free(sp.sp, s);
            dist_plan_free(&sp.dp, s, true);
            if (sp.cells) abx_cells_free(sp.cells);
        }
        if (c.items) abx_items_free(c.items);
        if (c.feats) cudaFreeAsync(c.feats, s);
    }
    if (b->err_mirror) b->ctx->pinned.release(b->err_mirror, s);
    Ctx *ctx = b->ctx;
    delete b;
    ctx_release(ctx);
}

}  // namespace

extern "C" {

int abx_batch_create_multi(abx_ctx *ctx_, int32_t n_tasks, const abx_task_input *tasks,
                           int32_t n_attr, int32_t n_specs, const abx_task_spec *specs,
                           int32_t mode, int32_t precision, int32_t weighted, int32_t recheck,
                           float margin, int32_t tune, void *stream, abx_batch **out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    REQUIRE(ctx && out && (n_tasks == 0 || tasks) && (n_specs == 0 || specs), ABX_E_INVALID,
            "NULL argument");
    REQUIRE(n_tasks > 0, ABX_E_INVALID, "no tasks");
    REQUIRE(n_specs > 0, ABX_E_INVALID, "no task specs");
    REQUIRE(n_attr > 0, ABX_E_INVALID, "bad attribute count");
    for (int32_t j = 0; j < n_specs; ++j) {
        const abx_task_spec &sp = specs[j];
        REQUIRE(sp.n_by >= 0 && sp.n_by <= 8 && sp.n_level_tokens >= 0 && sp.n_level_tokens <= 16,
                ABX_E_INVALID, "spec %d: bad sizes", j);
        REQUIRE(sp.on_attr >= 0 && sp.on_attr < n_attr, ABX_E_INVALID, "spec %d: bad on", j);
    }
    REQUIRE(recheck >= ABX_RECHECK_OFF && recheck <= ABX_RECHECK_MARGIN, ABX_E_INVALID,
            "bad recheck mode %d", recheck);
    *out = nullptr;
    Trace tr("batch");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(ctx->device));
    std::unique_ptr<Batch, void (*)(Batch *)> B(new (std::nothrow) Batch, free_batch);
    REQUIRE(B, ABX_E_OOM, "host allocation failed");
    Batch &b = *B;
    b.ctx = ctx;
    ctx_retain(ctx);  // released by free_batch
    b.n_tasks = n_tasks;
    b.n_specs = n_specs;
    b.mode = mode;
    b.precision = precision;
    b.recheck = recheck;
    b.weighted = weighted;
    b.s = s;
    const char *g = getenv("ABX_BATCH_GRAPH");
    b.use_graph = !(g && *g == '0');

    // dimension classes, in increasing dimension, tasks in input order
    std::map<int32_t, std::vector<int32_t>> by_dim;
    for (int32_t k = 0; k < n_tasks; ++k) {
        const abx_task_input &t = tasks[k];
        REQUIRE(t.feats && t.item_offsets && t.labels && t.dim > 0 && t.n_items > 0,
                ABX_E_INVALID, "task %d: bad input", k);
        REQUIRE(t.mem == ABX_MEM_HOST || t.mem == ABX_MEM_DEVICE_COPY, ABX_E_INVALID,
                "task %d: mem must be ABX_MEM_HOST or ABX_MEM_DEVICE_COPY", k);
        REQUIRE(t.item_offsets[0] == 0 && t.item_offsets[t.n_items] == t.n_frames, ABX_E_INVALID,
                "task %d: offsets do not span the frames", k);
        by_dim[t.dim].push_back(k);
    }
    b.task_class.assign(n_tasks, 0);
    b.task_pos.assign(n_tasks, 0);
    const int32_t n_attr2 = n_attr + 1;
    // attribute ids shifted by one behind the task attribute (id 0)
    std::vector<std::vector<int32_t>> by2(n_specs), lev2(n_specs);
    for (int32_t j = 0; j < n_specs; ++j) {
        by2[j].push_back(0);
        for (int32_t i = 0; i < specs[j].n_by; ++i) by2[j].push_back(specs[j].by[i] + 1);
        for (int32_t i = 0; i < specs[j].n_level_tokens; ++i) {
            const int32_t v = specs[j].levels[i];
            lev2[j].push_back(v < 0 ? v : v + 1);
        }
    }

    for (auto &kv : by_dim) {
        b.cls.emplace_back();
        BatchClass &c = b.cls.back();
        c.dim = kv.first;
        c.tasks = kv.second;
        int64_t frames = 0, items = 0;
        for (int32_t k : c.tasks) {
            frames += tasks[k].n_frames;
            items += tasks[k].n_items;
        }
        CU(cudaMallocAsync((void **)&c.feats, (size_t)std::max<int64_t>(frames, 1) * c.dim * 4, s));
        std::vector<int64_t> offs(items + 1, 0);
        std::vector<int32_t> lab((size_t)items * n_attr2);
        int64_t f0 = 0, i0 = 0;
        for (size_t pos = 0; pos < c.tasks.size(); ++pos) {
            const int32_t k = c.tasks[pos];
            const abx_task_input &t = tasks[k];
            b.task_class[k] = (int32_t)(b.cls.size() - 1);
            b.task_pos[k] = (int32_t)pos;
            CU(cudaMemcpyAsync(c.feats + f0 * c.dim, t.feats, (size_t)t.n_frames * c.dim * 4,
                               t.mem == ABX_MEM_HOST ? cudaMemcpyHostToDevice
                                                     : cudaMemcpyDeviceToDevice,
                               s));
            for (int64_t i = 0; i < t.n_items; ++i) {
                offs[i0 + i + 1] = f0 + t.item_offsets[i + 1];
                int32_t *row = &lab[(size_t)(i0 + i) * n_attr2];
                row[0] = (int32_t)pos;
                memcpy(row + 1, t.labels + (size_t)i * n_attr, n_attr * sizeof(int32_t));
            }
            f0 += t.n_frames;
            i0 += t.n_items;
        }
        tr.mark("copy+labels");
        RC(abx_load_items(ctx_, c.feats, frames, c.dim, offs.data(), items, lab.data(), n_attr2,
                          ABX_MEM_DEVICE_BORROW, stream, &c.items));
        tr.mark("items");
        const Items *it = reinterpret_cast<const Items *>(c.items);
        c.specs.resize(n_specs);
        for (int32_t j = 0; j < n_specs; ++j) {
            BatchSpec &sp = c.specs[j];
            RC(abx_build_cells(ctx_, c.items, specs[j].on_attr + 1, by2[j].data(),
                               (int32_t)by2[j].size(),
                               specs[j].across_attr >= 0 ? specs[j].across_attr + 1 : -1,
                               &sp.cells));
            tr.mark("cells");
            const Cells *cc = reinterpret_cast<const Cells *>(sp.cells);
            RC(dist_plan_build(ctx, it, cc, mode, ABX_DIST_ANGULAR, precision, s, &sp.dp));
            tr.mark("dist plan");
            RC(score_plan_b_build(ctx, cc, it, sp.dp, lev2[j].data(), (int32_t)lev2[j].size(),
                                  weighted, recheck, margin, s, &sp.sp));
            tr.mark("score plan");
            if (tune) RC(tune_plan(b, sp.dp));
        }
    }
    b.err_mirror = ctx->pinned.acquire(32 * b.cls.size() * n_specs);
    REQUIRE(b.err_mirror, ABX_E_OOM, "pinned host allocation failed");
    CU(cudaStreamSynchronize(s));
    tr.mark("sync");
    *out = reinterpret_cast<abx_batch *>(B.release());
    return ABX_OK;
}

int abx_batch_create(abx_ctx *ctx_, int32_t n_tasks, const abx_task_input *tasks, int32_t n_attr,
                     int32_t on_attr, const int32_t *by, int32_t n_by, int32_t across_attr,
                     int32_t mode, int32_t precision, const int32_t *levels,
                     int32_t n_level_tokens, int32_t weighted, int32_t recheck, float margin,
                     int32_t tune, void *stream, abx_batch **out) {
    REQUIRE(n_by >= 0 && n_by <= 8 && (n_by == 0 || by), ABX_E_INVALID, "bad by attributes");
    REQUIRE(n_level_tokens >= 0 && n_level_tokens <= 16 && (n_level_tokens == 0 || levels),
            ABX_E_INVALID, "bad levels");
    abx_task_spec sp;
    memset(&sp, 0, sizeof(sp));
    sp.on_attr = on_attr;
    sp.n_by = n_by;
    for (int32_t i = 0; i < n_by; ++i) sp.by[i] = by[i];
    sp.across_attr = across_attr;
    sp.n_level_tokens = n_level_tokens;
    for (int32_t i = 0; i < n_level_tokens; ++i) sp.levels[i] = levels[i];
    return abx_batch_create_multi(ctx_, n_tasks, tasks, n_attr, 1, &sp, mode, precision,
                                  weighted, recheck, margin, tune, stream, out);
}

int abx_batch_run(abx_batch *batch, void *stream) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    REQUIRE(b, ABX_E_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(b->ctx->device));
    b->last = s;
    ++b->runs;
    if (!b->use_graph) {
        for (size_t k = 0; k < b->cls.size(); ++k) RC(exec_class(*b, k, s));
        return ABX_OK;
    }
    if (!b->gexec) {
        // the capture stream must not be the legacy default stream
        cudaStream_t cap = s;
        cudaStream_t own = nullptr;
        if (cap == nullptr) {
            CU(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
            cap = own;
            CU(cudaStreamSynchronize(nullptr));
        }
        CU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        int rc = ABX_OK;
        for (size_t k = 0; k < b->cls.size() && !rc; ++k) rc = exec_class(*b, k, cap);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        if (own) cudaStreamDestroy(own);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CU(ce);
        b->graph = g;
        CU(cudaGraphInstantiate(&b->gexec, g, 0));
        size_t n = 0;
        CU(cudaGraphGetNodes(g, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        CU(cudaGraphGetNodes(g, nodes.data(), &n));
        b->graph_kernels = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            CU(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) ++b->graph_kernels;
        }
    }
    CU(cudaGraphLaunch(b->gexec, s));
    count_launches(b->graph_kernels);
    return ABX_OK;
}

int abx_batch_ready(abx_batch *batch) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    REQUIRE(b, ABX_E_INVALID, "NULL argument");
    REQUIRE(b->runs > 0, ABX_E_STATE, "abx_batch_run has not been called");
    const cudaError_t e = cudaStreamQuery(b->last);
    if (e == cudaErrorNotReady) return 0;
    CU(e);
    return 1;
}

int abx_batch_wait(abx_batch *batch, double *errors, int64_t *triplets, abx_score_stats *stats) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    REQUIRE(b && errors, ABX_E_INVALID, "NULL argument");
    REQUIRE(b->runs > 0, ABX_E_STATE, "abx_batch_run has not been called");
    CU(cudaSetDevice(b->ctx->device));
    CU(cudaStreamSynchronize(b->last));
    abx_score_stats tot{};
    const int32_t S = b->n_specs;
    for (size_t k = 0; k < b->cls.size(); ++k) {
        const BatchClass &c = b->cls[k];
        for (int32_t j = 0; j < S; ++j) {
            const int32_t *fl =
                (const int32_t *)((const uint8_t *)b->err_mirror + 32 * (k * S + j));
            REQUIRE(fl[0] == 0, ABX_E_ZERO_NORM, "a frame has zero L2 norm (angle undefined)");
            REQUIRE(fl[1] == 0, ABX_E_CUDA, "tile kernel pipeline wait expired (code %d)", fl[1]);
            std::vector<double> e(c.tasks.size());
            std::vector<int64_t> t(c.tasks.size());
            abx_score_stats st{};
            RC(score_plan_b_read(c.specs[j].sp, e.data(), t.data(), &st));
            for (size_t pos = 0; pos < c.tasks.size(); ++pos) {
                errors[(size_t)c.tasks[pos] * S + j] = e[pos];
                if (triplets) triplets[(size_t)c.tasks[pos] * S + j] = t[pos];
            }
            tot.n_cells += st.n_cells;
            tot.n_triplets += st.n_triplets;
            tot.n_undecided += st.n_undecided;
            tot.n_recheck_pairs += st.n_recheck_pairs;
            tot.n_flips += st.n_flips;
            tot.num2_total += st.num2_total;
            tot.count2_total += st.count2_total;
        }
    }
    if (stats) *stats = tot;
    return ABX_OK;
}

int abx_batch_get_info(const abx_batch *batch, abx_batch_info *info) {
    const Batch *b = reinterpret_cast<const Batch *>(batch);
    REQUIRE(b && info, ABX_E_INVALID, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_tasks = b->n_tasks;
    info->n_classes = (int32_t)b->cls.size();
    info->graph_kernels = b->graph_kernels;
    info->use_graph = b->use_graph ? 1 : 0;
    const int32_t S = b->n_specs;
    for (size_t k = 0; k < b->cls.size(); ++k) {
        const BatchClass &c = b->cls[k];
        info->device_bytes += (int64_t)c.dim * 4 * reinterpret_cast<const Items *>(c.items)->n_frames;
        for (int32_t j = 0; j < S; ++j) {
            const BatchSpec &sp = c.specs[j];
            abx_cells_info ci;
            RC(abx_cells_get_info(sp.cells, &ci));
            info->n_triplets += ci.n_triplets;
            info->n_pairs_cap += sp.dp.cap_total;
            info->device_bytes += dist_plan_bytes(sp.dp);
            if (b->runs > 0) {  // counts of the last waited-for run
                const int64_t *cnt =
                    (const int64_t *)((const uint8_t *)b->err_mirror + 32 * (k * S + j) + 16);
                info->n_pairs += cnt[0];
                info->n_frame_pairs += cnt[1];
                info->flops += 2.0 * (double)c.dim * (double)cnt[1];
            }
        }
        if (k < 8) {
            const DistPlan &dp = c.specs[0].dp;
            info->tile_variant[k] = dp.fused ? 4 : dp.umma_variant;
            info->dtw_variant[k] = dp.fused ? 4 : dp.dtw_variant;
            info->class_dim[k] = c.dim;
        }
    }
    return ABX_OK;
}

int abx_batch_set_graph(abx_batch *batch, int32_t on) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    REQUIRE(b, ABX_E_INVALID, "NULL argument");
    b->use_graph = on != 0;
    return ABX_OK;
}

int abx_batch_free(abx_batch *batch) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    if (!b) return ABX_OK;
    cudaSetDevice(b->ctx->device);
    free_batch(b);
    return ABX_OK;
}

}  // extern "C"
