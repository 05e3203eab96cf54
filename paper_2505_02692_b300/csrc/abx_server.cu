// Serving: continuous batching of ABX jobs on one GPU.
//
// max_inflight worker threads each own one launch slot (a stream).  A free
// worker takes queued jobs in arrival order while their estimated device
// memory fits the budget, joins them into one batch (one feature copy, shared
// launches per dimension class, every task spec), launches it on its stream
// and waits for it; the results go to the jobs and the memory back to the
// budget.  Jobs that arrive while batches run are taken by the next free
// worker, so one worker's host planning overlaps the others' GPU work and
// the batches of different workers share the GPU (separate streams).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "abx_internal.h"

namespace abx {
namespace {

struct Job {
    int64_t ticket = 0;
    abx_task_input in{};
    int64_t bytes = 0;  // admission estimate
    abx_job_result res{};
    bool done = false;
};

struct Server {
    Ctx *ctx = nullptr;
    abx_server_config cfg{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
    std::vector<cudaStream_t> streams;
    int64_t next_ticket = 1, next_batch = 1, used = 0;
    int32_t running = 0;
    abx_server_stats st{};
    bool stop = false;
    std::vector<std::thread> workers;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

// Device bytes a job will hold, before its batch exists: the feature copy,
// the packed rows, and per spec the group matrices (16 B per ordered pair of
// a group), the pair list and the tile buffer, from the group sizes of the
// spec's by attributes.
int64_t estimate_bytes(const abx_server_config &cfg, const abx_task_input &in, int32_t n_attr) {
    const int64_t dim_pad = (in.dim + 127) / 128 * 128;
    const int64_t elem = cfg.precision == ABX_BF16 ? 2 : cfg.precision == ABX_FP8 ? 1 : 4;
    int64_t b = in.n_frames * in.dim * 4 + in.n_frames * dim_pad * elem + in.n_frames * 16;
    std::vector<int32_t> mx(n_attr, 0);
    for (int64_t i = 0; i < in.n_items; ++i)
        for (int32_t k = 0; k < n_attr; ++k) mx[k] = std::max(mx[k], in.labels[i * n_attr + k]);
    for (int32_t j = 0; j < cfg.n_specs; ++j) {
        const abx_task_spec &sp = cfg.specs[j];
        int64_t space = 1;
        for (int32_t k = 0; k < sp.n_by; ++k) space *= (int64_t)mx[sp.by[k]] + 1;
        std::vector<int64_t> items, frames;
        std::unordered_map<int64_t, std::pair<int64_t, int64_t>> big;
        const bool dense = space <= (1 << 22);
        if (dense) {
            items.assign(space, 0);
            frames.assign(space, 0);
        }
        for (int64_t i = 0; i < in.n_items; ++i) {
            int64_t key = 0;
            for (int32_t k = 0; k < sp.n_by; ++k)
                key = key * ((int64_t)mx[sp.by[k]] + 1) + in.labels[i * n_attr + sp.by[k]];
            const int64_t T = in.item_offsets[i + 1] - in.item_offsets[i];
            if (dense) {
                items[key] += 1;
                frames[key] += T;
            } else {
                auto &e = big[key];
                e.first += 1;
                e.second += T;
            }
        }
        int64_t dm = 0, tiles = 0;
        auto add = [&](int64_t n, int64_t f) {
            dm += n * n;
            const int64_t p = (f + 127) / 128;
            tiles += p * (p + 1) / 2;
        };
        if (dense)
            for (int64_t g = 0; g < space; ++g) add(items[g], frames[g]);
        else
            for (auto &kv : big) add(kv.second.first, kv.second.second);
        const int64_t tile_buf = std::min<int64_t>(tiles, (8192LL << 20) / (128 * 128 * 4));
        b += dm * 16 + dm * 8 + tile_buf * 128 * 128 * 4 + dm * 8;
    }
    return b;
}

void finish(Server &S, abx_batch *bt, const std::vector<Job *> &take, int64_t bytes, int rc) {
    const int32_t ns = S.cfg.n_specs;
    std::vector<double> err(take.size() * ns, 0.0);
    std::vector<int64_t> trip(take.size() * ns, 0);
    if (rc == ABX_OK) rc = abx_batch_wait(bt, err.data(), trip.data(), nullptr);
    const double t = S.now();
    std::lock_guard<std::mutex> lk(S.mu);
    for (size_t k = 0; k < take.size(); ++k) {
        Job *j = take[k];
        j->res.status = rc;
        j->res.n_specs = ns;
        for (int32_t q = 0; q < ns; ++q) {
            j->res.errors[q] = err[k * ns + q];
            j->res.triplets[q] = trip[k * ns + q];
        }
        j->res.t_done = t;
        j->done = true;
        if (rc == ABX_OK)
            ++S.st.completed;
        else
            ++S.st.failed;
    }
    S.used -= bytes;
    --S.running;
    S.cv_done.notify_all();
    S.cv_work.notify_all();
}

void worker(Server *Sp, int slot) {
    Server &S = *Sp;
    cudaSetDevice(S.ctx->device);
    abx_ctx *ctx = reinterpret_cast<abx_ctx *>(S.ctx);
    cudaStream_t s = S.streams[slot];
    for (;;) {
        // admission: FIFO while the memory fits
        std::vector<Job *> take;
        int64_t bytes = 0, id = 0;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            S.cv_work.wait(lk, [&] { return S.stop || !S.queue.empty(); });
            if (S.stop) return;
            while (!S.queue.empty() && (int)take.size() < S.cfg.max_batch_jobs) {
                Job *j = S.queue.front();
                const bool fits = S.used + bytes + j->bytes <= S.cfg.hbm_budget;
                // the head job alone runs when nothing else holds memory
                if (!fits && !(take.empty() && S.running == 0)) break;
                take.push_back(j);
                bytes += j->bytes;
                S.queue.pop_front();
                if (!fits) break;
            }
            if (take.empty()) {  // wait for memory to come back
                S.cv_work.wait_for(lk, std::chrono::microseconds(500));
                continue;
            }
            S.used += bytes;
            S.st.peak_bytes = std::max(S.st.peak_bytes, S.used);
            ++S.running;
            S.st.max_inflight_seen = std::max(S.st.max_inflight_seen, S.running);
            ++S.st.batches;
            id = S.next_batch++;
            if (!S.queue.empty()) S.cv_work.notify_one();  // another worker may take more
        }
        // form and launch the batch (host planning here overlaps other
        // workers' GPU work), then wait for it on this worker's stream
        const double ta = S.now();
        std::vector<abx_task_input> in;
        for (Job *j : take) {
            j->res.t_admit = ta;
            in.push_back(j->in);
        }
        abx_batch *bt = nullptr;
        int rc = abx_batch_create_multi(ctx, (int32_t)in.size(), in.data(), S.cfg.n_attr,
                                        S.cfg.n_specs, S.cfg.specs, S.cfg.mode, S.cfg.precision,
                                        S.cfg.weighted, S.cfg.recheck, S.cfg.margin, S.cfg.tune,
                                        s, &bt);
        if (rc == ABX_OK) rc = abx_batch_set_graph(bt, 0);  // one run: no graph
        if (rc == ABX_OK) {
            abx_batch_info info;
            if (abx_batch_get_info(bt, &info) == ABX_OK) {
                std::lock_guard<std::mutex> lk(S.mu);
                S.used += info.device_bytes - bytes;  // the batch's own figure
                bytes = info.device_bytes;
                S.st.peak_bytes = std::max(S.st.peak_bytes, S.used);
            }
            rc = abx_batch_run(bt, s);
        }
        const double tl = S.now();
        for (Job *j : take) {
            j->res.t_launch = tl;
            j->res.batch_id = id;
            j->res.batch_jobs = (int32_t)take.size();
        }
        finish(S, bt, take, bytes, rc);  // abx_batch_wait synchronises the stream
        if (bt) abx_batch_free(bt);
    }
}

}  // namespace
}  // namespace abx

using namespace abx;

#define REQUIRE(cond, code, ...)      \
    do {                              \
        if (!(cond)) {                \
            set_error(__VA_ARGS__);   \
            return (code);            \
        }                             \
    } while (0)

extern "C" {

int abx_server_create(abx_ctx *ctx_, const abx_server_config *cfg, abx_server **out) {
    Ctx *ctx = reinterpret_cast<Ctx *>(ctx_);
    REQUIRE(ctx && cfg && out, ABX_E_INVALID, "NULL argument");
    REQUIRE(cfg->n_specs >= 1 && cfg->n_specs <= ABX_SERVER_MAX_SPECS, ABX_E_INVALID,
            "n_specs must be 1..%d", ABX_SERVER_MAX_SPECS);
    REQUIRE(cfg->n_attr >= 1, ABX_E_INVALID, "n_attr must be positive");
    for (int32_t j = 0; j < cfg->n_specs; ++j) {
        const abx_task_spec &sp = cfg->specs[j];
        REQUIRE(sp.n_by >= 0 && sp.n_by <= 8 && sp.on_attr >= 0 && sp.on_attr < cfg->n_attr,
                ABX_E_INVALID, "spec %d: bad attributes", j);
        for (int32_t k = 0; k < sp.n_by; ++k)
            REQUIRE(sp.by[k] >= 0 && sp.by[k] < cfg->n_attr, ABX_E_INVALID,
                    "spec %d: bad by attribute", j);
    }
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        set_error("cudaSetDevice failed");
        return ABX_E_CUDA;
    }
    std::unique_ptr<Server> S(new (std::nothrow) Server);
    REQUIRE(S, ABX_E_OOM, "host allocation failed");
    S->ctx = ctx;
    S->cfg = *cfg;
    if (S->cfg.max_inflight <= 0) S->cfg.max_inflight = 3;
    if (S->cfg.max_batch_jobs <= 0) S->cfg.max_batch_jobs = 32;
    if (S->cfg.hbm_budget <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->cfg.hbm_budget = (int64_t)(0.8 * (double)fr);
    }
    S->streams.resize(S->cfg.max_inflight);
    for (auto &s : S->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("stream creation failed");
            return ABX_E_CUDA;
        }
    S->t0 = std::chrono::steady_clock::now();
    ctx_retain(ctx);  // released by abx_server_destroy
    for (int i = 0; i < S->cfg.max_inflight; ++i) S->workers.emplace_back(worker, S.get(), i);
    *out = reinterpret_cast<abx_server *>(S.release());
    return ABX_OK;
}

int abx_server_submit(abx_server *srv, const abx_task_input *job, int64_t *ticket) {
    Server *S = reinterpret_cast<Server *>(srv);
    REQUIRE(S && job && ticket, ABX_E_INVALID, "NULL argument");
    REQUIRE(job->feats && job->item_offsets && job->labels && job->n_items > 0 && job->dim > 0,
            ABX_E_INVALID, "bad job");
    REQUIRE(job->mem == ABX_MEM_HOST || job->mem == ABX_MEM_DEVICE_COPY, ABX_E_INVALID,
            "job mem must be ABX_MEM_HOST or ABX_MEM_DEVICE_COPY");
    std::unique_ptr<Job> j(new (std::nothrow) Job);
    REQUIRE(j, ABX_E_OOM, "host allocation failed");
    j->in = *job;
    j->bytes = estimate_bytes(S->cfg, *job, S->cfg.n_attr);
    std::lock_guard<std::mutex> lk(S->mu);
    REQUIRE(!S->stop, ABX_E_STATE, "server is stopping");
    j->ticket = S->next_ticket++;
    j->res.t_submit = S->now();
    *ticket = j->ticket;
    S->queue.push_back(j.get());
    S->jobs[j->ticket] = std::move(j);
    ++S->st.submitted;
    S->cv_work.notify_one();
    return ABX_OK;
}

int abx_server_poll(abx_server *srv, int64_t ticket, abx_job_result *out) {
    Server *S = reinterpret_cast<Server *>(srv);
    REQUIRE(S && out, ABX_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    REQUIRE(it != S->jobs.end(), ABX_E_INVALID, "unknown ticket %lld", (long long)ticket);
    if (!it->second->done) return 0;
    *out = it->second->res;
    S->jobs.erase(it);
    return 1;
}

int abx_server_wait(abx_server *srv, int64_t ticket, abx_job_result *out) {
    Server *S = reinterpret_cast<Server *>(srv);
    REQUIRE(S && out, ABX_E_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    REQUIRE(it != S->jobs.end(), ABX_E_INVALID, "unknown ticket %lld", (long long)ticket);
    Job *j = it->second.get();
    S->cv_done.wait(lk, [&] { return j->done; });
    *out = j->res;
    S->jobs.erase(ticket);
    return ABX_OK;
}

int abx_server_get_stats(abx_server *srv, abx_server_stats *out) {
    Server *S = reinterpret_cast<Server *>(srv);
    REQUIRE(S && out, ABX_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    return ABX_OK;
}

double abx_server_now(abx_server *srv) {
    Server *S = reinterpret_cast<Server *>(srv);
    return S ? S->now() : 0.0;
}

int abx_server_destroy(abx_server *srv) {
    Server *S = reinterpret_cast<Server *>(srv);
    if (!S) return ABX_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Job *j : S->queue) {
            j->res.status = ABX_E_STATE;
            j->done = true;
            ++S->st.failed;
        }
        S->queue.clear();
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    for (auto &w : S->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(S->ctx->device);
    for (auto s : S->streams) cudaStreamDestroy(s);
    Ctx *ctx = S->ctx;
    delete S;
    ctx_release(ctx);
    return ABX_OK;
}

}  // extern "C"
