// Serving: continuous batching of ABX jobs on one GPU.
//
// n_planners planner threads and max_inflight executor threads (a stream
// each) form a two-stage pipeline.  A planner takes the queued jobs that fit
// the device-memory budget (up to max_batch_jobs) and builds one batch of
// them on the host (one feature copy, shared launches per dimension class,
// every task spec); an executor launches a planned batch on its stream, waits
// for it and hands the results to the jobs.  Planners plan just in time:
// with every executor busy a planner waits until the earliest one is expected
// to finish within the planning time of what is queued (running estimates of
// host planning and GPU time per item), so jobs that arrive in the meantime
// join the next batch instead of forming batches of one; with an executor
// idle it plans at once.  Host planning of batch k + 1 thus runs during the
// GPU work of batch k, and several planners plan batches side by side.
//
// Failures stay with the job that causes them.  A malformed job is refused
// at submission.  A batch of several jobs that fails (a zero-norm frame found
// on the GPU, an allocation that fails) is split: its jobs go back to the
// head of the queue to run alone, so only the faulty job fails.  A queued
// job can be cancelled.  The configuration's fail_inject field makes the
// n-th batch creation fail as an allocation failure would (host-side test
// hook; nothing on the GPU fails).
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
    bool queued = false;
    bool solo = false;  // after a failed shared batch: run alone
};

struct Planned {
    std::vector<Job *> jobs;
    abx_batch *bt = nullptr;
    int rc = ABX_OK;
    int64_t bytes = 0, id = 0, items = 0;
    cudaEvent_t created = nullptr;  // the creation's uploads are on the planner's stream
    double est_exec = 0.0;          // seconds
};

struct Server {
    Ctx *ctx = nullptr;
    abx_server_config cfg{};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_ready;
    std::deque<Job *> queue;
    std::deque<Planned *> ready;
    std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
    std::vector<cudaStream_t> plan_streams, streams;
    std::vector<double> busy_until;  // per executor: expected end of its batch, 0 when idle
    int64_t next_ticket = 1, next_batch = 1, used = 0, creations = 0;
    int32_t running = 0, planning = 0;
    // running estimates (exponential averages over batches), seconds per item
    double plan_s_per_item = 2e-7, exec_s_per_item = 2e-7;
    abx_server_stats st{};
    bool stop = false;
    std::vector<std::thread> planners, executors;

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

// Items of the jobs the planner would take now (a solo job alone, else the
// queue's head jobs in order while they fit the budget).
std::vector<Job *> next_batch_jobs(const Server &S) {
    std::vector<Job *> take;
    int64_t bytes = 0;
    for (Job *j : S.queue) {
        if ((int)take.size() >= S.cfg.max_batch_jobs) break;
        if (j->solo && !take.empty()) break;
        const bool fits = S.used + bytes + j->bytes <= S.cfg.hbm_budget;
        // the head job alone runs when nothing else holds memory
        if (!fits && !(take.empty() && S.running == 0 && S.ready.empty())) break;
        take.push_back(j);
        bytes += j->bytes;
        if (!fits || j->solo) break;
    }
    return take;
}

int64_t items_of(const std::vector<Job *> &v) {
    int64_t n = 0;
    for (const Job *j : v) n += j->in.n_items;
    return n;
}

// Hands a batch's results to its jobs.  A failed batch of several jobs is
// split: its jobs go back to the head of the queue, each to run alone.
void finish(Server &S, Planned &pb, int rc, int slot, double t_launch) {
    const int32_t ns = S.cfg.n_specs;
    std::vector<double> err(pb.jobs.size() * ns, 0.0);
    std::vector<int64_t> trip(pb.jobs.size() * ns, 0);
    if (rc == ABX_OK) rc = abx_batch_wait(pb.bt, err.data(), trip.data(), nullptr);
    const double t = S.now(), exec_s = t - t_launch;
    std::lock_guard<std::mutex> lk(S.mu);
    if (rc != ABX_OK && pb.jobs.size() > 1) {
        for (auto it = pb.jobs.rbegin(); it != pb.jobs.rend(); ++it) {
            Job *j = *it;
            j->solo = true;
            j->queued = true;
            S.queue.push_front(j);
        }
        ++S.st.retried;
    } else {
        for (size_t k = 0; k < pb.jobs.size(); ++k) {
            Job *j = pb.jobs[k];
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
        if (rc == ABX_OK && pb.items > 0 && exec_s > 0.0)
            S.exec_s_per_item = 0.7 * S.exec_s_per_item + 0.3 * exec_s / (double)pb.items;
    }
    S.used -= pb.bytes;
    --S.running;
    S.busy_until[slot] = 0.0;
    S.cv_done.notify_all();
    S.cv_work.notify_all();
}

void planner(Server *Sp, int slot) {
    Server &S = *Sp;
    cudaSetDevice(S.ctx->device);
    cudaStream_t ps = S.plan_streams[slot];
    abx_ctx *ctx = reinterpret_cast<abx_ctx *>(S.ctx);
    const int n_exec = (int)S.streams.size();
    // batches planned or being planned that no executor runs yet: one per
    // executor, plus one per further planner (planning in parallel)
    const int cap = n_exec + (int)S.plan_streams.size() - 1;
    for (;;) {
        std::vector<Job *> take;
        int64_t bytes = 0, id = 0, creation = 0;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            for (;;) {
                if (S.stop) return;
                if (S.queue.empty() || (int)S.ready.size() + S.planning >= cap) {
                    S.cv_work.wait(lk);
                    continue;
                }
                take = next_batch_jobs(S);
                if (take.empty()) {  // memory comes back when a batch finishes
                    S.cv_work.wait_for(lk, std::chrono::microseconds(500));
                    continue;
                }
                // just in time: with every executor busy (or spoken for by a
                // planned batch), wait while the earliest one is expected to
                // stay busy longer than planning what is queued takes
                const int busy = S.running + (int)S.ready.size() + S.planning;
                if (busy < n_exec || (int)take.size() >= S.cfg.max_batch_jobs || take[0]->solo)
                    break;
                double free_at = 1e300;
                for (double b : S.busy_until)
                    if (b > 0.0) free_at = std::min(free_at, b);
                for (const Planned *r : S.ready) free_at += r->est_exec / n_exec;
                const double lead = S.plan_s_per_item * (double)items_of(take) * 1.2 + 2e-4;
                const double wait = free_at - lead - S.now();
                if (wait <= 0.0 || free_at >= 1e299) break;
                S.cv_work.wait_for(lk, std::chrono::microseconds(
                                           (int64_t)(1e6 * std::min(wait, 2e-3)) + 1));
            }
            for (size_t k = 0; k < take.size(); ++k) {
                S.queue.pop_front();
                take[k]->queued = false;
                bytes += take[k]->bytes;
            }
            S.used += bytes;
            S.st.peak_bytes = std::max(S.st.peak_bytes, S.used);
            ++S.st.batches;
            id = S.next_batch++;
            creation = ++S.creations;  // this creation's number, taken under the lock
            ++S.planning;
        }
        std::unique_ptr<Planned> pb(new Planned);
        pb->jobs = take;
        pb->bytes = bytes;
        pb->id = id;
        pb->items = items_of(take);
        const double ta = S.now();
        std::vector<abx_task_input> in;
        for (Job *j : take) {
            j->res.t_admit = ta;
            in.push_back(j->in);
        }
        int rc = ABX_OK;
        if (S.cfg.fail_inject > 0 && creation == S.cfg.fail_inject) {
            set_error("abx_server: injected allocation failure (fail_inject)");
            rc = ABX_E_OOM;
        } else {
            rc = abx_batch_create_multi(ctx, (int32_t)in.size(), in.data(), S.cfg.n_attr,
                                        S.cfg.n_specs, S.cfg.specs, S.cfg.mode, S.cfg.precision,
                                        S.cfg.weighted, S.cfg.recheck, S.cfg.margin, S.cfg.tune,
                                        ps, &pb->bt);
        }
        if (rc == ABX_OK) rc = abx_batch_set_graph(pb->bt, 0);  // one run: no graph
        if (rc == ABX_OK) {
            abx_batch_info info;
            if (abx_batch_get_info(pb->bt, &info) == ABX_OK) {
                std::lock_guard<std::mutex> lk(S.mu);
                S.used += info.device_bytes - pb->bytes;  // the batch's own figure
                pb->bytes = info.device_bytes;
                S.st.peak_bytes = std::max(S.st.peak_bytes, S.used);
            }
            if (cudaEventCreateWithFlags(&pb->created, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(pb->created, ps) != cudaSuccess)
                rc = ABX_E_CUDA;
        }
        pb->rc = rc;
        const double tp = S.now() - ta;
        {
            std::lock_guard<std::mutex> lk(S.mu);
            if (rc == ABX_OK && pb->items > 0)
                S.plan_s_per_item = 0.7 * S.plan_s_per_item + 0.3 * tp / (double)pb->items;
            pb->est_exec = S.exec_s_per_item * (double)pb->items;
            --S.planning;
            S.ready.push_back(pb.release());
            S.cv_ready.notify_one();
        }
    }
}

void executor(Server *Sp, int slot) {
    Server &S = *Sp;
    cudaSetDevice(S.ctx->device);
    cudaStream_t s = S.streams[slot];
    for (;;) {
        Planned *pbp = nullptr;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            S.cv_ready.wait(lk, [&] { return S.stop || !S.ready.empty(); });
            if (S.ready.empty()) return;  // stopping, nothing left to run
            pbp = S.ready.front();
            S.ready.pop_front();
            ++S.running;
            S.st.max_inflight_seen = std::max(S.st.max_inflight_seen, S.running);
            S.busy_until[slot] = S.now() + pbp->est_exec;
            S.cv_work.notify_all();  // the planner may plan the next batch
        }
        std::unique_ptr<Planned> pb(pbp);
        int rc = pb->rc;
        const double tl = S.now();
        if (rc == ABX_OK && cudaStreamWaitEvent(s, pb->created, 0) != cudaSuccess) rc = ABX_E_CUDA;
        if (rc == ABX_OK) rc = abx_batch_run(pb->bt, s);
        for (Job *j : pb->jobs) {
            j->res.t_launch = tl;
            j->res.batch_id = pb->id;
            j->res.batch_jobs = (int32_t)pb->jobs.size();
        }
        finish(S, *pb, rc, slot, tl);  // abx_batch_wait synchronises the stream
        if (pb->bt) abx_batch_free(pb->bt);
        if (pb->created) cudaEventDestroy(pb->created);
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
    if (S->cfg.max_inflight <= 0) S->cfg.max_inflight = 1;
    if (S->cfg.n_planners <= 0) S->cfg.n_planners = 2;
    if (S->cfg.max_batch_jobs <= 0) S->cfg.max_batch_jobs = 32;
    if (S->cfg.hbm_budget <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->cfg.hbm_budget = (int64_t)(0.8 * (double)fr);
    }
    S->streams.resize(S->cfg.max_inflight);
    S->busy_until.assign(S->cfg.max_inflight, 0.0);
    for (auto &s : S->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("stream creation failed");
            return ABX_E_CUDA;
        }
    S->plan_streams.resize(S->cfg.n_planners);
    for (auto &s : S->plan_streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("stream creation failed");
            return ABX_E_CUDA;
        }
    S->t0 = std::chrono::steady_clock::now();
    ctx_retain(ctx);  // released by abx_server_destroy
    for (int i = 0; i < S->cfg.n_planners; ++i) S->planners.emplace_back(planner, S.get(), i);
    for (int i = 0; i < S->cfg.max_inflight; ++i) S->executors.emplace_back(executor, S.get(), i);
    *out = reinterpret_cast<abx_server *>(S.release());
    return ABX_OK;
}

// Host-side checks of a submitted job: item offsets from 0 to n_frames,
// every item at least one frame, labels non-negative.  A job that fails them
// never enters a batch.
static int validate_job(const abx_task_input *job, int32_t n_attr) {
    const int64_t *o = job->item_offsets;
    REQUIRE(o[0] == 0 && o[job->n_items] == job->n_frames, ABX_E_INVALID,
            "job: item offsets must run from 0 to n_frames");
    for (int64_t i = 0; i < job->n_items; ++i)
        REQUIRE(o[i + 1] > o[i], ABX_E_INVALID, "job: item %lld has no frames", (long long)i);
    for (int64_t i = 0; i < job->n_items * n_attr; ++i)
        REQUIRE(job->labels[i] >= 0, ABX_E_INVALID, "job: negative label code");
    return ABX_OK;
}

int abx_server_submit(abx_server *srv, const abx_task_input *job, int64_t *ticket) {
    Server *S = reinterpret_cast<Server *>(srv);
    REQUIRE(S && job && ticket, ABX_E_INVALID, "NULL argument");
    REQUIRE(job->feats && job->item_offsets && job->labels && job->n_items > 0 && job->dim > 0,
            ABX_E_INVALID, "bad job");
    REQUIRE(job->mem == ABX_MEM_HOST || job->mem == ABX_MEM_DEVICE_COPY, ABX_E_INVALID,
            "job mem must be ABX_MEM_HOST or ABX_MEM_DEVICE_COPY");
    const int vrc = validate_job(job, S->cfg.n_attr);
    if (vrc != ABX_OK) return vrc;
    std::unique_ptr<Job> j(new (std::nothrow) Job);
    REQUIRE(j, ABX_E_OOM, "host allocation failed");
    j->in = *job;
    j->bytes = estimate_bytes(S->cfg, *job, S->cfg.n_attr);
    std::lock_guard<std::mutex> lk(S->mu);
    REQUIRE(!S->stop, ABX_E_STATE, "server is stopping");
    j->ticket = S->next_ticket++;
    j->res.t_submit = S->now();
    *ticket = j->ticket;
    j->queued = true;
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

int abx_server_cancel(abx_server *srv, int64_t ticket) {
    Server *S = reinterpret_cast<Server *>(srv);
    REQUIRE(S, ABX_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    REQUIRE(it != S->jobs.end(), ABX_E_INVALID, "unknown ticket %lld", (long long)ticket);
    Job *j = it->second.get();
    REQUIRE(j->queued && !j->done, ABX_E_STATE,
            "job %lld is already in a batch or done; it cannot be cancelled", (long long)ticket);
    S->queue.erase(std::find(S->queue.begin(), S->queue.end(), j));
    j->queued = false;
    j->res.status = ABX_E_CANCELLED;
    j->res.t_done = S->now();
    j->done = true;
    ++S->st.cancelled;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
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
            j->queued = false;
            j->done = true;
            ++S->st.failed;
        }
        S->queue.clear();
        S->cv_work.notify_all();
        S->cv_ready.notify_all();
        S->cv_done.notify_all();
    }
    // the planners stop; the executors run the planned batches, then stop
    for (auto &w : S->planners)
        if (w.joinable()) w.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->cv_ready.notify_all();
    }
    for (auto &w : S->executors)
        if (w.joinable()) w.join();
    cudaSetDevice(S->ctx->device);
    for (auto s : S->streams) cudaStreamDestroy(s);
    for (auto s : S->plan_streams) cudaStreamDestroy(s);
    Ctx *ctx = S->ctx;
    delete S;
    ctx_release(ctx);
    return ABX_OK;
}

}  // extern "C"
