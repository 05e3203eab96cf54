// Launch accounting and optional per-kernel timing.
//
// Every kernel launch of the library goes through prof_begin / prof_end.
// The launch counter is always kept; when timing is enabled
// (abx_prof_enable(1)), a pair of CUDA events is recorded around the launch
// on the launching stream and the elapsed time is accumulated per kernel
// name at the next abx_prof_read.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "abx_internal.h"

namespace abx {
namespace {

std::atomic<long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_mu;

struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
std::map<std::string, std::pair<double, long long>> g_total;  // ms, launches

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void drain() {
    for (auto &p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto &t = g_total[p.name];
        t.first += ms;
        t.second += 1;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(const char *name, cudaStream_t s) : name_(name), s_(s) {
    // launches captured into a CUDA graph are counted by the graph's owner
    // per replay, and timed as a whole
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_timing.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_mu);
        a_ = take_event();
        cudaEventRecord((cudaEvent_t)a_, s);
    }
}

ProfScope::~ProfScope() {
    if (a_) {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaEvent_t b = take_event();
        cudaEventRecord(b, s_);
        g_pending.push_back(Pending{name_, (cudaEvent_t)a_, b});
    }
}

}  // namespace abx

using namespace abx;

extern "C" {

int64_t abx_kernel_launches(void) { return g_launches.load(); }

int abx_prof_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    g_timing.store(on ? 1 : 0);
    return ABX_OK;
}

int abx_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    g_total.clear();
    return ABX_OK;
}

int abx_prof_read(int32_t index, char *name, int32_t name_cap, double *ms, int64_t *launches) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    if (index < 0 || index >= (int32_t)g_total.size()) return ABX_E_INVALID;
    auto it = g_total.begin();
    std::advance(it, index);
    if (name && name_cap > 0) {
        strncpy(name, it->first.c_str(), (size_t)name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (ms) *ms = it->second.first;
    if (launches) *launches = it->second.second;
    return ABX_OK;
}

}  // extern "C"
