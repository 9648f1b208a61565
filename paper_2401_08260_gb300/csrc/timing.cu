// Kernel launch counting and optional CUDA-event timing (slk_timing_* calls).
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace slk {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

LaunchScope::LaunchScope(const char* name, cudaStream_t st) : name_(name), st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_enabled.load(std::memory_order_relaxed)) {
        start_ = take_event();
        if (start_) cudaEventRecord(start_, st_);
    }
}

LaunchScope::~LaunchScope() {
    if (!start_) return;
    cudaEvent_t stop = take_event();
    if (!stop) return;
    cudaEventRecord(stop, st_);
    std::lock_guard<std::mutex> g(g_mu);
    g_recs.push_back({name_, start_, stop});
}

}  // namespace slk

using namespace slk;

extern "C" {

slk_status slk_timing_enable(int32_t on) {
    g_enabled.store(on != 0);
    return SLK_OK;
}

int64_t slk_launch_count(void) { return g_launches.load(); }

slk_status slk_timing_read(slk_kernel_time* out, int32_t cap, int32_t* count) {
    if (!count || (cap > 0 && !out)) return SLK_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    std::map<std::string, std::pair<long long, double>> agg;
    std::vector<std::string> order;
    for (const Rec& r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            cudaGetLastError();
            return SLK_ERR_CUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            agg[r.name] = {1, ms};
        } else {
            it->second.first += 1;
            it->second.second += ms;
        }
    }
    int n = 0;
    for (const std::string& name : order) {
        if (n < cap) {
            std::memset(&out[n], 0, sizeof(out[n]));
            std::strncpy(out[n].name, name.c_str(), sizeof(out[n].name) - 1);
            out[n].launches = agg[name].first;
            out[n].total_ms = agg[name].second;
        }
        ++n;
    }
    *count = n;
    return SLK_OK;
}

slk_status slk_timing_reset(void) {
    std::lock_guard<std::mutex> g(g_mu);
    for (const Rec& r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    cudaGetLastError();
    return SLK_OK;
}

}  // extern "C"
