// hc_profile.cu -- per-kernel device timing with CUDA events (hc_profile_*).
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hc_internal.h"

namespace hc {

namespace {

struct Record {
    const char *name;
    cudaEvent_t start, stop;
};

std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event()
{
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

bool profile_enabled() { return g_enabled.load(std::memory_order_relaxed) != 0; }

ProfileScope::ProfileScope(const char *name, cudaStream_t s) : name_(name), s_(s)
{
    if (!profile_enabled()) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;  // no timing in graphs
    std::lock_guard<std::mutex> lk(g_mu);
    start_ = take_event();
    stop_ = take_event();
    if (start_ && stop_) {
        cudaEventRecord(start_, s_);
        active_ = true;
    }
}

ProfileScope::~ProfileScope()
{
    if (!active_) return;
    cudaEventRecord(stop_, s_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_records.push_back(Record{name_, start_, stop_});
}

}  // namespace hc

extern "C" {

void hc_profile_enable(int on) { hc::g_enabled.store(on ? 1 : 0); }

hc_status hc_profile_collect(hc_kernel_time *entries, size_t cap, size_t *n_out)
{
    std::vector<hc::Record> recs;
    {
        std::lock_guard<std::mutex> lk(hc::g_mu);
        recs.swap(hc::g_records);
    }
    std::map<std::string, std::pair<uint64_t, double>> agg;
    hc_status st = HC_OK;
    for (const auto &r : recs) {
        cudaError_t e = cudaEventSynchronize(r.stop);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess && st == HC_OK) st = hc::cuda_error(e, "hc_profile_collect");
        auto &a = agg[r.name];
        a.first += 1;
        a.second += ms;
    }
    {
        std::lock_guard<std::mutex> lk(hc::g_mu);
        for (const auto &r : recs) {
            hc::g_pool.push_back(r.start);
            hc::g_pool.push_back(r.stop);
        }
    }
    size_t i = 0;
    for (const auto &kv : agg) {
        if (entries && i < cap) {
            memset(&entries[i], 0, sizeof(hc_kernel_time));
            strncpy(entries[i].name, kv.first.c_str(), sizeof(entries[i].name) - 1);
            entries[i].launches = kv.second.first;
            entries[i].total_ms = kv.second.second;
        }
        ++i;
    }
    if (n_out) *n_out = i;
    return st;
}

}  // extern "C"
