// trace.cu -- implementation of the launch tracing declared in trace.h and of
// its C-ABI entry points (randutv_trace_*).
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/randutv.h"
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

struct Record {
    std::string cls;
    double flops, bytes;
    int kernels;
    cudaEvent_t e0, e1;
};

std::atomic<int> g_enabled{0};
std::atomic<long long> g_launches{0};
std::mutex g_mu;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

void trace_count(int kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }

TraceScope::TraceScope(const char* cls, double flops, double bytes, cudaStream_t st)
    : cls_(cls), flops_(flops), bytes_(bytes), st_(st), slot_(-1), start_(g_launches.load()) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    // launches under a device gate may not run: their class is marked and
    // their algorithmic work is not counted
    const bool gated = current_gate().flag != nullptr;
    Record r{gated ? std::string(cls) + "_gated" : std::string(cls), gated ? 0.0 : flops, gated ? 0.0 : bytes, 0,
             get_event(), get_event()};
    cudaEventRecord(r.e0, st);
    g_records.push_back(r);
    slot_ = (int)g_records.size() - 1;
}

TraceScope::~TraceScope() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_records[slot_].e1, st_);
    g_records[slot_].kernels = (int)(g_launches.load() - start_);
}

}  // namespace rutv

using namespace rutv;

extern "C" {

int randutv_trace_enable(int on) {
    int prev = g_enabled.exchange(on ? 1 : 0);
    return prev;
}

long long randutv_launch_count(void) { return g_launches.load(); }

int randutv_trace_read(randutv_trace_class* out, int max_classes) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<randutv_trace_class> acc;
    for (Record& r : g_records) {
        cudaEventSynchronize(r.e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        size_t k = 0;
        for (; k < acc.size(); ++k)
            if (std::strncmp(acc[k].name, r.cls.c_str(), sizeof(acc[k].name)) == 0) break;
        if (k == acc.size()) {
            randutv_trace_class c{};
            std::strncpy(c.name, r.cls.c_str(), sizeof(c.name) - 1);
            acc.push_back(c);
        }
        acc[k].scopes += 1;
        acc[k].kernels += r.kernels;
        acc[k].ms += ms;
        acc[k].flops += r.flops;
        acc[k].bytes += r.bytes;
    }
    int n = (int)acc.size();
    for (int i = 0; i < n && i < max_classes; ++i) out[i] = acc[i];
    return n;
}

void randutv_trace_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (Record& r : g_records) {
        g_pool.push_back(r.e0);
        g_pool.push_back(r.e1);
    }
    g_records.clear();
}

}  // extern "C"
