// Kernel tracing: CUDA events recorded around every kernel the library
// launches, on the launching stream, accumulated per kernel name.  Off by
// default; when off a TraceScope costs one relaxed atomic load.  Launches made
// while the stream is being captured into a graph are not traced (events
// recorded under capture would become graph nodes).
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rlfc_internal.h"

namespace rlfc {
namespace {

struct Pending {
    const char *name;
    cudaEvent_t a, b;
};

struct Totals {
    uint64_t launches = 0;
    double ms = 0.0;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
std::map<std::string, Totals> g_totals;

cudaEvent_t take_event()
{
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// folds finished pairs into the totals; with `wait` it first waits for each
int drain(bool wait)
{
    std::vector<Pending> keep;
    int rc = RLFC_OK;
    for (const Pending &p : g_pending) {
        if (wait) {
            cudaError_t e = cudaEventSynchronize(p.b);
            if (e != cudaSuccess) rc = cuda_fail(e, "trace event");
        }
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            keep.push_back(p);
            continue;
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "trace elapsed time");
        } else {
            Totals &t = g_totals[p.name];
            t.launches += 1;
            t.ms += ms;
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.swap(keep);
    return rc;
}

}  // namespace

TraceScope::TraceScope(const char *name, cudaStream_t st) : name_(name), st_(st)
{
    if (!g_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    b_ = take_event();
    if (!a_ || !b_ || cudaEventRecord(a_, st) != cudaSuccess) {
        if (a_) g_free.push_back(a_);
        if (b_) g_free.push_back(b_);
        a_ = b_ = nullptr;
        cudaGetLastError();
    }
}

TraceScope::~TraceScope()
{
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaEventRecord(b_, st_) != cudaSuccess) {
        cudaGetLastError();
        g_free.push_back(a_);
        g_free.push_back(b_);
        return;
    }
    g_pending.push_back({name_, a_, b_});
    if (g_pending.size() > 4096) drain(false);
}

}  // namespace rlfc

extern "C" {

RLFC_API int rlfc_trace_enable(int on)
{
    rlfc::g_on.store(on != 0);
    return RLFC_OK;
}

RLFC_API int rlfc_trace_read(rlfc_trace_entry *out, size_t cap, size_t *n, int reset)
{
    if (!n || (cap && !out)) {
        rlfc::set_error("rlfc_trace_read: null argument");
        return RLFC_E_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(rlfc::g_mu);
    int rc = rlfc::drain(true);
    size_t k = 0;
    for (const auto &kv : rlfc::g_totals) {
        if (k < cap) {
            std::memset(&out[k], 0, sizeof(out[k]));
            std::strncpy(out[k].kernel, kv.first.c_str(), sizeof(out[k].kernel) - 1);
            out[k].launches = kv.second.launches;
            out[k].total_ms = kv.second.ms;
        }
        ++k;
    }
    *n = k;
    if (reset) rlfc::g_totals.clear();
    return rc;
}

}  // extern "C"
