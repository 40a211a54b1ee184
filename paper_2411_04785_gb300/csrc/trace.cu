// trace.cu - per-stage launch counts and CUDA-event timing of the library's
// kernels, recorded on the launching stream (no synchronisation until read).
#include <mutex>
#include <vector>

#include "cc_internal.cuh"

namespace cc {
namespace {

struct Pending {
    int stage;
    cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
cc_stage_time g_acc[CC_STAGE_COUNT];
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

TraceScope::TraceScope(int stage, cudaStream_t s, int kernels) : stage_(stage), s_(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_acc[stage].launches += kernels;
    if (!g_on) return;
    a_ = take_event();
    if (a_ && cudaEventRecord(a_, s_) != cudaSuccess) {
        g_pool.push_back(a_);
        a_ = nullptr;
    }
}

TraceScope::~TraceScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = take_event();
    if (b && cudaEventRecord(b, s_) == cudaSuccess) {
        g_pending.push_back(Pending{stage_, a_, b});
    } else {
        g_pool.push_back(a_);
        if (b) g_pool.push_back(b);
    }
}

}  // namespace cc

using namespace cc;

extern "C" {

cc_status cc_trace_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return CC_OK;
}

cc_status cc_trace_read(cc_stage_time *out, int32_t n, int32_t reset) {
    if (!out || n < 0) return fail(CC_EINVAL, "out must be non-NULL and n >= 0");
    std::lock_guard<std::mutex> lk(g_mu);
    cc_status st = CC_OK;
    for (const Pending &p : g_pending) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) st = cuda_fail(e, "trace event");
        else g_acc[p.stage].ms += ms;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
    for (int i = 0; i < n && i < CC_STAGE_COUNT; i++) out[i] = g_acc[i];
    if (reset)
        for (auto &a : g_acc) a = cc_stage_time{0, 0.0};
    return st;
}

}  // extern "C"
