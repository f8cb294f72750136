// tg_timing.cu -- optional per-kernel timing of the projector launches.
//
// When enabled (tg_kernel_timing), every launch of the timed kernel classes
// is bracketed by two CUDA events on the launching stream; tg_kernel_timing_read
// waits for them and returns the summed device time and the launch count of
// one class.  Disabled (the default), the launchers record nothing.  The
// events cost a few microseconds per launch, against launches of
// milliseconds to seconds.
#include <atomic>
#include <mutex>
#include <vector>

#include "tg_internal.cuh"

namespace tg {
namespace {

struct Pending {
    int cls;
    cudaEvent_t e0, e1;
};

std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
double g_ms[TG_KT_COUNT] = {};
uint64_t g_count[TG_KT_COUNT] = {};

// Folds completed pairs into the totals (waits for them).
cudaError_t drain_locked() {
    cudaError_t first = cudaSuccess;
    for (const Pending &p : g_pending) {
        cudaError_t e = cudaEventSynchronize(p.e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.e0, p.e1);
        if (e == cudaSuccess) {
            g_ms[p.cls] += ms;
            g_count[p.cls] += 1;
        } else if (first == cudaSuccess) {
            first = e;
        }
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    g_pending.clear();
    return first;
}

}  // namespace

KernelTimer::KernelTimer(int cls, cudaStream_t s) : cls_(cls), s_(s) {
    if (!g_enabled.load(std::memory_order_relaxed) || cls < 0 || cls >= TG_KT_COUNT) return;
    if (cudaEventCreate(&e0_) != cudaSuccess || cudaEventCreate(&e1_) != cudaSuccess ||
        cudaEventRecord(e0_, s_) != cudaSuccess) {
        if (e0_) cudaEventDestroy(e0_);
        if (e1_) cudaEventDestroy(e1_);
        e0_ = e1_ = nullptr;
        cudaGetLastError();
    }
}

KernelTimer::~KernelTimer() {
    if (!e0_) return;
    if (cudaEventRecord(e1_, s_) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0_);
        cudaEventDestroy(e1_);
        return;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    g_pending.push_back({cls_, e0_, e1_});
}

}  // namespace tg

using namespace tg;

extern "C" {

tg_status tg_kernel_timing(int enable) {
    std::lock_guard<std::mutex> lock(g_mu);
    drain_locked();
    for (int c = 0; c < TG_KT_COUNT; ++c) {
        g_ms[c] = 0.0;
        g_count[c] = 0;
    }
    g_enabled.store(enable ? 1 : 0);
    return TG_OK;
}

tg_status tg_kernel_timing_read(int kernel_class, double *ms, uint64_t *launches) {
    if (kernel_class < 0 || kernel_class >= TG_KT_COUNT || !ms || !launches) return TG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    const cudaError_t e = drain_locked();
    *ms = g_ms[kernel_class];
    *launches = g_count[kernel_class];
    return e == cudaSuccess ? TG_OK : TG_ERR_CUDA;
}

}  // extern "C"
