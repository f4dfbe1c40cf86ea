// ews_mem.cu -- accounting of the device memory libews allocates, and an
// optional process-wide cap on it.
//
// Every device allocation of the library (simulations, adjoint state,
// checkpoints, history, batch tables, inversion buffers) goes through
// dev_malloc / dev_free.  dev_malloc refuses a request that would take the
// bytes held by the library above the cap (ews_set_memory_limit) before
// asking CUDA, with the same error CUDA gives when the device is full, so
// every caller's out-of-memory path (EWS_ENOMEM, partial set-up released,
// the simulation still usable) runs the same way in both cases.  A service
// that shares its GPU with other work can so bound what the solver takes.
// (ews_forward_noalloc allocates nothing and is not counted.)
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <unordered_map>

#include "ews_internal.cuh"

namespace ews {
namespace {

std::mutex g_mu;
std::unordered_map<void*, size_t> g_live;   // pointer -> bytes
size_t g_in_use = 0;
double g_limit = -1.0;                      // < 0: no cap

}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
    *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_limit >= 0.0 && (double)g_in_use + (double)bytes > g_limit)
            return cudaErrorMemoryAllocation;
        // reserve before the (slow) CUDA call so concurrent requests see it
        g_in_use += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    std::lock_guard<std::mutex> lk(g_mu);
    if (e != cudaSuccess) {
        g_in_use -= bytes;
        *p = nullptr;
        return e;
    }
    g_live[*p] = bytes;
    return cudaSuccess;
}

void dev_free(void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            g_in_use -= it->second;
            g_live.erase(it);
        }
    }
    cudaFree(p);
}

double dev_headroom() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_limit < 0.0) return INFINITY;
    return g_limit > (double)g_in_use ? g_limit - (double)g_in_use : 0.0;
}

}  // namespace ews

extern "C" ews_status ews_set_memory_limit(double bytes) {
    if (std::isnan(bytes)) return ews::report(EWS_EINVAL, "memory limit is NaN");
    std::lock_guard<std::mutex> lk(ews::g_mu);
    ews::g_limit = bytes < 0.0 ? -1.0 : bytes;
    return EWS_OK;
}

extern "C" double ews_memory_limit(void) {
    std::lock_guard<std::mutex> lk(ews::g_mu);
    return ews::g_limit;
}

extern "C" double ews_memory_in_use(void) {
    std::lock_guard<std::mutex> lk(ews::g_mu);
    return (double)ews::g_in_use;
}
