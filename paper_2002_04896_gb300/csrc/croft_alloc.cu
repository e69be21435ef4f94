// croft_alloc.cu - every device / pinned-host allocation of the library goes through here,
// so that tests can make the k-th allocation fail (host-side fault injection) and check
// that the failing call returns CROFT_ERR_OOM and leaks nothing.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/croft.h"
#include "croft_internal.h"

namespace croft {

static std::atomic<long> g_live{0};       // live allocations made through croft_dev_alloc / croft_host_alloc
static std::atomic<long> g_fail_at{0};    // countdown: the allocation that brings it to 0 fails
static std::atomic<long> g_countdown{0};

static bool inject_failure() {
    if (g_fail_at.load() <= 0) return false;
    if (--g_countdown == 0) {
        g_fail_at = 0;
        return true;
    }
    return false;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live;
    return e;
}

void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    --g_live;
}

cudaError_t host_alloc(void** p, size_t bytes) {
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) ++g_live;
    return e;
}

void host_free(void* p) {
    if (!p) return;
    cudaFreeHost(p);
    --g_live;
}

}  // namespace croft

extern "C" {

void croft_debug_fail_allocation(int k) {
    croft::g_countdown = k;
    croft::g_fail_at = k;
}

long croft_debug_live_allocations(void) { return croft::g_live.load(); }

}  // extern "C"
