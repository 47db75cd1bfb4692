// snap_api.cu — thread-local error messages shared by every entry point.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "snap_internal.h"

namespace snapgpu {

static thread_local char g_err[512] = {0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

int cuda_fail(cudaError_t e, const char* what) {
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky launch error where possible
    return (e == cudaErrorMemoryAllocation) ? SNAP_E_NOMEM : SNAP_E_CUDA;
}

// The dynamic shared-memory limit is a property of the kernel for the whole
// process; concurrent callers with different layouts must never lower it under
// each other's launches, so it only grows.
std::recursive_mutex& capture_alloc_mutex() {
    static std::recursive_mutex mu;
    return mu;
}

int raise_smem_limit(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[{dev, func}];
    if (bytes <= cur) return SNAP_OK;
    const cudaError_t e =
        cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory limit");
    cur = bytes;
    return SNAP_OK;
}

}  // namespace snapgpu

extern "C" const char* snap_last_error(void) { return snapgpu::g_err; }
