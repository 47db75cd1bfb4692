// snap_api.cu — thread-local error messages shared by every entry point.
#include <cstdarg>
#include <cstdio>
#include <cstring>

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

}  // namespace snapgpu

extern "C" const char* snap_last_error(void) { return snapgpu::g_err; }
