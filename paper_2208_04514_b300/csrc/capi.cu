// Error reporting and small ABI helpers shared by every entry point.
#include <cstdarg>
#include <cstring>

#include "dawn_internal.cuh"

namespace {
thread_local char g_last_error[512] = {0};
}

namespace dawn {

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    fail(DAWN_E_CUDA, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
    if (e == cudaErrorMemoryAllocation) return DAWN_E_NOMEM;
    return DAWN_E_CUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace dawn

extern "C" {

DAWN_API const char* dawn_last_error(void) { return g_last_error; }

DAWN_API int dawn_version(void) { return (0 << 16) | 3; }

}  // extern "C"
