// Diagnostic: this GPU's L2 read bandwidth, the denominator for kernels whose
// working set lives in L2 (the batched loop on graphs of a few MB).  A buffer
// that fits in L2 is read repeatedly with 16-byte loads by every SM; the
// first pass brings it in, the timed passes hit L2.
#include <algorithm>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

__global__ void l2_read_kernel(const int4* __restrict__ buf, long long n4, int passes, int* sink) {
    int acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const int4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x7fffffff) *sink = acc;  // keeps the loads; never true for a zeroed buffer
}

}  // namespace
}  // namespace dawn

extern "C" {

DAWN_API int dawn_l2_read_gbs(int64_t bytes, int32_t passes, double* gbs, void* stream) {
    using namespace dawn;
    if (!gbs || bytes < (1 << 20) || passes < 1) return fail(DAWN_E_INVALID, "need bytes >= 1 MiB, passes >= 1, gbs");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    DAWN_CUDA_TRY(cudaGetDevice(&dev));
    DAWN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long n4 = bytes / 16;
    int4* buf = nullptr;
    int* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&buf, (size_t)n4 * 16 + 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, (size_t)n4 * 16, st);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sink, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        const int grid = sms * 4;
        l2_read_kernel<<<grid, 512, 0, st>>>(buf, n4, 2, sink);  // bring the buffer into L2
        cudaEventRecord(e0, st);
        l2_read_kernel<<<grid, 512, 0, st>>>(buf, n4, passes, sink);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "dawn_l2_read_gbs", __FILE__, __LINE__);
    *gbs = (double)n4 * 16.0 * passes / (ms * 1e-3) / 1e9;
    return DAWN_OK;
}

}  // extern "C"
