// Multi-source bit-lane level loop (placeholder until the kernel lands).
#include "dawn_internal.cuh"

extern "C" {

DAWN_API int dawn_msbfs_ex(dawn_graph_t g, const int32_t* sources, int32_t k, void* dist_block,
                           int dist_bytes, int layout, int32_t* ecc, int64_t* dsum, int32_t* reached,
                           const dawn_msbfs_opts* opts, void* stream) {
    (void)g; (void)sources; (void)k; (void)dist_block; (void)dist_bytes; (void)layout;
    (void)ecc; (void)dsum; (void)reached; (void)opts; (void)stream;
    return dawn::fail(DAWN_E_STATE, "dawn_msbfs is not available in this build");
}

DAWN_API int dawn_msbfs(dawn_graph_t g, const int32_t* sources, int32_t k, void* dist_block,
                        int dist_bytes, int layout, int32_t* ecc, int64_t* dsum, void* stream) {
    return dawn_msbfs_ex(g, sources, k, dist_block, dist_bytes, layout, ecc, dsum, nullptr, nullptr, stream);
}

}  // extern "C"
