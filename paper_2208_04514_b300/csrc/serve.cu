// Continuous-batching server (placeholder until the serving loop lands).
#include "dawn_internal.cuh"

extern "C" {

DAWN_API int dawn_serve_create(const dawn_graph_t*, int, size_t, int, dawn_server_t* out) {
    if (out) *out = nullptr;
    return dawn::fail(DAWN_E_STATE, "serving is not available in this build");
}
DAWN_API int dawn_serve_submit(dawn_server_t, int, const int32_t*, int32_t, int, void*, uint64_t*) {
    return dawn::fail(DAWN_E_STATE, "serving is not available in this build");
}
DAWN_API int dawn_serve_poll(dawn_server_t, uint64_t, int*) {
    return dawn::fail(DAWN_E_STATE, "serving is not available in this build");
}
DAWN_API int dawn_serve_drain(dawn_server_t, int64_t) {
    return dawn::fail(DAWN_E_STATE, "serving is not available in this build");
}
DAWN_API int dawn_serve_destroy(dawn_server_t) { return DAWN_OK; }

}  // extern "C"
