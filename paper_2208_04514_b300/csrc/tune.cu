// Autotuner: short timed trials of the level loops on one graph; the fastest
// settings are stored in the graph handle and used by later calls whose
// options leave the fields at 0.  Every setting yields the same distances.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

// Mean device time (us) of one source over the sample, or < 0 on failure.
double time_sssp(dawn_graph* g, const std::vector<int32_t>& srcs, int32_t* dist, const dawn_sssp_opts& o,
                 cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int* rc) {
    *rc = DAWN_OK;
    if (cudaEventRecord(e0, st) != cudaSuccess) { *rc = DAWN_E_CUDA; return -1; }
    for (int32_t s : srcs) {
        *rc = sssp_launch(g, s, dist, &o, nullptr, st);
        if (*rc != DAWN_OK) return -1;
    }
    cudaEventRecord(e1, st);
    *rc = graph_sync_status(g, st);
    if (*rc != DAWN_OK) return -1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return 1e3 * (double)ms / (double)srcs.size();
}

}  // namespace
}  // namespace dawn

extern "C" {

DAWN_API int dawn_set_tuning(dawn_graph_t g, const dawn_tuning* t) {
    using namespace dawn;
    if (!g || !t) return fail(DAWN_E_INVALID, "graph / tuning is NULL");
    if (t->alpha < 0 || t->beta < 0 || t->pull_serial < 0 || t->pull_serial > 1024)
        return fail(DAWN_E_INVALID, "tuning fields out of range");
    if (t->lanes != 0 && t->lanes != 64 && t->lanes != 128 && t->lanes != 256)
        return fail(DAWN_E_INVALID, "lanes = %d: need 0, 64, 128 or 256", t->lanes);
    g->tuning = *t;
    return DAWN_OK;
}

DAWN_API int dawn_autotune(dawn_graph_t g, const int32_t* sample, int32_t k, dawn_tuning* out, void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!sample || k < 1) return fail(DAWN_E_INVALID, "need k >= 1 sample sources");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> all((size_t)k);
    DAWN_CUDA_TRY(cudaMemcpy(all.data(), sample, sizeof(int32_t) * (size_t)k, cudaMemcpyDefault));
    for (int32_t i = 0; i < k; ++i)
        if (all[i] < 0 || all[i] >= g->n) return fail(DAWN_E_INVALID, "sample[%d] = %d outside [0, %d)", i, all[i], g->n);
    std::vector<int32_t> srcs(all.begin(), all.begin() + std::min<int32_t>(k, 16));

    int32_t* dist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DAWN_CUDA_TRY(cudaMalloc((void**)&dist, sizeof(int32_t) * (size_t)g->n));
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = DAWN_OK;
    dawn_sssp_opts o;
    std::memset(&o, 0, sizeof(o));
    o.alpha = 15;
    o.beta = 18;
    o.pull_serial = 8;
    // one warm-up pass, then keep the sample small enough for ~2 s of trials
    double best = time_sssp(g, srcs, dist, o, st, e0, e1, &rc);
    if (rc == DAWN_OK) best = time_sssp(g, srcs, dist, o, st, e0, e1, &rc);
    while (rc == DAWN_OK && srcs.size() > 1 && best * srcs.size() * 9 > 2e6) {
        srcs.resize(srcs.size() / 2);
        best = time_sssp(g, srcs, dist, o, st, e0, e1, &rc);
    }
    // coordinate search: pull length, then alpha, then beta
    const int pulls[] = {4, 16, 32};
    const int alphas[] = {4, 30, 60};
    const int betas[] = {6, 54, 150};
    for (int stage = 0; stage < 3 && rc == DAWN_OK; ++stage) {
        for (int i = 0; i < 3 && rc == DAWN_OK; ++i) {
            dawn_sssp_opts c = o;
            if (stage == 0) c.pull_serial = pulls[i];
            else if (stage == 1) c.alpha = alphas[i];
            else c.beta = betas[i];
            const double t = time_sssp(g, srcs, dist, c, st, e0, e1, &rc);
            if (rc == DAWN_OK && t < best) { best = t; o = c; }
        }
    }
    cudaFree(dist);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DAWN_OK) return rc;

    // lanes per pass of the batched loop, on the sample repeated to 1024 sources
    std::vector<int32_t> batch(1024);
    for (size_t i = 0; i < batch.size(); ++i) batch[i] = all[i % all.size()];
    int best_lanes = 256;
    double best_sps = 0.0;
    rc = dawn_msbfs_ex(g, batch.data(), 64, nullptr, 2, DAWN_SOURCE_MAJOR, nullptr, nullptr, nullptr, nullptr, stream);
    if (rc != DAWN_OK) return rc;  // warm-up: work buffers allocated outside the timed trials
    for (int lanes : {256, 128, 64}) {
        dawn_msbfs_opts mo;
        mo.lanes = lanes;
        mo.trace_cap = 0;
        mo.spin_limit = 0;
        mo.trace = nullptr;
        const auto t0 = std::chrono::steady_clock::now();
        rc = dawn_msbfs_ex(g, batch.data(), (int32_t)batch.size(), nullptr, 2, DAWN_SOURCE_MAJOR, nullptr, nullptr,
                           nullptr, &mo, stream);
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (rc != DAWN_OK) return rc;
        const double sps = (double)batch.size() / sec;
        if (sps > best_sps) { best_sps = sps; best_lanes = lanes; }
        if (sec > 1.0) break;  // high-diameter graphs: keep the trials short
    }
    dawn_tuning t;
    t.alpha = o.alpha;
    t.beta = o.beta;
    t.pull_serial = o.pull_serial;
    t.lanes = best_lanes;
    t.sssp_us = best;
    t.msbfs_sources_per_s = best_sps;
    g->tuning = t;
    if (out) *out = t;
    return DAWN_OK;
}

}  // extern "C"
