// Many single-source searches in one call: k level loops back to back (the
// SSSP of Alg. 3 / Alg. 1 per source, Sec. 3.3's APSP-by-repetition), each
// writing its own distance row.  For host outputs the rows are staged in two
// device buffers, and the device-to-host copy of source i runs on a copy
// stream while the level loop of source i + 1 runs, so the transfer hides
// behind the computation (pinned host memory is needed for the overlap).
// With device rows the k launches are captured once as a CUDA graph and the
// graph is replayed while the same call repeats.
#include <algorithm>
#include <cstring>
#include <vector>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

// The k launches of a device-row call, captured once as a CUDA graph and
// replayed while the same call repeats (same sources, rows, statistics and
// options).  Consecutive grid launches alternate between two barrier
// counters, so a replay is valid only when the next launch would start on the
// parity the capture started on; the host's launch count then advances by k.
struct ManyGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int32_t> src;
    int32_t* dist = nullptr;
    dawn_sssp_stats* stats = nullptr;
    dawn_sssp_opts opts;
    bool has_opts = false;
    unsigned parity0 = 0;
    unsigned launches = 0;  // grid launches in the graph
};

bool same_opts(const ManyGraph& c, const dawn_sssp_opts* o) {
    if (c.has_opts != (o != nullptr)) return false;
    return !o || std::memcmp(&c.opts, o, sizeof(dawn_sssp_opts)) == 0;
}

// Capture the k launches into a new graph (on a private stream, so that the
// caller's stream may be the legacy default stream).  nullptr when capture
// is not possible; the launch count is then left unchanged.
ManyGraph* capture(dawn_graph* g, const std::vector<int32_t>& src, int32_t* dist, dawn_sssp_stats* stats,
                   const dawn_sssp_opts* opts) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const unsigned before = g->sssp_launches;
    ManyGraph* c = new ManyGraph();
    c->parity0 = before & 1u;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    for (size_t i = 0; ok && i < src.size(); ++i)
        ok = sssp_launch(g, src[i], dist + i * (size_t)g->n, opts, stats ? stats + i : nullptr, cs) == DAWN_OK;
    const bool ended = cudaStreamEndCapture(cs, &graph) == cudaSuccess;
    ok = ok && ended && graph && cudaGraphInstantiate(&c->exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    c->launches = g->sssp_launches - before;
    g->sssp_launches = before;  // nothing ran yet: the count advances when the graph is launched
    if (!ok) {
        cudaGetLastError();
        if (c->exec) cudaGraphExecDestroy(c->exec);
        delete c;
        return nullptr;
    }
    c->src = src;
    c->dist = dist;
    c->stats = stats;
    c->has_opts = opts != nullptr;
    if (opts) c->opts = *opts;
    return c;
}

}  // namespace

void many_release(dawn_graph* g) {
    ManyGraph* c = static_cast<ManyGraph*>(g->many_graph);
    if (c) {
        if (c->exec) cudaGraphExecDestroy(c->exec);
        delete c;
    }
    g->many_graph = nullptr;
}

}  // namespace dawn

extern "C" {

DAWN_API int dawn_sssp_many(dawn_graph_t g, const int32_t* sources, int32_t k, int32_t* dist,
                            dawn_sssp_stats* stats, const dawn_sssp_opts* opts, void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!sources || k < 1) return fail(DAWN_E_INVALID, "need k >= 1 sources (k = %d)", k);
    if (!dist) return fail(DAWN_E_INVALID, "dist is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> src((size_t)k);
    DAWN_CUDA_TRY(cudaMemcpy(src.data(), sources, sizeof(int32_t) * (size_t)k, cudaMemcpyDefault));
    for (int32_t i = 0; i < k; ++i)
        if (src[i] < 0 || src[i] >= g->n) return fail(DAWN_E_INVALID, "sources[%d] = %d outside [0, %d)", i, src[i], g->n);
    const size_t row = (size_t)g->n;
    const bool ddev = is_device_ptr(dist);
    const bool sdev = stats && is_device_ptr(stats);
    // per-source statistics land in device memory first
    dawn_sssp_stats* st_dev = sdev ? stats : nullptr;
    int32_t* stage = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    if (stats && !sdev) e = cudaMallocAsync((void**)&st_dev, sizeof(dawn_sssp_stats) * (size_t)k, st);
    if (e == cudaSuccess && !ddev) {
        e = cudaMallocAsync((void**)&stage, sizeof(int32_t) * 2 * row, st);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
        }
    }
    int rc = e == cudaSuccess ? DAWN_OK : cuda_fail(e, "dawn_sssp_many (set-up)", __FILE__, __LINE__);
    // device rows on the grid engine: replay (or capture) the launches as one CUDA graph
    const bool cluster = (opts && opts->engine == DAWN_ENGINE_CLUSTER) ||
                         ((!opts || opts->engine == DAWN_ENGINE_AUTO) && g->m < 8 * (int64_t)g->n &&
                          (!opts || (opts->mode != DAWN_MODE_PULL && !opts->trace)));
    int32_t direct = k;  // launches issued one by one below
    // several sources on the cluster engine: one launch of as many clusters as
    // the device holds, each taking the next source (host rows go through a
    // device staging block of one row per cluster, copied out per batch)
    if (rc == DAWN_OK && cluster && k > 1) {
        int32_t* srcs_dev = nullptr;
        int32_t* block = nullptr;
        e = cudaMallocAsync((void**)&srcs_dev, sizeof(int32_t) * (size_t)k, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(srcs_dev, src.data(), sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st);
        int crc = e == cudaSuccess ? DAWN_OK : cuda_fail(e, "dawn_sssp_many (sources)", __FILE__, __LINE__);
        if (crc == DAWN_OK && ddev) {
            crc = cluster_launch_many(g, srcs_dev, k, dist, (long long)row, opts, st_dev, st);
        } else if (crc == DAWN_OK) {
            // the batch: one row per cluster the device holds at once (known after the first call)
            const int32_t kb = std::max(1, std::min<int32_t>(k, g->cl_active > 0 ? g->cl_active : 8));
            e = cudaMallocAsync((void**)&block, sizeof(int32_t) * row * (size_t)kb, st);
            if (e != cudaSuccess) crc = cuda_fail(e, "dawn_sssp_many (staging)", __FILE__, __LINE__);
            for (int32_t b0 = 0; crc == DAWN_OK && b0 < k; b0 += kb) {
                const int32_t nb = std::min(kb, k - b0);
                crc = cluster_launch_many(g, srcs_dev + b0, nb, block, (long long)row, opts,
                                          st_dev ? st_dev + b0 : nullptr, st);
                if (crc == DAWN_OK) {
                    e = cudaMemcpyAsync(dist + (size_t)b0 * row, block, sizeof(int32_t) * row * (size_t)nb,
                                        cudaMemcpyDeviceToHost, st);
                    if (e != cudaSuccess) crc = cuda_fail(e, "dawn_sssp_many (rows)", __FILE__, __LINE__);
                }
            }
        }
        if (srcs_dev) cudaFreeAsync(srcs_dev, st);
        if (block) cudaFreeAsync(block, st);
        if (crc == DAWN_OK) direct = 0;
        else if (g->cl_size >= 0 || (opts && opts->engine == DAWN_ENGINE_CLUSTER)) rc = crc;
        // else the cluster engine is unavailable on this graph: one launch per source below
    }
    if (rc == DAWN_OK && direct > 0 && ddev && !cluster && (!stats || sdev)) {
        ManyGraph* c = static_cast<ManyGraph*>(g->many_graph);
        const bool hit = c && c->src == src && c->dist == dist && c->stats == st_dev && same_opts(*c, opts) &&
                         c->parity0 == (g->sssp_launches & 1u);
        if (!hit) {
            many_release(g);
            c = capture(g, src, dist, st_dev, opts);
            g->many_graph = c;
        }
        if (c) {
            e = cudaGraphLaunch(c->exec, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "dawn_sssp_many (graph launch)", __FILE__, __LINE__);
            else g->sssp_launches += c->launches;
            direct = 0;  // every launch is in the graph
        }
    }
    for (int32_t i = 0; i < direct && rc == DAWN_OK; ++i) {
        dawn_sssp_stats* si = st_dev ? st_dev + i : nullptr;
        if (ddev) {
            rc = sssp_launch(g, src[i], dist + (size_t)i * row, opts, si, st);
            continue;
        }
        const int b = i & 1;
        int32_t* buf = stage + (size_t)b * row;
        // the copy of source i - 2 must have read this buffer
        if (i >= 2 && (e = cudaStreamWaitEvent(st, copied[b], 0)) != cudaSuccess) break;
        rc = sssp_launch(g, src[i], buf, opts, si, st);
        if (rc != DAWN_OK) break;
        if ((e = cudaEventRecord(done[b], st)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(cs, done[b], 0)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(dist + (size_t)i * row, buf, sizeof(int32_t) * row, cudaMemcpyDeviceToHost, cs)) !=
            cudaSuccess)
            break;
        if ((e = cudaEventRecord(copied[b], cs)) != cudaSuccess) break;
    }
    if (rc == DAWN_OK && e != cudaSuccess) rc = cuda_fail(e, "dawn_sssp_many", __FILE__, __LINE__);
    if (cs) {
        // the main stream waits for the last copies before the buffers go
        for (int b = 0; b < 2; ++b)
            if (copied[b]) cudaEventRecord(copied[b], cs);
        for (int b = 0; b < 2; ++b)
            if (copied[b]) cudaStreamWaitEvent(st, copied[b], 0);
    }
    if (rc == DAWN_OK && stats && !sdev) {
        e = cudaMemcpyAsync(stats, st_dev, sizeof(dawn_sssp_stats) * (size_t)k, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "dawn_sssp_many (stats)", __FILE__, __LINE__);
    }
    if (stage) cudaFreeAsync(stage, st);
    if (stats && !sdev && st_dev) cudaFreeAsync(st_dev, st);
    const int rs = graph_sync_status(g, st);
    if (cs) cudaStreamDestroy(cs);
    for (int b = 0; b < 2; ++b) {
        if (done[b]) cudaEventDestroy(done[b]);
        if (copied[b]) cudaEventDestroy(copied[b]);
    }
    return rc != DAWN_OK ? rc : rs;
}

}  // extern "C"
