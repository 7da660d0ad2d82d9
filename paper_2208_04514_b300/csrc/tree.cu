// Shortest-path tree: the distances of the level loop plus one predecessor per
// reached vertex.
//
// Fact 1 / Thm 1: v is first reached at level d(v) through an arc (u, v) with
// d(u) = d(v) - 1; every such u is the predecessor of v on some shortest
// path.  Several can qualify, so the tree is fixed by a tie-break: the
// smallest such u.  parent[v] = min { u : (u, v) is an arc, d(u) = d(v) - 1 }
// for d(v) > 0, and -1 for the source and for unreached vertices.
//
// The pass runs after the level loop on the same stream and reads the
// in-adjacency (the CSR itself for symmetric graphs).  When its rows are in
// ascending order (checked at upload) a row scan stops at the first
// qualifying arc; otherwise every in-arc of every reached vertex is read.
//
// Level 2 goes the other way.  Its predecessors are the source's
// out-neighbours, usually few, while on skewed graphs its vertices include
// hubs.  A hub would scan thousands of in-arcs to meet the smallest of those
// few, so the out-rows of the level-1 vertices are pushed instead: every arc
// (u, v) with d(u) = 1 and d(v) = 2 takes an atomic minimum on parent[v].  It
// is the same minimum, reached from the other end of the arcs.  The push is
// taken only while the level-1 rows are a small share of the graph.
#include <algorithm>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

constexpr int kTreeThreads = 1024;
constexpr int kTreeSerial = 8;      // arcs a thread tests by itself
constexpr int kTreeWarpMax = 512;   // rows with more arcs left are scanned by the whole CTA
constexpr int kTreeHeavyMax = 64;   // such rows per CTA and round
constexpr unsigned kNone = 0xffffffffu;
constexpr int kTreePushMax = 2048;  // source rows up to this long push level 2

// One thread per vertex.  A vertex at level 1 hangs on the source (the only
// vertex at level 0).  Otherwise the thread tests the first kTreeSerial arcs
// of its row itself (loads issued four at a time); a row with arcs left is
// scanned 32 arcs per step by its warp, or 1024 per step by the whole CTA
// when more than kTreeWarpMax are left.  With rows in ascending order the
// first qualifying arc is the smallest, so a scan stops at the first step
// that finds one; otherwise the whole row is read.
// Level 2 by push: the out-arcs of the source row's vertices (k of them, the
// arcs [srb, srb + k) of col_idx) split evenly over the grid.  Every CTA
// builds the offsets of those rows in shared memory; vertices other than
// level 1 (the source itself on a self-loop) contribute no arcs.  It runs
// after parent_kernel, which leaves -1 (all bits set) at level 2, so the
// atomic minimum over unsigned values keeps the smallest predecessor.
// Whether level 2 is pushed: the arcs of the level-1 vertices' rows (the
// push reads each once; a repeated arc of the source row counts twice, as
// the push reads it twice) against `limit`.  One CTA.
__global__ void __launch_bounds__(kTreeThreads, 1) level2_decide_kernel(const int32_t* __restrict__ row_ptr,
                                                                        const int32_t* __restrict__ col_idx,
                                                                        const int32_t* __restrict__ dist, int srb,
                                                                        int k, long long limit, int32_t* push2) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0ull;
    __syncthreads();
    unsigned long long sum = 0ull;
    for (int i = threadIdx.x; i < k; i += kTreeThreads) {
        const int u = col_idx[srb + i];
        if (dist[u] == 1) sum += (unsigned long long)(row_ptr[u + 1] - row_ptr[u]);
    }
    if (sum) atomicAdd(&s_sum, sum);
    __syncthreads();
    if (threadIdx.x == 0) *push2 = s_sum <= (unsigned long long)limit ? 1 : 0;
}

__global__ void __launch_bounds__(kTreeThreads, 1) push_level2_kernel(const int32_t* __restrict__ row_ptr,
                                                                      const int32_t* __restrict__ col_idx,
                                                                      const int32_t* __restrict__ dist,
                                                                      int32_t* parent, int srb, int k,
                                                                      const int32_t* __restrict__ push2) {
    if (!*push2) return;  // level2_decide_kernel left level 2 to parent_kernel
    __shared__ long long s_off[kTreePushMax + 1];
    __shared__ int s_u[kTreePushMax], s_rb[kTreePushMax];
    __shared__ long long s_part[kTreeThreads / 32];
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int kPer = kTreePushMax / kTreeThreads;  // rows per thread, consecutive
    long long mine[kPer];
    long long sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int i = threadIdx.x * kPer + q;
        mine[q] = 0;
        if (i < k) {
            const int u = col_idx[srb + i];
            const int rb = row_ptr[u];
            s_u[i] = u;
            s_rb[i] = rb;
            if (dist[u] == 1) mine[q] = row_ptr[u + 1] - rb;
        }
        sum += mine[q];
    }
    // exclusive offsets over the CTA: warp scans, then the warps' totals
    long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_part[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long x = s_part[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        s_part[lane] = x;  // inclusive totals of warps 0..lane
    }
    __syncthreads();
    long long off = (w > 0 ? s_part[w - 1] : 0) + incl - sum;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int i = threadIdx.x * kPer + q;
        if (i < k) s_off[i] = off;
        off += mine[q];
    }
    if (threadIdx.x == kTreeThreads - 1) s_off[k] = off;
    __syncthreads();
    const long long T = s_off[k];
    for (long long t = (long long)blockIdx.x * kTreeThreads + threadIdx.x; t < T;
         t += (long long)gridDim.x * kTreeThreads) {
        int lo = 0, hi = k;  // the last row i with s_off[i] <= t
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= t) lo = mid;
            else hi = mid;
        }
        const int v = col_idx[s_rb[lo] + (int)(t - s_off[lo])];
        if (dist[v] == 2) atomicMin(reinterpret_cast<unsigned*>(parent) + v, (unsigned)s_u[lo]);
    }
}

__global__ void __launch_bounds__(kTreeThreads, 2) parent_kernel(const int32_t* __restrict__ in_ptr,
                                                                 const int32_t* __restrict__ in_idx,
                                                                 const int32_t* __restrict__ dist, int32_t* parent,
                                                                 int32_t n, int32_t src, int sorted,
                                                                 const int32_t* __restrict__ push2) {
    const bool level2_done = push2 && *push2;  // level 2 is left to push_level2_kernel
    const unsigned kFull = 0xffffffffu;
    __shared__ int s_hcount;
    __shared__ int s_hv[kTreeHeavyMax], s_hj[kTreeHeavyMax], s_hie[kTreeHeavyMax], s_hd[kTreeHeavyMax];
    __shared__ unsigned s_hbest[kTreeHeavyMax];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_hcount = 0;
    __syncthreads();
    // the loop bound is the same for the whole CTA
    for (long long base = (long long)blockIdx.x * kTreeThreads; base < n; base += (long long)gridDim.x * kTreeThreads) {
        const long long v0 = base + threadIdx.x;
        const bool valid = v0 < n;
        const int v = (int)v0;
        const int d = valid ? dist[v] : -1;
        unsigned best = kNone;  // smallest qualifying predecessor found so far
        bool done = true;
        int j = 0, ie = 0;
        const bool pushed = level2_done && d == 2;  // -1 here, then push_level2_kernel
        if (d == 1) {
            best = (unsigned)src;
        } else if (d > 1 && !pushed) {
            const int ib = in_ptr[v];
            ie = in_ptr[v + 1];
            const int jl = min(ie, ib + kTreeSerial);
            done = false;
            for (int jb = ib; jb < jl && !done; jb += 4) {
                int u[4], du[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) u[q] = jb + q < jl ? in_idx[jb + q] : -1;
#pragma unroll
                for (int q = 0; q < 4; ++q) du[q] = u[q] >= 0 ? dist[u[q]] : -2;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (du[q] == d - 1 && (unsigned)u[q] < best) best = (unsigned)u[q];
                done = sorted && best != kNone;
            }
            j = jl;
            done = done || j >= ie;
        }
        bool heavy = false;
        if (!done && ie - j > kTreeWarpMax) {
            const int slot = atomicAdd(&s_hcount, 1);
            if (slot < kTreeHeavyMax) {
                heavy = true;
                s_hv[slot] = v;
                s_hj[slot] = j;
                s_hie[slot] = ie;
                s_hd[slot] = d;
                s_hbest[slot] = best;
            }
        }
        unsigned wl = __ballot_sync(kFull, !done && !heavy);
        while (wl) {  // the warp scans one row at a time, 32 arcs per step
            const int sl = __ffs(wl) - 1;
            wl &= wl - 1;
            const int jb = __shfl_sync(kFull, j, sl);
            const int je = __shfl_sync(kFull, ie, sl);
            const int dl = __shfl_sync(kFull, d, sl);
            unsigned m = __shfl_sync(kFull, best, sl);
            for (int j0 = jb; j0 < je; j0 += 32) {
                const int jj = j0 + lane;
                const int u = jj < je ? in_idx[jj] : -1;
                const bool hit = u >= 0 && dist[u] == dl - 1;
                m = min(m, __reduce_min_sync(kFull, hit ? (unsigned)u : kNone));
                if (sorted && m != kNone) break;  // m is the same in every lane
            }
            if (lane == sl) best = m;
        }
        __syncthreads();
        const int nh = min(s_hcount, kTreeHeavyMax);
        for (int h = 0; h < nh; ++h) {  // long rows: the whole CTA, 1024 arcs per step
            const int hie = s_hie[h], hd = s_hd[h];
            for (int j0 = s_hj[h]; j0 < hie; j0 += kTreeThreads) {
                const int jj = j0 + threadIdx.x;
                if (jj < hie) {
                    const int u = in_idx[jj];
                    if (dist[u] == hd - 1) atomicMin(&s_hbest[h], (unsigned)u);
                }
                __syncthreads();
                const bool stop = sorted && s_hbest[h] != kNone;
                __syncthreads();
                if (stop) break;
            }
        }
        if (valid && !heavy) parent[v] = best == kNone || pushed ? -1 : (int)best;
        if (threadIdx.x < nh) parent[s_hv[threadIdx.x]] = s_hbest[threadIdx.x] == kNone ? -1 : (int)s_hbest[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) s_hcount = 0;
        __syncthreads();
    }
}

}  // namespace

int tree_pass(dawn_graph* g, int32_t src, const int32_t* dist_dev, int32_t* parent_dev, cudaStream_t st) {
    if (g->n == 0) return DAWN_OK;
    const long long want = ((long long)g->n + kTreeThreads - 1) / kTreeThreads;
    const int blocks = (int)std::min<long long>(want, 2LL * g->sms);
    const int srb = g->row_ptr_host[src];
    const int k = g->row_ptr_host[src + 1] - srb;
    // Level 2 is pushed when the source row is short and the level-1 rows
    // hold at most an eighth of the arcs (level2_decide_kernel counts them on
    // the device, at least 2^16 allowed); past that the push would read a
    // large share of the graph, and the level-2 vertices' in-row scans, which
    // stop at the first qualifying arc, are left to do it.  parent_kernel leaves -1 at
    // level 2 when the flag is set and push_level2_kernel then takes its
    // atomic minimum over them: the three launches stay on stream `st`, in
    // this order.
    const bool push = k > 0 && k <= kTreePushMax;
    if (push) {
        if (!g->tree_flag) DAWN_CUDA_TRY(cudaMalloc((void**)&g->tree_flag, sizeof(int32_t)));
        const long long limit = std::max<long long>(1LL << 16, (long long)g->m / 8);
        level2_decide_kernel<<<1, kTreeThreads, 0, st>>>(g->row_ptr, g->col_idx, dist_dev, srb, k, limit, g->tree_flag);
        DAWN_CUDA_TRY(cudaGetLastError());
    }
    parent_kernel<<<blocks, kTreeThreads, 0, st>>>(g->in_ptr, g->in_idx, dist_dev, parent_dev, g->n, src,
                                                   g->in_sorted, push ? g->tree_flag : nullptr);
    if (push) {
        DAWN_CUDA_TRY(cudaGetLastError());
        push_level2_kernel<<<g->sms, kTreeThreads, 0, st>>>(g->row_ptr, g->col_idx, dist_dev, parent_dev, srb, k,
                                                            g->tree_flag);
    }
    DAWN_CUDA_TRY(cudaGetLastError());
    return DAWN_OK;
}

}  // namespace dawn

extern "C" {

DAWN_API int dawn_sssp_tree(dawn_graph_t g, int32_t src, int32_t* dist, int32_t* parent, void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!dist || !parent) return fail(DAWN_E_INVALID, "dist / parent is NULL");
    if (src < 0 || src >= g->n) return fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, g->n);
    cudaStream_t st = (cudaStream_t)stream;
    const bool ddev = is_device_ptr(dist), pdev = is_device_ptr(parent);
    int32_t* d = ddev ? dist : g->dist_tmp;
    int32_t* p = parent;
    const size_t bytes = sizeof(int32_t) * (size_t)g->n;
    if (!pdev) DAWN_CUDA_TRY(cudaMallocAsync((void**)&p, bytes, st));
    int rc = sssp_launch(g, src, d, nullptr, g->stats_dev, st);
    if (rc == DAWN_OK) rc = tree_pass(g, src, d, p, st);
    cudaError_t e = cudaSuccess;
    if (rc == DAWN_OK && !ddev) e = cudaMemcpyAsync(dist, d, bytes, cudaMemcpyDeviceToHost, st);
    if (rc == DAWN_OK && e == cudaSuccess && !pdev) e = cudaMemcpyAsync(parent, p, bytes, cudaMemcpyDeviceToHost, st);
    if (rc == DAWN_OK && e != cudaSuccess) rc = cuda_fail(e, "dawn_sssp_tree (copy out)", __FILE__, __LINE__);
    if (!pdev) cudaFreeAsync(p, st);
    const int rs = graph_sync_status(g, st);
    return rc != DAWN_OK ? rc : rs;
}

DAWN_API int dawn_sssp_tree_async(dawn_graph_t g, int32_t src, int32_t* dist_dev, int32_t* parent_dev, void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!dist_dev || !is_device_ptr(dist_dev) || !parent_dev || !is_device_ptr(parent_dev))
        return fail(DAWN_E_INVALID, "dist_dev / parent_dev must be device memory");
    if (src < 0 || src >= g->n) return fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, g->n);
    cudaStream_t st = (cudaStream_t)stream;
    const int rc = sssp_launch(g, src, dist_dev, nullptr, nullptr, st);
    return rc != DAWN_OK ? rc : tree_pass(g, src, dist_dev, parent_dev, st);
}

}  // extern "C"
