// Device graph store: CSR upload, validation, in-adjacency (CSC) build and the
// per-graph work buffers of the single-source level loop.
//
// The paper's BOVM (Alg. 1) reads the CSC and SOVM (Alg. 3) the CSR (Sec. 3.3:
// "SOVM operates on CSR matrices, while BOVM operates on CSC matrices").  For a
// symmetric graph both are the same array, so nothing is built.
#include <climits>
#include <cstring>

#include <algorithm>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

constexpr int kThreads = 256;

int grid_for(int64_t work, int sms) {
    int64_t b = (work + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sms * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// bad[0]: smallest bad row_ptr index; bad[1]: smallest bad col_idx index.
__global__ void validate_csr_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    int32_t n, long long m, unsigned long long* bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = t0; i <= n; i += stride) {
        int v = rp[i];
        bool ok = v >= 0 && v <= m;
        if (i == 0) ok = ok && v == 0;
        else ok = ok && v >= rp[i - 1];
        if (i == n) ok = ok && v == m;
        if (!ok) atomicMin(&bad[0], (unsigned long long)i);
    }
    for (long long j = t0; j < m; j += stride) {
        int c = ci[j];
        if (c < 0 || c >= n) atomicMin(&bad[1], (unsigned long long)j);
    }
}

// ---- symmetry of a graph uploaded as DAWN_SYMMETRIC.  The arc multiset must
// equal its reverse (every arc (u, v) appears as often as (v, u)), since the
// CSR then serves as its own in-adjacency.  One pass adds, over every arc,
// h(u, v) - h(v, u) for two independent 64-bit hashes of the ordered pair
// (mod 2^64): both sums are zero when the multisets are equal, and a graph
// whose multisets differ leaves them both zero with probability about 2^-128.
__device__ __forceinline__ unsigned long long pair_hash(unsigned long long x, unsigned long long seed) {
    // the splitmix64 output function (a published 64-bit mixer) of the pair's key
    x += seed;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}
constexpr unsigned long long kSymSeed1 = 0x9e3779b97f4a7c15ull, kSymSeed2 = 0x6a09e667f3bcc909ull;

// One warp per row (lanes over its arcs); sums[0], sums[1] the two sums.
__global__ void symmetry_sum_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                    unsigned long long* sums) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long s1 = 0, s2 = 0;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        for (int j = rp[u] + lane; j < rp[u + 1]; j += 32) {
            const unsigned long long v = (unsigned)ci[j];
            const unsigned long long fwd = ((unsigned long long)u << 32) | v, rev = (v << 32) | (unsigned long long)u;
            s1 += pair_hash(fwd, kSymSeed1) - pair_hash(rev, kSymSeed1);
            s2 += pair_hash(fwd, kSymSeed2) - pair_hash(rev, kSymSeed2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0 && (s1 | s2)) {
        atomicAdd(&sums[0], s1);
        atomicAdd(&sums[1], s2);
    }
}

// When the sums differ, find a witness: per vertex v, the hash sums of its
// out-neighbours and of its in-neighbours (scattered from every arc) differ
// for some v.  out_h[v] / in_h[v] start at zero.
__global__ void symmetry_vertex_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                       unsigned long long* out_h, unsigned long long* in_h) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        unsigned long long s = 0;
        for (int j = rp[u] + lane; j < rp[u + 1]; j += 32) {
            const int v = ci[j];
            s += pair_hash((unsigned)v, kSymSeed1);
            atomicAdd(&in_h[v], pair_hash((unsigned long long)u, kSymSeed1));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out_h[u] = s;
    }
}

// The smallest vertex whose two sums differ (bad[0]); then, in a second
// launch with that vertex, the smallest arc index j of its row whose head x
// has fewer arcs back to it than the row has to x (bad[1]; a linear scan of
// both rows, an error path only).
__global__ void symmetry_witness_kernel(const unsigned long long* out_h, const unsigned long long* in_h, int32_t n,
                                        unsigned long long* bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (out_h[v] != in_h[v]) atomicMin(&bad[0], (unsigned long long)v);
}

__global__ void symmetry_arc_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int v,
                                    unsigned long long* bad) {
    const int b = rp[v], e = rp[v + 1];
    for (int j = b + (int)(blockIdx.x * blockDim.x + threadIdx.x); j < e; j += gridDim.x * blockDim.x) {
        const int x = ci[j];
        int fwd = 0, back = 0;
        for (int k = b; k < e; ++k) fwd += ci[k] == x;
        for (int k = rp[x]; k < rp[x + 1]; ++k) back += ci[k] == v;
        if (back < fwd) atomicMin(&bad[1], (unsigned long long)j);
    }
}

// No out-arc of v lacks its reverse: then an arc (y, v) into v does.  Every
// row y is scanned for arcs into v (one warp per row); an arc j = (y, v) with
// more copies in row y than arcs back from v to y is a witness (bad[1]).
__global__ void symmetry_in_arc_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                       int v, unsigned long long* bad) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long y = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; y < n; y += nw) {
        for (int j = rp[y] + lane; j < rp[y + 1]; j += 32) {
            if (ci[j] != v) continue;
            int fwd = 0, back = 0;
            for (int k = rp[y]; k < rp[y + 1]; ++k) fwd += ci[k] == v;
            for (int k = rp[v]; k < rp[v + 1]; ++k) back += ci[k] == (int)y;
            if (back < fwd) atomicMin(&bad[1], (unsigned long long)j);
        }
    }
}

__global__ void indegree_kernel(const int32_t* __restrict__ ci, long long m, int32_t* indeg) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride)
        atomicAdd(&indeg[ci[j]], 1);
}

// Exclusive scan of x[0..n) into y[0..n], y[0] = 0, in three kernels:
// per-block scan, one-block scan of the block totals, add-back.
constexpr int kScanBlock = 1024;

__global__ void scan_blocks_kernel(const int32_t* __restrict__ x, int32_t n, int32_t* y, int32_t* sums) {
    __shared__ int32_t warp_tot[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    int v = i < n ? x[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int s = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) warp_tot[w] = s;
    __syncthreads();
    if (w == 0) {
        int t = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (w > 0) s += warp_tot[w - 1];
    if (i < n) y[i + 1] = s;  // inclusive value lands one slot to the right
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = s;
}

__global__ void scan_sums_kernel(int32_t* sums, int32_t nb) {
    __shared__ int32_t carry_s;
    __shared__ int32_t warp_tot[32];
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += kScanBlock) {
        int i = base + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        int s = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane == 31) warp_tot[w] = s;
        __syncthreads();
        if (w == 0) {
            int t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        if (w > 0) s += warp_tot[w - 1];
        int carry = carry_s;
        if (i < nb) sums[i] = carry + s - v;  // exclusive block offsets
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry_s = carry + s;
        __syncthreads();
    }
}

__global__ void scan_add_kernel(int32_t* y, int32_t n, const int32_t* __restrict__ sums) {
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) y[i + 1] += sums[blockIdx.x];
    if (i == 0) y[0] = 0;
}

// Scatter every arc u -> c into column c of the CSC; one warp per row.
__global__ void csc_scatter_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   int32_t n, int32_t* cursor, int32_t* in_idx) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nwarps) {
        for (int j = rp[u] + lane; j < rp[u + 1]; j += 32) {
            int pos = atomicAdd(&cursor[ci[j]], 1);
            in_idx[pos] = (int32_t)u;
        }
    }
}

// excl bit v = (v >= n) or v has no in-arc: such a vertex is never reached
// from another vertex, so the pull step never scans it.
// Pull order: a copy of the in-adjacency whose rows are ordered by the
// neighbour's out-degree, largest first (smallest id on ties).  Pull levels
// stop at the first reached in-neighbour, and on skewed graphs the
// high-degree vertices are reached in the first levels, so this order makes
// the stop come early.  Key of an arc: (~out-degree, id), sorted ascending.
__device__ __forceinline__ unsigned long long pull_key(const int32_t* __restrict__ row_ptr, int u) {
    return ((unsigned long long)(0xffffffffu - (unsigned)(row_ptr[u + 1] - row_ptr[u])) << 32) | (unsigned)u;
}

// Rows of at most 32 arcs: one warp per row, bitonic sort in registers.
__global__ void pull_order_warp_kernel(const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ in_idx,
                                       const int32_t* __restrict__ row_ptr, int32_t n, int32_t* out) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
        const int ib = in_ptr[v], len = in_ptr[v + 1] - ib;
        if (len > 32) continue;  // warp-uniform
        unsigned long long key = lane < len ? pull_key(row_ptr, in_idx[ib + lane]) : ~0ull;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, jj);
                const bool up = (lane & k) == 0;
                const bool lower = (lane & jj) == 0;
                const bool take_min = up == lower;
                key = take_min ? (key < other ? key : other) : (key > other ? key : other);
            }
        }
        if (lane < len) out[ib + lane] = (int32_t)(key & 0xffffffffull);
    }
}

// Longer rows: one CTA per row, bitonic sort in shared memory over chunks of
// kPullChunk arcs (rows up to a chunk are fully ordered; longer ones chunk by chunk).
constexpr int kPullChunk = 2048;
__global__ void pull_order_cta_kernel(const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ in_idx,
                                      const int32_t* __restrict__ row_ptr, int32_t n, int32_t* out) {
    __shared__ unsigned long long sk[kPullChunk];
    for (long long v = blockIdx.x; v < n; v += gridDim.x) {
        const int ib = in_ptr[v], ie = in_ptr[v + 1];
        if (ie - ib <= 32) continue;  // the warp kernel's rows (CTA-uniform)
        for (int cb = ib; cb < ie; cb += kPullChunk) {
            const int len = min(kPullChunk, ie - cb);
            int p2 = 64;
            while (p2 < len) p2 <<= 1;
            for (int i = threadIdx.x; i < p2; i += blockDim.x) sk[i] = i < len ? pull_key(row_ptr, in_idx[cb + i]) : ~0ull;
            __syncthreads();
            for (int k = 2; k <= p2; k <<= 1) {
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                        const int ixj = i ^ jj;
                        if (ixj > i) {
                            const unsigned long long x = sk[i], y = sk[ixj];
                            const bool up = (i & k) == 0;
                            if ((x > y) == up) {
                                sk[i] = y;
                                sk[ixj] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int i = threadIdx.x; i < len; i += blockDim.x) out[cb + i] = (int32_t)(sk[i] & 0xffffffffull);
            __syncthreads();
        }
    }
}

// Connected components of a symmetric graph (lock-free union-find): every
// vertex starts as its own root; each arc u -> v with v < u links the two
// roots, the larger under the smaller, by compare-and-swap (so no cycle can
// form), finds halving paths as they go; a final pass points every vertex
// at its root.  The level loop uses the component sizes: on a symmetric
// graph the vertices reachable from s are exactly s's component.
__device__ int cc_find(int* p, int v) {
    while (true) {
        const int q = p[v];
        if (q == v) return v;
        const int r = p[q];
        if (r != q) p[v] = r;  // path halving (a stale write only lengthens a later walk)
        v = q;
    }
}

__global__ void cc_init_kernel(int* p, int32_t n) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        p[v] = (int)v;
}

// one warp per vertex, lanes over its row
__global__ void cc_hook_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n, int* p) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        for (int j = rp[u] + lane; j < rp[u + 1]; j += 32) {
            int a = (int)u, b = ci[j];
            if (b >= a) continue;
            while (true) {
                int ra = cc_find(p, a), rb = cc_find(p, b);
                if (ra == rb) break;
                if (ra < rb) { const int t = ra; ra = rb; rb = t; }
                const int old = atomicCAS(p + ra, ra, rb);
                if (old == ra) break;
                a = ra;  // ra gained a parent meanwhile: retry from there
                b = rb;
            }
        }
    }
}

__global__ void cc_count_kernel(int* p, int32_t n, int32_t* size) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int r = cc_find(p, (int)v);
        atomicAdd(size + r, 1);
    }
}

__global__ void cc_size_kernel(int* p, int32_t n, const int32_t* size, int32_t* csize) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        csize[v] = size[cc_find(p, (int)v)];
}

// first2[v] = the first two in-neighbours of v in pull order (-1 past the row's
// end): a pull tests them from one coalesced load per warp, before any
// scattered read of the row itself.
__global__ void first2_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, int32_t n,
                              int2* __restrict__ first2) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int b = ptr[v], e = ptr[v + 1];
        first2[v] = make_int2(e > b ? idx[b] : -1, e > b + 1 ? idx[b + 1] : -1);
    }
}

// flag = 1 when some in-adjacency row is not in ascending order (one warp per row).
__global__ void unsorted_rows_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, int32_t n,
                                     int* flag) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
        const int ib = ptr[v], ie = ptr[v + 1];
        bool bad = false;
        for (int j = ib + lane; j + 1 < ie; j += 32) bad |= idx[j] > idx[j + 1];
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) *flag = 1;
        }
    }
}

__global__ void excl_kernel(const int32_t* __restrict__ in_ptr, int32_t n, int32_t nwords, uint32_t* excl) {
    const int stride = gridDim.x * blockDim.x;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += stride) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            long long v = (long long)w * 32 + b;
            if (v >= n || in_ptr[v + 1] == in_ptr[v]) bits |= 1u << b;
        }
        excl[w] = bits;
    }
}

int exclusive_scan(const int32_t* x, int32_t n, int32_t* y, cudaStream_t st) {
    int32_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb < 1) nb = 1;
    int32_t* sums = nullptr;
    DAWN_CUDA_TRY(cudaMallocAsync((void**)&sums, sizeof(int32_t) * nb, st));
    scan_blocks_kernel<<<nb, kScanBlock, 0, st>>>(x, n, y, sums);
    scan_sums_kernel<<<1, kScanBlock, 0, st>>>(sums, nb);
    scan_add_kernel<<<nb, kScanBlock, 0, st>>>(y, n, sums);
    DAWN_CUDA_TRY(cudaGetLastError());
    DAWN_CUDA_TRY(cudaFreeAsync(sums, st));
    return DAWN_OK;
}

void release(dawn_graph* g) {
    if (!g) return;
    auto f = [](void* p) { if (p) cudaFree(p); };
    f(g->row_ptr);
    f(g->col_idx);
    if (g->in_ptr != g->row_ptr) f(g->in_ptr);
    if (g->in_idx != g->col_idx) f(g->in_idx);
    f(g->excl);
    f(g->vis[0]);
    f(g->vis[1]);
    f(g->queue[0]);
    f(g->queue[1]);
    f(g->queue_off[0]);
    f(g->queue_off[1]);
    f(g->dist_tmp);
    f(g->pull_idx);
    f(g->first2);
    f(g->cand[0]);
    f(g->cand[1]);
    f(g->cl_ovf);
    f(g->cl_ovf_n);
    many_release(g);
    weighted_release(g);
    f(g->ctl);
    f(g->stats_dev);
    f(g->ms_vis[0]);
    f(g->ms_vis[1]);
    f(g->ms_acc);
    f(g->ms_scratch);
    f(g->ms_counts);
    ms_release(g);
    f(g->tree_flag);
    if (g->stats_host) cudaFreeHost(g->stats_host);
    if (g->status_host) cudaFreeHost(g->status_host);
    delete g;
}

// DAWN_E_INVALID, naming a witness, when the graph's arc multiset differs
// from its reverse (see symmetry_sum_kernel).
int check_symmetric(dawn_graph* g, cudaStream_t st) {
    unsigned long long* buf = nullptr;
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMallocAsync((void**)&buf, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        symmetry_sum_kernel<<<grid_for((int64_t)g->n * 32, g->sms), kThreads, 0, st>>>(g->row_ptr, g->col_idx, g->n, buf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, buf, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (buf) cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "symmetry check", __FILE__, __LINE__);
    if (h[0] == 0 && h[1] == 0) return DAWN_OK;
    // locate a witness (error path)
    unsigned long long* vh = nullptr;
    unsigned long long bad[2] = {ULLONG_MAX, ULLONG_MAX};
    const size_t nb = sizeof(unsigned long long) * (size_t)g->n;
    e = cudaMallocAsync((void**)&vh, 2 * nb + 2 * sizeof(unsigned long long), st);
    unsigned long long* badd = vh ? vh + 2 * (size_t)g->n : nullptr;
    if (e == cudaSuccess) e = cudaMemsetAsync(vh, 0, 2 * nb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(badd, 0xff, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        symmetry_vertex_kernel<<<grid_for((int64_t)g->n * 32, g->sms), kThreads, 0, st>>>(g->row_ptr, g->col_idx, g->n,
                                                                                         vh, vh + g->n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        symmetry_witness_kernel<<<grid_for(g->n, g->sms), kThreads, 0, st>>>(vh, vh + g->n, g->n, badd);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, badd, sizeof(bad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int32_t vb[2] = {0, 0};
    if (e == cudaSuccess && bad[0] != ULLONG_MAX)
        e = cudaMemcpy(vb, g->row_ptr + bad[0], 2 * sizeof(int32_t), cudaMemcpyDeviceToHost);
    // the arc search scans the row once per arc: only on rows of modest length
    if (e == cudaSuccess && bad[0] != ULLONG_MAX && vb[1] - vb[0] <= 4096) {
        symmetry_arc_kernel<<<8, kThreads, 0, st>>>(g->row_ptr, g->col_idx, (int)bad[0], badd);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(bad, badd, sizeof(bad), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess && bad[0] != ULLONG_MAX && bad[1] == ULLONG_MAX && vb[1] - vb[0] <= 4096) {
        symmetry_in_arc_kernel<<<grid_for((int64_t)g->n * 32, g->sms), kThreads, 0, st>>>(g->row_ptr, g->col_idx, g->n,
                                                                                         (int)bad[0], badd);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(bad, badd, sizeof(bad), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (vh) cudaFreeAsync(vh, st);
    if (e != cudaSuccess) return cuda_fail(e, "symmetry witness", __FILE__, __LINE__);
    if (bad[1] != ULLONG_MAX) {
        // the arc's tail: the row holding col_idx[bad[1]]
        std::vector<int32_t> rp((size_t)g->n + 1);
        int32_t x = -1;
        long long y = -1;
        if (cudaMemcpy(rp.data(), g->row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost) == cudaSuccess &&
            cudaMemcpy(&x, g->col_idx + bad[1], sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess)
            y = (long long)(std::upper_bound(rp.begin(), rp.end(), (int32_t)bad[1]) - rp.begin()) - 1;
        return fail(DAWN_E_INVALID,
                    "DAWN_SYMMETRIC: arc (%lld, %d) (col_idx[%llu]) has no matching reverse arc; upload it as DAWN_DIRECTED",
                    y, x, bad[1]);
    }
    if (bad[0] != ULLONG_MAX)
        return fail(DAWN_E_INVALID,
                    "DAWN_SYMMETRIC: the arcs into vertex %llu differ from the arcs out of it; upload it as DAWN_DIRECTED",
                    bad[0]);
    return fail(DAWN_E_INVALID, "DAWN_SYMMETRIC: the arc multiset differs from its reverse; upload it as DAWN_DIRECTED");
}

int upload(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t m, uint32_t flags,
           cudaStream_t st, dawn_graph** out) {
    dawn_graph* g = new dawn_graph();
    g->n = n;
    g->m = m;
    g->flags = flags;
    g->nwords = (int32_t)(((int64_t)n + 31) / 32);
    DAWN_CUDA_TRY(cudaGetDevice(&g->device));
    DAWN_CUDA_TRY(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device));
    const size_t mb = sizeof(int32_t) * (size_t)(m > 0 ? m : 1);
    // words rounded up to a multiple of 4 so that 16-byte vector access stays in bounds
    const size_t wb = sizeof(uint32_t) * (size_t)((g->nwords + 3) / 4 * 4);
    auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes); };
    cudaError_t e = cudaSuccess;
    if ((e = alloc((void**)&g->row_ptr, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess ||
        (e = alloc((void**)&g->col_idx, mb)) != cudaSuccess) {
        release(g);
        return cuda_fail(e, "cudaMalloc(csr)", __FILE__, __LINE__);
    }
    e = cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDefault, st);
    if (e == cudaSuccess && m > 0)
        e = cudaMemcpyAsync(g->col_idx, col_idx, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, st);
    if (e != cudaSuccess) { release(g); return cuda_fail(e, "cudaMemcpyAsync(csr)", __FILE__, __LINE__); }

    // ---- validation on the device
    unsigned long long* bad = nullptr;
    unsigned long long bad_h[2];
    e = cudaMallocAsync((void**)&bad, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        validate_csr_kernel<<<grid_for((int64_t)n + 1 > m ? (int64_t)n + 1 : m, g->sms), kThreads, 0, st>>>(
            g->row_ptr, g->col_idx, n, (long long)m, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad_h, bad, sizeof(bad_h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (bad) cudaFreeAsync(bad, st);
    if (e != cudaSuccess) { release(g); return cuda_fail(e, "validate", __FILE__, __LINE__); }
    if (bad_h[0] != ULLONG_MAX) {
        release(g);
        return fail(DAWN_E_INVALID, "row_ptr[%llu] breaks row_ptr[0] = 0 <= ... <= row_ptr[n] = m", bad_h[0]);
    }
    if (bad_h[1] != ULLONG_MAX) {
        release(g);
        return fail(DAWN_E_INVALID, "col_idx[%llu] is outside [0, n)", bad_h[1]);
    }

    // ---- a symmetric upload must be symmetric: the CSR stands in for the CSC
    if ((flags & DAWN_SYMMETRIC) && m > 0) {
        const int rc = check_symmetric(g, st);
        if (rc != DAWN_OK) {
            release(g);
            return rc;
        }
    }

    // ---- in-adjacency
    if (flags & DAWN_SYMMETRIC) {
        g->in_ptr = g->row_ptr;
        g->in_idx = g->col_idx;
    } else {
        int32_t* indeg = nullptr;
        int32_t* cursor = nullptr;
        if ((e = alloc((void**)&g->in_ptr, sizeof(int32_t) * ((size_t)n + 1))) != cudaSuccess ||
            (e = alloc((void**)&g->in_idx, mb)) != cudaSuccess ||
            (e = cudaMallocAsync((void**)&indeg, sizeof(int32_t) * (size_t)n, st)) != cudaSuccess) {
            release(g);
            return cuda_fail(e, "cudaMalloc(csc)", __FILE__, __LINE__);
        }
        e = cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (size_t)n, st);
        if (e == cudaSuccess && m > 0) {
            indegree_kernel<<<grid_for(m, g->sms), kThreads, 0, st>>>(g->col_idx, (long long)m, indeg);
            e = cudaGetLastError();
        }
        int rc = e == cudaSuccess ? exclusive_scan(indeg, n, g->in_ptr, st) : DAWN_OK;
        if (e == cudaSuccess && rc == DAWN_OK) {
            // reuse indeg as the scatter cursor: cursor[c] = in_ptr[c]
            cursor = indeg;
            e = cudaMemcpyAsync(cursor, g->in_ptr, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && m > 0) {
                csc_scatter_kernel<<<grid_for((int64_t)n * 32, g->sms), kThreads, 0, st>>>(
                    g->row_ptr, g->col_idx, n, cursor, g->in_idx);
                e = cudaGetLastError();
            }
        }
        cudaFreeAsync(indeg, st);
        if (rc != DAWN_OK) { release(g); return rc; }
        if (e != cudaSuccess) { release(g); return cuda_fail(e, "csc build", __FILE__, __LINE__); }
    }

    // ---- work buffers of the single-source level loop
    g->queue_cap = (int64_t)n + m / kEntryArcs + 64;
    // each CTA of the level loop owns ceil(words / warps) words per warp of the
    // grid's bitmap; with at most 2 CTAs of 32 warps per SM this bounds the lists
    g->cand_cap = (int64_t)n + 64 + (int64_t)g->sms * 2 * 32 * 32;
    if ((e = alloc((void**)&g->excl, wb)) != cudaSuccess ||
        (e = alloc((void**)&g->vis[0], wb)) != cudaSuccess ||
        (e = alloc((void**)&g->vis[1], wb)) != cudaSuccess ||
        (e = alloc((void**)&g->queue[0], sizeof(int2) * (size_t)g->queue_cap)) != cudaSuccess ||
        (e = alloc((void**)&g->queue[1], sizeof(int2) * (size_t)g->queue_cap)) != cudaSuccess ||
        (e = alloc((void**)&g->queue_off[0], sizeof(int32_t) * (size_t)g->queue_cap)) != cudaSuccess ||
        (e = alloc((void**)&g->queue_off[1], sizeof(int32_t) * (size_t)g->queue_cap)) != cudaSuccess ||
        (e = alloc((void**)&g->dist_tmp, sizeof(int32_t) * (size_t)n)) != cudaSuccess ||
        // rounded up to whole 16-byte groups: the pull levels read it with aligned int4 loads
        (e = alloc((void**)&g->pull_idx, sizeof(int32_t) * (size_t)((m + 3) / 4 * 4 + 4))) != cudaSuccess ||
        (e = alloc((void**)&g->first2, sizeof(int2) * (size_t)n)) != cudaSuccess ||
        (e = alloc((void**)&g->cand[0], sizeof(int32_t) * (size_t)g->cand_cap)) != cudaSuccess ||
        (e = alloc((void**)&g->cand[1], sizeof(int32_t) * (size_t)g->cand_cap)) != cudaSuccess ||
        (e = alloc((void**)&g->ctl, sizeof(Ctl))) != cudaSuccess ||
        (e = alloc((void**)&g->stats_dev, sizeof(dawn_sssp_stats))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&g->stats_host, sizeof(dawn_sssp_stats))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&g->status_host, sizeof(int))) != cudaSuccess) {
        release(g);
        return cuda_fail(e, "cudaMalloc(work buffers)", __FILE__, __LINE__);
    }
    e = cudaMemsetAsync(g->excl, 0, wb, st);
    if (e == cudaSuccess) {
        excl_kernel<<<grid_for(g->nwords, g->sms), kThreads, 0, st>>>(g->in_ptr, n, g->nwords, g->excl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), st);
    // in-adjacency rows in ascending order let the tree pass stop at the first
    // qualifying predecessor
    int* unsorted = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&unsorted, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(unsorted, 0, sizeof(int), st);
    if (e == cudaSuccess && m > 0) {
        pull_order_warp_kernel<<<grid_for((int64_t)n * 32, g->sms), kThreads, 0, st>>>(g->in_ptr, g->in_idx,
                                                                                       g->row_ptr, n, g->pull_idx);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            pull_order_cta_kernel<<<g->sms * 2, 1024, 0, st>>>(g->in_ptr, g->in_idx, g->row_ptr, n, g->pull_idx);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        first2_kernel<<<grid_for(n, g->sms), kThreads, 0, st>>>(g->in_ptr, g->pull_idx, n, g->first2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && m > 0) {
        unsorted_rows_kernel<<<grid_for((int64_t)n * 32, g->sms), kThreads, 0, st>>>(g->in_ptr, g->in_idx, n,
                                                                                      unsorted);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->status_host, unsorted, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (unsorted) cudaFreeAsync(unsorted, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { release(g); return cuda_fail(e, "graph setup", __FILE__, __LINE__); }
    g->in_sorted = *g->status_host == 0;
    *g->status_host = 0;
    g->row_ptr_host.resize((size_t)n + 1);
    e = cudaMemcpy(g->row_ptr_host.data(), g->row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { release(g); return cuda_fail(e, "graph setup (row_ptr copy)", __FILE__, __LINE__); }
    if (flags & DAWN_SYMMETRIC) {
        // component size per vertex (host copy: it travels as a launch argument)
        int* p = nullptr;
        int32_t* size = nullptr;
        int32_t* csize = nullptr;
        const int grid = grid_for(n, g->sms);
        e = cudaMallocAsync((void**)&p, sizeof(int) * (size_t)n, st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&size, sizeof(int32_t) * (size_t)n, st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&csize, sizeof(int32_t) * (size_t)n, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(size, 0, sizeof(int32_t) * (size_t)n, st);
        if (e == cudaSuccess) {
            cc_init_kernel<<<grid, kThreads, 0, st>>>(p, n);
            cc_hook_kernel<<<grid_for((int64_t)n * 32, g->sms), kThreads, 0, st>>>(g->row_ptr, g->col_idx, n, p);
            cc_count_kernel<<<grid, kThreads, 0, st>>>(p, n, size);
            cc_size_kernel<<<grid, kThreads, 0, st>>>(p, n, size, csize);
            e = cudaGetLastError();
        }
        g->csize_host.resize((size_t)n);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->csize_host.data(), csize, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
        if (p) cudaFreeAsync(p, st);
        if (size) cudaFreeAsync(size, st);
        if (csize) cudaFreeAsync(csize, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { release(g); return cuda_fail(e, "graph setup (components)", __FILE__, __LINE__); }
    }
    int rc = sssp_occupancy(g);
    if (rc != DAWN_OK) { release(g); return rc; }
    *out = g;
    return DAWN_OK;
}

}  // namespace

int graph_sync_status(dawn_graph* g, cudaStream_t st) {
    DAWN_CUDA_TRY(cudaMemcpyAsync(g->status_host, &g->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DAWN_CUDA_TRY(cudaStreamSynchronize(st));
    int s = *g->status_host;
    if (s == DEV_OK) return DAWN_OK;
    // clear the sticky word and the barrier state a timed-out launch left behind
    DAWN_CUDA_TRY(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), st));
    if (weighted_reset(g, st) != DAWN_OK) return DAWN_E_CUDA;
    DAWN_CUDA_TRY(cudaStreamSynchronize(st));
    if (s == DEV_TIMEOUT) return fail(DAWN_E_TIMEOUT, "a grid-barrier wait on the device ran out of its spin budget");
    if (s == DEV_OVERFLOW) return fail(DAWN_E_OVERFLOW, "a distance exceeded the int16 range (32767)");
    return fail(DAWN_E_CUDA, "unknown device status %d", s);
}

}  // namespace dawn

extern "C" {

DAWN_API int dawn_graph_upload(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t m,
                               uint32_t flags, void* stream, dawn_graph_t* out) {
    if (!out) return dawn::fail(DAWN_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!row_ptr || (m > 0 && !col_idx)) return dawn::fail(DAWN_E_INVALID, "row_ptr / col_idx is NULL");
    if (n < 1) return dawn::fail(DAWN_E_INVALID, "n = %d: need n >= 1", n);
    if (m < 0 || m >= (int64_t)INT32_MAX) return dawn::fail(DAWN_E_INVALID, "m = %lld: need 0 <= m < 2^31", (long long)m);
    if (flags & ~DAWN_SYMMETRIC) return dawn::fail(DAWN_E_INVALID, "unknown flags 0x%x", flags);
    return dawn::upload(row_ptr, col_idx, n, m, flags, (cudaStream_t)stream, out);
}

DAWN_API int dawn_graph_free(dawn_graph_t g) {
    dawn::release(g);
    return DAWN_OK;
}

DAWN_API int dawn_graph_info(dawn_graph_t g, int32_t* n, int64_t* m, uint32_t* flags) {
    if (!g) return dawn::fail(DAWN_E_INVALID, "graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (flags) *flags = g->flags;
    return DAWN_OK;
}

DAWN_API int dawn_graph_sync(dawn_graph_t g, void* stream) {
    if (!g) return dawn::fail(DAWN_E_INVALID, "graph is NULL");
    return dawn::graph_sync_status(g, (cudaStream_t)stream);
}

}  // extern "C"
