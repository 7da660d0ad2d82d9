// Multi-source (APSP-style) DAWN: many single-source level loops advanced
// together as bit lanes.
//
// Sec. 3.3 runs APSP as one SSSP per source (cost T < 2 S_wcc E_wcc).  Here
// 64 * W sources share each vertex's W uint64 visited words: bit s of
// V[v][s / 64] says that source s has reached v.  One level is the BOVM pull
// of Alg. 1 / Eq. 4 done for all lanes at once:
//     new[v] = (OR over in-neighbours u of V_start[u]) AND NOT V_start[v]
// against the visited words as they were at the start of the level (the
// merge happens after the whole vertex loop), and every new bit s of v gets
// dist[s][v] = level.  Testing against every reached vertex is exact per lane
// for the same reason as in the single-source pull: an unreached v has
// d_s(v) >= t, a reached u has d_s(u) <= t - 1.
//
// A lane whose level reached nothing is finished (its frontier is empty);
// finished and unused lanes count as covered, so a vertex stops scanning its
// in-neighbours as soon as every still-running lane is covered, and a vertex
// covered for every running lane is skipped.  Both kernels are persistent and
// cooperative: batches, their levels and the per-batch reductions
// (eccentricity = largest finite distance, distance sum, reached count) all
// run in one launch, separated by the bounded grid barrier.
//
// Two kernels compute the same results.  msbfs_kernel (per level) writes each
// distance as its bit appears and counts each level's vertices per lane; it
// handles any depth and serves centrality past 15 levels.  msbfs_sliced_kernel
// (the default, further down) cuts the in-arc rows by in-degree into warp
// tasks, pushes level 1 from the sources, and writes every distance cell once
// per pass from per-level new-bit arrays.
#include <algorithm>
#include <climits>
#include <functional>
#include <queue>
#include <vector>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

constexpr int kMsThreads = 1024;
constexpr int kMsWarps = kMsThreads / 32;
constexpr int kMsMaxLanes = 256;
constexpr int kMsSerial = 8;  // in-neighbours a lane tests before the warp takes over
// In-lists longer than this (after the lane's own tests) are deferred to the
// end of the level and scanned by the whole CTA: a hub's row is split over
// 1024 threads instead of one warp walking it 32 arcs at a time.
constexpr int kMsHeavy = 256;
constexpr int kMsHeavyMax = 64;  // deferred vertices per CTA per level
constexpr unsigned kFull = 0xffffffffu;

struct alignas(128) MsCtl {
    BarCounter bar[2];
    int status;
    int pad[31];
    // per level (t % 3): lanes that reached a vertex (words 0..3), vertices
    // that needed a scan (4) and of those, vertices covered afterwards (5)
    unsigned long long lanes_new[3][6];
};

struct MsArgs {
    const int32_t* __restrict__ in_ptr;
    const int32_t* __restrict__ in_idx;
    const uint32_t* __restrict__ excl;
    const int32_t* __restrict__ sources;  // device, k
    uint64_t* V0;                         // [n][W]
    uint64_t* V1;
    unsigned long long* acc;              // [n][W] per-vertex OR of in-neighbours (dense levels); kept zero
    void* out;                            // distance rows, see layout
    int32_t* ecc;                         // device, k
    long long* dsum;
    int32_t* reached;
    int32_t* part_i;                      // [gridDim][2][kMsMaxLanes]: reached, ecc
    long long* part_l;                    // [gridDim][kMsMaxLanes]: dsum
    MsCtl* ctl;
    long long spin_limit;
    long long out_row_stride;             // source-major: n (elements between rows); vertex-major: k
    int32_t n;
    int32_t k;
    int32_t layout;                       // DAWN_SOURCE_MAJOR or DAWN_VERTEX_MAJOR
    int32_t dist_bytes;
    int32_t per_pass;                     // 1: one block of 64*W rows reused by every pass (no caller block)
    int32_t bar_parity;
    long long* trace;                     // device, may be null: 4 int64 per level
    int32_t trace_cap;
    int32_t nostore;                      // 1: no distance rows at all (reductions only)
    int32_t* ring;                        // device, may be null: [3][kMsMaxLanes] vertices found per level
    double* harm;                         // device, k: harmonic centrality (needs ring)
    double* clos;                         // device, k, may be null: closeness
};

__device__ __forceinline__ unsigned ms_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ms_ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ms_ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Same protocol as the single-source barrier: release-add on the launch's
// arrival counter, acquire polls up to a running target, bounded spin.  With
// `snap`, thread 0 copies nsnap words after the acquire into s_snap for the
// whole CTA (one L2 request per CTA, not one per warp on a hot line).
__device__ bool ms_barrier(MsCtl* ctl, unsigned* count, unsigned& target, long long spin_limit,
                           const unsigned long long* snap = nullptr, int nsnap = 0,
                           unsigned long long* s_snap = nullptr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const long long t0 = clock64();
        unsigned polls = 0;
        while ((int)(ms_ld_acquire(count) - target) < 0) {
            if (clock64() - t0 > spin_limit) {
                atomicCAS(&ctl->status, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
            if ((++polls & 15u) == 0 && ms_ld_relaxed_s32(&ctl->status) != DEV_OK) { ok = 0; break; }
        }
        if (ok)
            for (int i = 0; i < nsnap; ++i) s_snap[i] = ms_ld_relaxed_u64(snap + i);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(kFull, x, o);
    return x;
}

// dist of source (s0 + s) at vertex v.
__device__ __forceinline__ long long dist_index(const MsArgs& a, int s0, int s, int v) {
    if (a.layout == DAWN_SOURCE_MAJOR) return (long long)(a.per_pass ? s : s0 + s) * a.out_row_stride + v;
    return (long long)v * a.out_row_stride + (s0 + s);
}

__device__ __forceinline__ void store_dist(const MsArgs& a, int s0, int s, int v, int value) {
    if (a.nostore) return;
    const long long idx = dist_index(a, s0, s, v);
    if (a.dist_bytes == 2) static_cast<int16_t*>(a.out)[idx] = (int16_t)value;
    else static_cast<int32_t*>(a.out)[idx] = value;
}

// Fill the batch's distance cells with -1.
__device__ void fill_batch(const MsArgs& a, int s0, int kb) {
    if (a.nostore) return;
    const int n = a.n;
    if (a.layout == DAWN_SOURCE_MAJOR) {
        // one row per CTA at a time, 16-byte stores when the row allows it
        for (int s = blockIdx.x; s < kb; s += gridDim.x) {
            char* row = static_cast<char*>(a.out) + dist_index(a, s0, s, 0) * a.dist_bytes;
            const long long bytes = (long long)n * a.dist_bytes;
            if ((reinterpret_cast<uintptr_t>(row) & 15u) == 0 && (bytes & 15) == 0) {
                int4* r4 = reinterpret_cast<int4*>(row);
                for (long long i = threadIdx.x; i < bytes / 16; i += blockDim.x) r4[i] = make_int4(-1, -1, -1, -1);
            } else {
                for (int v = threadIdx.x; v < n; v += blockDim.x) store_dist(a, s0, s, v, -1);
            }
        }
    } else {
        const long long cells = (long long)n * kb;
        const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (long long i = gtid; i < cells; i += (long long)gridDim.x * blockDim.x) {
            const int v = (int)(i / kb), s = (int)(i - (long long)v * kb);
            store_dist(a, s0, s, v, -1);
        }
    }
}

// Dense level, first phase: the in-arcs of the whole CSC are cut into equal
// ranges (a multiple of 32 long), one per warp of the grid.  A warp finds the
// vertex holding its first arc with a 32-ary search over the row pointer,
// keeps a batch of 32 consecutive vertices' row starts in its lanes, and walks
// its range 32 arcs at a time: lane i loads the visited words of the arc's
// source vertex, a segmented OR scan across lanes combines arcs of the same
// target vertex, and the last lane of each segment ORs the result into
// acc[target] (global atomics: a row may span two warps).  Rows of any
// length are split evenly this way; no early exit.
template <int W>
__device__ void dense_accumulate(const MsArgs& a, const uint64_t* vcur) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kMsWarps;
    const long long gw = (long long)blockIdx.x * kMsWarps + (threadIdx.x >> 5);
    const int n = a.n;
    const long long M = __ldg(a.in_ptr + n);
    long long chunk = (M + nw - 1) / nw;
    chunk = (chunk + 31) & ~31LL;
    const long long a0 = gw * chunk;
    if (a0 >= M) return;
    const long long a1 = min(M, a0 + chunk);
    int lo = 0, hi = n;  // largest v with in_ptr[v] <= a0 lies in [lo, hi)
    while (hi - lo > 32) {
        const int stp = (hi - lo + 31) >> 5;
        const int p = lo + lane * stp;
        const int val = p < hi ? __ldg(a.in_ptr + p) : INT_MAX;
        const unsigned b = __ballot_sync(kFull, (long long)val <= a0);
        lo += (31 - __clz(b)) * stp;
        hi = min(hi, lo + stp);
    }
    int vb = lo;
    int beg = vb + lane < n ? __ldg(a.in_ptr + vb + lane) : INT_MAX;
    long long endb = __ldg(a.in_ptr + min(n, vb + 32));
    long long r = a0;
    while (r < a1) {
        if (r >= endb) {  // past this batch's rows (empty rows can leave it short of 32 arcs)
            vb += 32;
            beg = vb + lane < n ? __ldg(a.in_ptr + vb + lane) : INT_MAX;
            endb = __ldg(a.in_ptr + min(n, vb + 32));
            continue;
        }
        const int span = (int)min(min(32LL, a1 - r), endb - r);
        const long long tt = r + lane;
        const bool act = lane < span;
        int o = 0;
#pragma unroll
        for (int bb = 16; bb > 0; bb >>= 1) {
            const int cand = o + bb;
            const int pv = __shfl_sync(kFull, beg, cand);
            if ((long long)pv <= tt) o = cand;
        }
        const int key = act ? vb + o : -1 - lane;
        unsigned long long x[W];
        const int u = act ? __ldg(a.in_idx + tt) : 0;
#pragma unroll
        for (int w = 0; w < W; ++w) x[w] = act ? __ldcg(vcur + (long long)u * W + w) : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int k2 = __shfl_up_sync(kFull, key, d);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const unsigned long long y = __shfl_up_sync(kFull, x[w], d);
                if (lane >= d && k2 == key) x[w] |= y;
            }
        }
        const int knext = __shfl_down_sync(kFull, key, 1);
        if (act && (lane == span - 1 || knext != key)) {
#pragma unroll
            for (int w = 0; w < W; ++w)
                if (x[w]) atomicOr(a.acc + (long long)key * W + w, x[w]);
        }
        r += span;
    }
}

template <int W>
__global__ void __launch_bounds__(kMsThreads, 1) msbfs_kernel(MsArgs a) {
    __shared__ int s_cnt[kMsMaxLanes];
    __shared__ int s_reached[kMsMaxLanes];
    __shared__ int s_ecc[kMsMaxLanes];
    __shared__ long long s_dsum[kMsMaxLanes];
    __shared__ double s_harm[kMsMaxLanes];  // CTA 0: harmonic sums, added level by level
    __shared__ unsigned long long s_newmask[4];
    __shared__ int s_hcount;
    __shared__ int s_hv[kMsHeavyMax], s_hj[kMsHeavyMax], s_hie[kMsHeavyMax];
    __shared__ unsigned long long s_hvv[kMsHeavyMax][W], s_hacc[kMsHeavyMax][W];

    MsCtl* ctl = a.ctl;
    __shared__ unsigned long long s_lanes[6];
    __shared__ int s_need, s_cover;
    __shared__ int s_status;
    if (threadIdx.x == 0) s_status = ms_ld_relaxed_s32(&ctl->status);
    __syncthreads();
    if (s_status != DEV_OK) return;
    unsigned* bar = &ctl->bar[a.bar_parity].count;
    unsigned bar_target = 0;
    int tslot = 0;
    constexpr int L = 64 * W;
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * kMsThreads + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * kMsThreads;
    const int n = a.n;
    const int nbatches = (a.k + L - 1) / L;

    for (int i = threadIdx.x; i < kMsMaxLanes; i += kMsThreads) {
        s_cnt[i] = 0;
        s_reached[i] = 0;
        s_ecc[i] = 0;
        s_dsum[i] = 0;
        s_harm[i] = 0.0;
    }
    if (threadIdx.x < 4) s_newmask[threadIdx.x] = 0;
    if (threadIdx.x == 0) { s_hcount = 0; s_need = 0; s_cover = 0; }

    // This CTA's vertices: a range of whole 32-vertex groups holding about
    // 1/gridDim of the in-arcs (the CSC row pointer is the arc prefix), found
    // once per launch; warps take its groups one at a time from a shared
    // counter, so a warp that drew heavy rows does not hold up the others.
    __shared__ int s_range[2];
    __shared__ int s_next;
    if (threadIdx.x < 2) {
        const long long m_in = __ldg(a.in_ptr + n);
        const long long target = m_in * (blockIdx.x + threadIdx.x) / gridDim.x;
        int lo = 0, hi = n;  // first vertex whose row starts at or after target
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((long long)__ldg(a.in_ptr + mid) < target) lo = mid + 1; else hi = mid;
        }
        if (blockIdx.x + threadIdx.x == gridDim.x) lo = n;
        s_range[threadIdx.x] = ((lo + 31) >> 5) << 5;
    }
    __syncthreads();
    const int cv0 = min(s_range[0], n), cv1 = min(s_range[1], ((n + 31) >> 5) << 5);
    if (threadIdx.x == 0) s_next = cv0;

    for (int b = 0; b < nbatches; ++b) {
        const int s0 = b * L;
        const int kb = min(L, a.k - s0);
        uint64_t* vcur = a.V0;
        uint64_t* vnext = a.V1;
        // ---- batch init: clear visited words and this batch's distances
        for (long long i = gtid; i < (long long)n * W; i += gthreads) vcur[i] = 0ull;
        fill_batch(a, s0, kb);
        if (blockIdx.x == 0 && threadIdx.x < 18) (&ctl->lanes_new[0][0])[threadIdx.x] = 0ull;
        if (!ms_barrier(ctl, bar, bar_target, a.spin_limit)) return;
        // ---- seeds: V[src_s] gets bit s, dist[s][src_s] = 0
        if (gtid < kb) {
            const int s = (int)gtid;
            const int src = __ldg(a.sources + s0 + s);
            atomicOr(reinterpret_cast<unsigned long long*>(&vcur[(long long)src * W + (s >> 6)]), 1ull << (s & 63));
            store_dist(a, s0, s, src, 0);
        }
        if (!ms_barrier(ctl, bar, bar_target, a.spin_limit)) return;

        // lanes that can no longer grow: unused lanes now, finished lanes later
        unsigned long long fin[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int lo = w * 64;
            fin[w] = kb >= lo + 64 ? 0ull : (kb <= lo ? ~0ull : ~0ull << (kb - lo));
        }
        bool dense = true;  // the first level covers almost nothing: arc-parallel
        for (int t = 1;; ++t) {
            if (a.dist_bytes == 2 && t > 32767) {
                if (gtid == 0) atomicCAS(&ctl->status, DEV_OK, DEV_OVERFLOW);
                return;
            }
            if (dense) {
                // arc-parallel phase: every in-arc of the graph once, in equal
                // ranges per warp; then the per-vertex pass below finishes
                dense_accumulate<W>(a, vcur);
                if (!ms_barrier(ctl, bar, bar_target, a.spin_limit)) return;
            }
            // ---- one level: lane = vertex, 32 consecutive vertices per warp
            while (true) {
                int vb = 0;
                if (lane == 0) vb = atomicAdd(&s_next, 32);
                vb = __shfl_sync(kFull, vb, 0);
                if (vb >= cv1) break;
                const int v = vb + lane;
                const bool valid = v < n;
                unsigned long long vv[W], acc[W];
                bool need = false;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    vv[w] = valid ? __ldcg(vcur + (long long)v * W + w) : ~0ull;
                    acc[w] = 0ull;
                    need |= (vv[w] | fin[w]) != ~0ull;
                }
                if (valid && need && ((__ldg(a.excl + (v >> 5)) >> (v & 31)) & 1u)) need = false;
                bool deferred = false;
                if (dense) {
                    // the arc-parallel phase left the OR over v's in-neighbours in
                    // acc_g[v]: take it and leave the slot zero for the next level
                    bool nz = false;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        const unsigned long long x = valid ? __ldcg(a.acc + (long long)v * W + w) : 0ull;
                        acc[w] = need ? x : 0ull;
                        nz |= x != 0ull;
                    }
                    if (nz) {
#pragma unroll
                        for (int w = 0; w < W; ++w) a.acc[(long long)v * W + w] = 0ull;
                    }
                } else {
                    int j = 0, ie = 0;
                    if (need) {
                        const int ib = __ldg(a.in_ptr + v);
                        ie = __ldg(a.in_ptr + v + 1);
                        j = ib;
                        const int jl = min(ie, ib + kMsSerial);
                        for (; j < jl; ++j) {
                            const int u = __ldg(a.in_idx + j);
                            bool all = true;
    #pragma unroll
                            for (int w = 0; w < W; ++w) {
                                acc[w] |= __ldcg(vcur + (long long)u * W + w);
                                all &= (acc[w] | vv[w] | fin[w]) == ~0ull;
                            }
                            if (all) { j = ie; break; }
                        }
                    }
                    if (need && ie - j > kMsHeavy) {
                        const int slot = atomicAdd(&s_hcount, 1);
                        if (slot < kMsHeavyMax) {
                            deferred = true;
                            s_hv[slot] = v;
                            s_hj[slot] = j;
                            s_hie[slot] = ie;
    #pragma unroll
                            for (int w = 0; w < W; ++w) {
                                s_hvv[slot][w] = vv[w];
                                s_hacc[slot][w] = acc[w];
                            }
                        }
                    }
                    unsigned rest = __ballot_sync(kFull, need && !deferred && j < ie);
                    while (rest) {
                        const int src_lane = __ffs(rest) - 1;
                        rest &= rest - 1;
                        const int jb = __shfl_sync(kFull, j, src_lane);
                        const int je = __shfl_sync(kFull, ie, src_lane);
                        unsigned long long accL[W], vvL[W];
    #pragma unroll
                        for (int w = 0; w < W; ++w) {
                            accL[w] = __shfl_sync(kFull, acc[w], src_lane);
                            vvL[w] = __shfl_sync(kFull, vv[w], src_lane);
                        }
                        for (int base = jb; base < je; base += 32) {
                            const int jj = base + lane;
                            const int u = jj < je ? __ldg(a.in_idx + jj) : -1;
                            bool all = true;
    #pragma unroll
                            for (int w = 0; w < W; ++w) {
                                const unsigned long long x = u >= 0 ? __ldcg(vcur + (long long)u * W + w) : 0ull;
                                accL[w] |= warp_or64(x);
                                all &= (accL[w] | vvL[w] | fin[w]) == ~0ull;
                            }
                            if (all) break;
                        }
                        if (lane == src_lane) {
    #pragma unroll
                            for (int w = 0; w < W; ++w) acc[w] = accL[w];
                        }
                    }
                }
                {
                    bool cov = true;
#pragma unroll
                    for (int w = 0; w < W; ++w) cov &= (acc[w] | vv[w] | fin[w]) == ~0ull;
                    const unsigned mn = __ballot_sync(kFull, need && !deferred);
                    const unsigned mc = __ballot_sync(kFull, need && !deferred && cov);
                    if (lane == 0 && mn) {
                        atomicAdd(&s_need, __popc(mn));
                        if (mc) atomicAdd(&s_cover, __popc(mc));
                    }
                }
                // new bits, next visited words, distances, counts
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const unsigned long long nb = (need && !deferred) ? (acc[w] & ~vv[w] & ~fin[w]) : 0ull;
                    if (valid && !deferred) vnext[(long long)v * W + w] = vv[w] | nb;
                    unsigned long long uni = warp_or64(nb);
                    if (lane == 0 && uni) atomicOr(&s_newmask[w], uni);
                    while (uni) {
                        const int bit = __ffsll((long long)uni) - 1;
                        uni &= uni - 1;
                        const bool mine = (nb >> bit) & 1ull;
                        const unsigned m = __ballot_sync(kFull, mine);
                        const int s = w * 64 + bit;
                        if (mine) store_dist(a, s0, s, v, t);
                        if (lane == 0) atomicAdd(&s_cnt[s], __popc(m));
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_next = cv0;  // every warp has left the group loop
            // deferred long in-lists: the whole CTA scans each one
            const int nh = min(s_hcount, kMsHeavyMax);
            for (int h = 0; h < nh; ++h) {
                unsigned long long part[W];
#pragma unroll
                for (int w = 0; w < W; ++w) part[w] = 0ull;
                const int hie = s_hie[h];
                for (int jj = s_hj[h] + threadIdx.x; jj < hie; jj += kMsThreads) {
                    const int u = __ldg(a.in_idx + jj);
#pragma unroll
                    for (int w = 0; w < W; ++w) part[w] |= __ldcg(vcur + (long long)u * W + w);
                }
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    part[w] = warp_or64(part[w]);
                    if (lane == 0 && part[w]) atomicOr(&s_hacc[h][w], part[w]);
                }
            }
            __syncthreads();
            for (int h = threadIdx.x >> 5; h < nh; h += kMsWarps) {
                const int v = s_hv[h];
                unsigned long long nbw[W];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    nbw[w] = s_hacc[h][w] & ~s_hvv[h][w] & ~fin[w];
                    if (lane == w) vnext[(long long)v * W + w] = s_hvv[h][w] | nbw[w];
                    if (lane == 0 && nbw[w]) atomicOr(&s_newmask[w], nbw[w]);
                }
                for (int i = lane; i < L; i += 32) {
                    if ((nbw[i >> 6] >> (i & 63)) & 1ull) {
                        store_dist(a, s0, i, v, t);
                        atomicAdd(&s_cnt[i], 1);
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_hcount = 0;
            // fold this level's counts into the batch accumulators
            for (int s = threadIdx.x; s < L; s += kMsThreads) {
                const int c = s_cnt[s];
                if (c) {
                    s_reached[s] += c;
                    s_dsum[s] += (long long)c * t;
                    s_ecc[s] = t;
                    s_cnt[s] = 0;
                    if (a.ring) atomicAdd(&a.ring[(t % 3) * kMsMaxLanes + s], c);
                }
            }
            if (threadIdx.x < W && s_newmask[threadIdx.x]) {
                atomicOr(&ctl->lanes_new[t % 3][threadIdx.x], s_newmask[threadIdx.x]);
                s_newmask[threadIdx.x] = 0;
            }
            if (threadIdx.x == 32) {
                if (s_need) atomicAdd(&ctl->lanes_new[t % 3][4], (unsigned long long)s_need);
                if (s_cover) atomicAdd(&ctl->lanes_new[t % 3][5], (unsigned long long)s_cover);
                s_need = 0;
                s_cover = 0;
            }
            if (blockIdx.x == 0 && threadIdx.x >= 32 && threadIdx.x < 38)
                ctl->lanes_new[(t + 1) % 3][threadIdx.x - 32] = 0ull;
            if (!ms_barrier(ctl, bar, bar_target, a.spin_limit, ctl->lanes_new[t % 3], 6, s_lanes)) return;
            // harmonic centrality: CTA 0 adds (vertices at distance t) / t per
            // lane, level after level, so the sum runs in ascending distance
            // order whatever the grid; the slot is next used at level t + 3
            if (a.ring && blockIdx.x == 0) {
                int* slot = a.ring + (t % 3) * kMsMaxLanes;
                for (int s = threadIdx.x; s < L; s += kMsThreads) {
                    const int c = __ldcg(slot + s);
                    if (c) {
                        s_harm[s] += (double)c / (double)t;
                        slot[s] = 0;
                    }
                }
            }
            // next level: arc-parallel while most scanned vertices stay uncovered
            // and a good share of the lanes is still growing
            {
                int growing = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) growing += __popcll(s_lanes[w]);
                dense = 2 * s_lanes[5] < s_lanes[4] && 4 * growing > L;
            }
            if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && tslot < a.trace_cap) {
                unsigned long long tnow;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
                long long* r = a.trace + 4 * (long long)tslot;
                r[0] = b;
                r[1] = t;
                r[2] = 0;
                for (int w = 0; w < W; ++w) r[2] += __popcll(s_lanes[w]);
                r[3] = (long long)tnow;
            }
            ++tslot;
            bool done = true;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                fin[w] |= ~s_lanes[w];
                done &= fin[w] == ~0ull;
            }
            uint64_t* tmp = vcur;
            vcur = vnext;
            vnext = tmp;
            if (done) break;
        }
        // ---- batch reductions: per-CTA partials, then one thread per lane
        if (a.ring && blockIdx.x == 0) {
            for (int s = threadIdx.x; s < L; s += kMsThreads) {
                if (s < kb) a.harm[s0 + s] = s_harm[s];
                s_harm[s] = 0.0;
            }
        }
        for (int s = threadIdx.x; s < L; s += kMsThreads) {
            a.part_i[((long long)blockIdx.x * 2 + 0) * kMsMaxLanes + s] = s_reached[s];
            a.part_i[((long long)blockIdx.x * 2 + 1) * kMsMaxLanes + s] = s_ecc[s];
            a.part_l[(long long)blockIdx.x * kMsMaxLanes + s] = s_dsum[s];
            s_reached[s] = 0;
            s_ecc[s] = 0;
            s_dsum[s] = 0;
        }
        if (!ms_barrier(ctl, bar, bar_target, a.spin_limit)) return;
        if (gtid < kb) {
            const int s = (int)gtid;
            int r = 1, e = 0;  // the source itself: reached, distance 0
            long long sum = 0;
            for (int c = 0; c < (int)gridDim.x; ++c) {
                r += __ldcg(a.part_i + ((long long)c * 2 + 0) * kMsMaxLanes + s);
                e = max(e, __ldcg(a.part_i + ((long long)c * 2 + 1) * kMsMaxLanes + s));
                sum += __ldcg(a.part_l + (long long)c * kMsMaxLanes + s);
            }
            a.reached[s0 + s] = r;
            a.ecc[s0 + s] = e;
            a.dsum[s0 + s] = sum;
            if (a.clos) a.clos[s0 + s] = r > 1 ? (double)(r - 1) / (double)sum : 0.0;
        }
        // the next batch's first barrier orders these reads before the partials are rewritten
    }
    if (gtid == 0) ctl->bar[a.bar_parity ^ 1].count = 0;
}

template <int W>
int ms_launch_w(dawn_graph* g, MsArgs& a, cudaStream_t st) {
    dim3 grid(g->sms), block(kMsThreads);
    void* args[] = {&a};
    DAWN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)msbfs_kernel<W>, grid, block, args, 0, st));
    return DAWN_OK;
}

// Device buffers of the batched loop, kept on the graph and grown on demand.
int ms_workspace(dawn_graph* g, int W) {
    if (!g->ms_vis[0] || g->ms_words_cap < W) {
        if (g->ms_vis[0]) cudaFree(g->ms_vis[0]);
        if (g->ms_vis[1]) cudaFree(g->ms_vis[1]);
        g->ms_vis[0] = g->ms_vis[1] = nullptr;
        // room for W = 4; row n stays zero (the sliced kernel's padding arcs point there)
        const size_t bytes = sizeof(uint64_t) * ((size_t)g->n + 1) * 4;
        DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_vis[0], bytes));
        DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_vis[1], bytes));
        DAWN_CUDA_TRY(cudaMemset(g->ms_vis[0], 0, bytes));
        DAWN_CUDA_TRY(cudaMemset(g->ms_vis[1], 0, bytes));
        if (g->ms_acc) cudaFree(g->ms_acc);
        g->ms_acc = nullptr;
        DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_acc, bytes));
        DAWN_CUDA_TRY(cudaMemset(g->ms_acc, 0, bytes));
        g->ms_words_cap = 4;
    }
    if (!g->ms_counts) {
        // partials: [sms][2][256] int32 + [sms][256] int64, then the control block
        const size_t bytes = (size_t)g->sms * kMsMaxLanes * (2 * sizeof(int32_t) + sizeof(long long)) +
                             sizeof(MsCtl) + 256;
        DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_counts, bytes));
        DAWN_CUDA_TRY(cudaMemset(g->ms_counts, 0, bytes));
        g->ms_counts_cap = bytes;
    }
    return DAWN_OK;
}

// ---------------------------------------------------------------------------
// Sliced batched kernel.
//
// The same level, new[v] = (OR over in-neighbours u of V[u]) AND NOT V[v]
// for all 64 * W lanes at once, with the work cut by in-degree once per
// graph (ms_plan_build): vertices are sorted by in-degree, largest first.
//   * a row longer than kSellDeg is a warp task: the warp reads 32
//     consecutive in-arcs at a time and ORs their visited words lane by lane,
//     then across the warp once per task.  Rows longer than the plan's piece
//     length are split into pieces, all given to one CTA; the pieces OR into
//     a shared-memory row that the CTA finishes after its tasks.
//   * the other rows are cut into slices of 32 vertices, one vertex per
//     lane; a slice's in-arcs are stored column by column (arc j of lane i at
//     32 j + i), so each step reads 32 consecutive indices.
// Tasks are split over the CTAs by estimated time and taken by the CTA's
// warps from a shared counter.  A level reads one visited buffer and writes
// the other for every vertex of a task; vertices without in-arcs keep the
// seeded words that both buffers hold.  A vertex is covered once every lane
// still growing has reached it: it can gain no bit in this pass.  A task
// whose vertices were all covered in two consecutive levels has written its
// final words to both buffers and is skipped for the rest of the pass.
//
// Nothing is written per (source, vertex) while the levels run: each level
// t <= nb_levels stores the vertex's new bits in its own array NB[t] (zeroed
// one level ahead, so only nonzero words are stored); later levels OR them
// into bit-sliced planes (plane p = bit p of the level).  After the last
// level each warp turns 32 consecutive vertices' arrays into their distance
// cells, writing every cell of each row once, and reduces them per source
// (reached, distance sum, largest distance) after a 32 x 32 bit transpose of
// the level bits puts one source in each lane.
// ---------------------------------------------------------------------------
constexpr int kSellDeg = 16;     // in-degree of the one-vertex-per-lane class
constexpr int kHubMax = 128;     // rows split into pieces, per CTA
constexpr int kPieceMin = 256;   // arcs of a row piece, at least
constexpr int kTaskSmem = 1536;  // tasks a CTA keeps in shared memory (and may skip)
constexpr int kTrip = 4;         // a dependent memory round trip, in warp steps of 32 arcs
constexpr int kNbLevelsMax = 15; // levels with their own new-bit array
constexpr int kPlanesMax = 15;   // levels up to 32767
constexpr size_t kNbBudget = 1ull << 30;      // device bytes for the new-bit arrays
constexpr size_t kPlanesBudget = 8ull << 30;  // and for the planes of deeper levels

struct MsPlan {
    int sms = 0;
    int32_t ntasks = 0, nhubs = 0, nslices = 0, piece = 0, max_hubs = 0, max_tasks = 0;
    long long sell_len = 0;
    void* blob = nullptr;        // one device allocation holding the arrays below
    int4* tasks = nullptr;       // piece {v, first arc, end arc, -1 or CTA slot | pieces << 8}; slice {-1 - id, offset, width, 0}
    int32_t* cta_task = nullptr; // [sms + 1]: CTA c runs tasks [cta_task[c], cta_task[c + 1])
    int32_t* cta_hub = nullptr;  // [sms + 1]: and owns split rows [cta_hub[c], cta_hub[c + 1]) of hub_v
    int32_t* hub_v = nullptr;
    int2* sell_vd = nullptr;     // [nslices * 32]: {vertex or -1, in-degree}
    int32_t* sell_idx = nullptr; // slice columns; entries past a vertex's degree hold -1
};

struct MsSliced {
    const int32_t* __restrict__ out_ptr;  // CSR: level 1 pushes along the sources' out-arcs
    const int32_t* __restrict__ out_idx;
    const int4* __restrict__ tasks;
    const int32_t* __restrict__ cta_task;
    const int32_t* __restrict__ cta_hub;
    const int32_t* __restrict__ hub_v;
    const int2* __restrict__ sell_vd;
    const int32_t* __restrict__ sell_idx;
    uint64_t* nbl;               // NB[t] of vertex v (1 <= t <= nb_levels): nbl + ((t - 1) * (n + 1) + v) * W
    uint64_t* planes;            // plane p of vertex v: planes + (p * (n + 1) + v) * W; may be null
    int32_t nb_levels;
    int32_t planes_cap;          // levels below 2^planes_cap fit (0: planes absent)
    int32_t* hist;               // harmonic centrality: [kNbLevelsMax + 1][kMsMaxLanes] vertices per level of
                                 // the pass (null: not wanted); zero between passes
};

__device__ __forceinline__ unsigned long long warp_or_redux(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(kFull, (unsigned)x);
    const unsigned hi = __reduce_or_sync(kFull, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Lane j receives column j of the 32 x 32 bit matrix whose row i lane i holds.
__device__ __forceinline__ unsigned bit_transpose32(unsigned x) {
    const int lane = threadIdx.x & 31;
    constexpr unsigned kMask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int k = 16 >> i;
        const unsigned m = kMask[i];
        const unsigned y = __shfl_xor_sync(kFull, x, k);
        x = (lane & k) ? ((x & ~m) | ((y & ~m) >> k)) : ((x & m) | ((y & m) << k));
    }
    return x;
}

// W visited words of one vertex.  The visited buffers are written during the
// launch, so reads go to L2 (a CTA could otherwise keep an older level's
// line in L1).
template <int W>
__device__ __forceinline__ void vload(const uint64_t* p, unsigned long long (&x)[W]) {
    if constexpr (W == 1) {
        x[0] = __ldcg(reinterpret_cast<const unsigned long long*>(p));
    } else {
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const ulonglong2 t = __ldcg(reinterpret_cast<const ulonglong2*>(p) + i);
            x[2 * i] = t.x;
            x[2 * i + 1] = t.y;
        }
    }
}

template <int W>
__device__ __forceinline__ void vor(const uint64_t* p, unsigned long long (&acc)[W]) {
    unsigned long long x[W];
    vload<W>(p, x);
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] |= x[w];
}

// OR of one in-neighbour's visited words into acc.  With DAWN_MS_GATHER_L1
// the loads may be served from L1: the grid barrier's acquire orders them
// after the previous level's stores (PTX memory model: a weak load that
// follows an acquire, here through the CTA barrier, observes what the
// release made visible), and a buffer is read only in the level after the
// one that wrote it.
#ifndef DAWN_MS_GATHER_L1
#define DAWN_MS_GATHER_L1 1
#endif
template <int W>
__device__ __forceinline__ void gor(const uint64_t* p, unsigned long long (&acc)[W]) {
#if DAWN_MS_GATHER_L1
    if constexpr (W == 1) {
        acc[0] |= *reinterpret_cast<const unsigned long long*>(p);
    } else {
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const ulonglong2 t = reinterpret_cast<const ulonglong2*>(p)[i];
            acc[2 * i] |= t.x;
            acc[2 * i + 1] |= t.y;
        }
    }
#else
    vor<W>(p, acc);
#endif
}

template <int W>
__device__ __forceinline__ void vstore(uint64_t* p, const unsigned long long (&x)[W]) {
    if constexpr (W == 1) {
        *reinterpret_cast<unsigned long long*>(p) = x[0];
    } else {
#pragma unroll
        for (int i = 0; i < W / 2; ++i) reinterpret_cast<ulonglong2*>(p)[i] = make_ulonglong2(x[2 * i], x[2 * i + 1]);
    }
}

template <int W>
__device__ __forceinline__ bool vcovered(const unsigned long long (&acc)[W], const unsigned long long (&vv)[W],
                                         const unsigned long long (&fin)[W]) {
    bool c = true;
#pragma unroll
    for (int w = 0; w < W; ++w) c &= (acc[w] | vv[w] | fin[w]) == ~0ull;
    return c;
}

// Zero `words` words from p on with the whole grid (16-byte stores; p is
// 8-byte aligned: a level array of W = 1 starts mid-line when n + 1 is odd).
__device__ __forceinline__ void grid_zero(uint64_t* p, long long words) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    if (words <= 0) return;
    if (reinterpret_cast<uintptr_t>(p) & 15u) {
        if (gtid == 0) p[0] = 0ull;
        ++p;
        --words;
    }
    ulonglong2* p2 = reinterpret_cast<ulonglong2*>(p);
    for (long long i = gtid; i < (words >> 1); i += nthreads) p2[i] = make_ulonglong2(0ull, 0ull);
    if ((words & 1) && gtid == 0) p[words - 1] = 0ull;
}

// A vertex's new bits at level t: next visited words, level record, growing lanes.
template <int W>
__device__ __forceinline__ void settle(const MsArgs& a, const MsSliced& p, uint64_t* vn, int t, int v,
                                       const unsigned long long (&vv)[W], const unsigned long long (&acc)[W],
                                       const unsigned long long (&fin)[W], unsigned long long (&grow)[W]) {
    unsigned long long nb[W], nx[W];
    bool any = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        nb[w] = acc[w] & ~vv[w] & ~fin[w];
        nx[w] = vv[w] | nb[w];
        grow[w] |= nb[w];
        any |= nb[w] != 0ull;
    }
    vstore<W>(vn + (long long)v * W, nx);
    if (!any) return;
    const long long stride = (long long)(a.n + 1) * W;
    if (t <= p.nb_levels) {
        vstore<W>(p.nbl + (t - 1) * stride + (long long)v * W, nb);
    } else {
        uint64_t* pv = p.planes + (long long)v * W;
        for (int b = 0; b < p.planes_cap; ++b) {
            if (!((t >> b) & 1)) continue;
#pragma unroll
            for (int w = 0; w < W; ++w)
                if (nb[w]) atomicOr(reinterpret_cast<unsigned long long*>(pv + b * stride + w), nb[w]);
        }
    }
}

// Level 1 as a push: bit s to every out-neighbour v != src of source s, in
// the next visited words and NB[1]; the grid splits the sources' out-arcs
// evenly (s_pre: prefix of their out-degrees).  Kept out of line: it runs
// once per pass and its registers would crowd the level loop.
template <int W>
__device__ __noinline__ void push_sources(const MsArgs& a, const MsSliced& p, int kb, const int* s_pre,
                                          const int* s_src, unsigned long long* s_newmask) {
    const long long total = s_pre[kb];
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += nthreads) {
        int lo = 0, hi = kb - 1;  // the last s with s_pre[s] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int src = s_src[lo];
        const int v = __ldg(p.out_idx + __ldg(p.out_ptr + src) + (e - s_pre[lo]));
        if (v == src) continue;
        const unsigned long long bit = 1ull << (lo & 63);
        atomicOr(reinterpret_cast<unsigned long long*>(&a.V1[(long long)v * W + (lo >> 6)]), bit);
        atomicOr(reinterpret_cast<unsigned long long*>(&p.nbl[(long long)v * W + (lo >> 6)]), bit);
        atomicOr(&s_newmask[lo >> 6], bit);
    }
}

// After a level's barrier (s_lanes = lanes that grew at level t): finished
// lanes, the last level with growth, the trace record.  True when every
// lane has finished.
template <int W>
__device__ __forceinline__ bool level_end(const MsArgs& a, int b, int t, const unsigned long long* s_lanes,
                                          unsigned long long* s_fin, int& tlast, int& tslot) {
    int growing = 0;
    bool done = true;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        growing += __popcll(s_lanes[w]);
        done &= (s_fin[w] | ~s_lanes[w]) == ~0ull;
    }
    __syncthreads();  // every thread has read s_fin
    if (threadIdx.x < W) s_fin[threadIdx.x] |= ~s_lanes[threadIdx.x];
    __syncthreads();
    if (growing) tlast = t;
    if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && tslot < a.trace_cap) {
        unsigned long long tnow;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tnow));
        long long* r = a.trace + 4 * (long long)tslot;
        r[0] = b;
        r[1] = t;
        r[2] = growing;
        r[3] = (long long)tnow;
    }
    ++tslot;
    return done;
}

template <int W>
__global__ void __launch_bounds__(kMsThreads, 1) msbfs_sliced_kernel(MsArgs a, MsSliced p) {
    __shared__ unsigned long long s_hacc[kHubMax][W];
    __shared__ unsigned long long s_newmask[W];
    __shared__ unsigned long long s_lanes[W];
    __shared__ unsigned long long s_fin[W];  // lanes that can no longer grow: unused, then finished
    __shared__ int s_reached[kMsMaxLanes];
    __shared__ int s_ecc[kMsMaxLanes];
    __shared__ long long s_dsum[kMsMaxLanes];
    __shared__ int4 s_tasks[kTaskSmem];
    __shared__ unsigned char s_cov[kTaskSmem];  // consecutive levels a task was fully covered
    __shared__ int s_hcnt[kHubMax];             // pieces of each split row done this level
    __shared__ int s_pre[kMsMaxLanes + 1];      // level 1: prefix of the sources' out-degrees
    __shared__ int s_src[kMsMaxLanes];
    __shared__ int s_next, s_status;
    extern __shared__ int s_hist[];  // with p.hist: [kNbLevelsMax + 1][64 * W] this CTA's level counts

    MsCtl* ctl = a.ctl;
    if (threadIdx.x == 0) s_status = ms_ld_relaxed_s32(&ctl->status);
    __syncthreads();
    if (s_status != DEV_OK) return;
    unsigned* bar = &ctl->bar[a.bar_parity].count;
    unsigned bar_target = 0;
    int tslot = 0;
    constexpr int L = 64 * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (p.hist)
        for (int i = threadIdx.x; i < (kNbLevelsMax + 1) * L; i += kMsThreads) s_hist[i] = 0;
    const long long gtid = (long long)blockIdx.x * kMsThreads + threadIdx.x;
    const int n = a.n;
    const long long stride = (long long)(n + 1) * W;
    const int nbatches = (a.k + L - 1) / L;
    const int tbeg = __ldg(p.cta_task + blockIdx.x), tend = __ldg(p.cta_task + blockIdx.x + 1);
    const int tsm = min(tend - tbeg, kTaskSmem);
    const int h0 = __ldg(p.cta_hub + blockIdx.x);
    const int ngroups = (n + 31) >> 5;
    const int gA = (int)((long long)ngroups * blockIdx.x / gridDim.x);
    const int gB = (int)((long long)ngroups * (blockIdx.x + 1) / gridDim.x);

    for (int i = threadIdx.x; i < kHubMax * W; i += kMsThreads) (&s_hacc[0][0])[i] = 0ull;
    for (int i = threadIdx.x; i < kHubMax; i += kMsThreads) s_hcnt[i] = 0;
    for (int i = threadIdx.x; i < tsm; i += kMsThreads) s_tasks[i] = __ldg(p.tasks + tbeg + i);
    for (int i = threadIdx.x; i < kMsMaxLanes; i += kMsThreads) {
        s_reached[i] = 0;
        s_ecc[i] = 0;
        s_dsum[i] = 0;
    }
    if (threadIdx.x < W) s_newmask[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) s_next = tbeg;

    for (int b = 0; b < nbatches; ++b) {
        const int s0 = b * L;
        const int kb = min(L, a.k - s0);
        // ---- seeds and level 1.  The visited buffers and NB[1] are zero here
        // (cleared by the previous pass's read-out, or since allocation).
        // Level 1's frontier is the sources alone, so it is a push over their
        // out-arcs: bit s goes to every out-neighbour of source s but itself.
        const unsigned long long (&fin)[W] = s_fin;
        for (int s = threadIdx.x; s < kb; s += kMsThreads) {
            const int src = __ldg(a.sources + s0 + s);
            s_src[s] = src;
            s_pre[s + 1] = __ldg(p.out_ptr + src + 1) - __ldg(p.out_ptr + src);
        }
        if (threadIdx.x == 0) s_pre[0] = 0;
        if (threadIdx.x < W) {
            const int lo = threadIdx.x * 64;
            s_fin[threadIdx.x] = kb >= lo + 64 ? 0ull : (kb <= lo ? ~0ull : ~0ull << (kb - lo));
        }
        for (int i = threadIdx.x; i < tsm; i += kMsThreads) s_cov[i] = 0;
        __syncthreads();
        if (warp == 0) {  // inclusive scan of s_pre[1..kb], 8 entries per lane
            int run = 0;
            for (int c = 0; c < kMsMaxLanes / 32; ++c) {
                const int i = 1 + lane * (kMsMaxLanes / 32) + c;
                if (i <= kb) run += s_pre[i];
            }
            int incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            int acc = incl - run;
            for (int c = 0; c < kMsMaxLanes / 32; ++c) {
                const int i = 1 + lane * (kMsMaxLanes / 32) + c;
                if (i <= kb) {
                    acc += s_pre[i];
                    s_pre[i] = acc;
                }
            }
        }
        __syncthreads();
        if (gtid < kb) {
            const int s = (int)gtid;
            const int src = s_src[s];
            const unsigned long long bit = 1ull << (s & 63);
            atomicOr(reinterpret_cast<unsigned long long*>(&a.V0[(long long)src * W + (s >> 6)]), bit);
            atomicOr(reinterpret_cast<unsigned long long*>(&a.V1[(long long)src * W + (s >> 6)]), bit);
            a.reached[s0 + s] = 0;  // the read-out adds every CTA's sums
            a.dsum[s0 + s] = 0;
            a.ecc[s0 + s] = 0;
        }
        push_sources<W>(a, p, kb, s_pre, s_src, s_newmask);
        if (p.nb_levels >= 2) grid_zero(p.nbl + stride, stride);  // NB[2]
        __syncthreads();
        if (threadIdx.x < W && s_newmask[threadIdx.x]) {
            atomicOr(&ctl->lanes_new[1][threadIdx.x], s_newmask[threadIdx.x]);
            s_newmask[threadIdx.x] = 0ull;
        }
        if (blockIdx.x == 0 && threadIdx.x >= 32 && threadIdx.x < 32 + W) ctl->lanes_new[2][threadIdx.x - 32] = 0ull;
        if (!ms_barrier(ctl, bar, bar_target, a.spin_limit, ctl->lanes_new[1], W, s_lanes)) return;

        int tlast = 0;
        bool finished = level_end<W>(a, b, 1, s_lanes, s_fin, tlast, tslot);
        const uint64_t* vp = a.V1;
        uint64_t* vn = a.V0;
        for (int t = 2; !finished; ++t) {
            if (a.dist_bytes == 2 && t > 32767) {
                if (gtid == 0) atomicCAS(&ctl->status, DEV_OK, DEV_OVERFLOW);
                return;
            }
            // (harmonic centrality counts levels in the level arrays only)
            if (t > p.nb_levels && (t >= (1 << p.planes_cap) || p.hist)) {
                if (gtid == 0) atomicCAS(&ctl->status, DEV_OK, DEV_PLANES);
                return;
            }
            // the next level's record starts zero
            if (t + 1 <= p.nb_levels) grid_zero(p.nbl + t * stride, stride);
            else if (t == p.nb_levels) grid_zero(p.planes, (long long)p.planes_cap * stride);
            unsigned long long grow[W];
#pragma unroll
            for (int w = 0; w < W; ++w) grow[w] = 0ull;
            // ---- this CTA's tasks, one warp at a time
            while (true) {
                int i = 0;
                if (lane == 0) i = atomicAdd(&s_next, 1);
                i = __shfl_sync(kFull, i, 0);
                if (i >= tend) break;
                const int li = i - tbeg;
                if (li < kTaskSmem && s_cov[li] >= 2) continue;  // never a split row's piece
                const int4 tk = li < kTaskSmem ? s_tasks[li] : __ldg(p.tasks + i);
                unsigned long long vv[W], acc[W];
#pragma unroll
                for (int w = 0; w < W; ++w) acc[w] = 0ull;
                bool covered;
                bool settle_it;  // this lane settles vertex sv below
                int sv;
                if (tk.x >= 0) {
                    // row piece: arcs [tk.y, tk.z) of vertex tk.x, 128 per round;
                    // each round's indices load with the previous round's words
                    const int v = tk.x;
                    sv = v;
                    const int j1 = tk.z;
                    int j = tk.y + lane;
                    int u0 = j < j1 ? __ldg(a.in_idx + j) : -1;
                    int u1 = j + 32 < j1 ? __ldg(a.in_idx + j + 32) : -1;
                    int u2 = j + 64 < j1 ? __ldg(a.in_idx + j + 64) : -1;
                    int u3 = j + 96 < j1 ? __ldg(a.in_idx + j + 96) : -1;
                    vload<W>(vp + (long long)v * W, vv);
                    bool need = false;
#pragma unroll
                    for (int w = 0; w < W; ++w) need |= (vv[w] | fin[w]) != ~0ull;
                    covered = !need;
                    if (need) {
                        for (int base = tk.y; base < j1; base += 128) {
                            j += 128;
                            int n0 = -1, n1 = -1, n2 = -1, n3 = -1;
                            if (base + 128 < j1) {
                                n0 = j < j1 ? __ldg(a.in_idx + j) : -1;
                                n1 = j + 32 < j1 ? __ldg(a.in_idx + j + 32) : -1;
                                n2 = j + 64 < j1 ? __ldg(a.in_idx + j + 64) : -1;
                                n3 = j + 96 < j1 ? __ldg(a.in_idx + j + 96) : -1;
                            }
                            if (u0 >= 0) gor<W>(vp + (long long)u0 * W, acc);
                            if (u1 >= 0) gor<W>(vp + (long long)u1 * W, acc);
                            if (u2 >= 0) gor<W>(vp + (long long)u2 * W, acc);
                            if (u3 >= 0) gor<W>(vp + (long long)u3 * W, acc);
                            u0 = n0;
                            u1 = n1;
                            u2 = n2;
                            u3 = n3;
                        }
#pragma unroll
                        for (int w = 0; w < W; ++w) acc[w] = warp_or_redux(acc[w]);
                    }
                    settle_it = lane == 0;
                    if (tk.w >= 0) {
                        // a split row: the CTA's last piece to finish settles it
                        settle_it = false;
                        if (lane == 0) {
                            const int slot = tk.w & 255, npieces = tk.w >> 8;
                            if (need) {
#pragma unroll
                                for (int w = 0; w < W; ++w)
                                    if (acc[w]) atomicOr(&s_hacc[slot][w], acc[w]);
                            }
                            __threadfence_block();
                            if (atomicAdd(&s_hcnt[slot], 1) == npieces - 1) {
                                __threadfence_block();
#pragma unroll
                                for (int w = 0; w < W; ++w) acc[w] = atomicExch(&s_hacc[slot][w], 0ull);
                                s_hcnt[slot] = 0;
                                settle_it = true;
                            }
                        }
                        covered = false;  // split rows are never skipped
                    }
                } else {
                    // slice: lane = vertex, its in-arcs four columns per round.  The
                    // first two rounds' indices load with the vertex, the first
                    // round's words with its own words (before it is known whether
                    // the vertex still needs them), later indices a round ahead.
                    const int sid = -1 - tk.x;
                    const int D = tk.z;
                    const int32_t* col = p.sell_idx + tk.y + lane;
                    const int2 vd = __ldg(p.sell_vd + (long long)sid * 32 + lane);
                    sv = vd.x;
                    int u0 = D > 0 ? __ldg(col) : -1;
                    int u1 = D > 1 ? __ldg(col + 32) : -1;
                    int u2 = D > 2 ? __ldg(col + 64) : -1;
                    int u3 = D > 3 ? __ldg(col + 96) : -1;
                    int n0 = D > 4 ? __ldg(col + 128) : -1;
                    int n1 = D > 5 ? __ldg(col + 160) : -1;
                    int n2 = D > 6 ? __ldg(col + 192) : -1;
                    int n3 = D > 7 ? __ldg(col + 224) : -1;
                    const int v = vd.x;
                    bool need = false;
                    if (v >= 0) vload<W>(vp + (long long)v * W, vv);
                    if (u0 >= 0) gor<W>(vp + (long long)u0 * W, acc);
                    if (u1 >= 0) gor<W>(vp + (long long)u1 * W, acc);
                    if (u2 >= 0) gor<W>(vp + (long long)u2 * W, acc);
                    if (u3 >= 0) gor<W>(vp + (long long)u3 * W, acc);
                    if (v >= 0) {
#pragma unroll
                        for (int w = 0; w < W; ++w) need |= (vv[w] | fin[w]) != ~0ull;
                    }
                    covered = __all_sync(kFull, !need);
                    for (int j = 4; !covered && j < D; j += 4) {
                        if (__all_sync(kFull, !need || vcovered<W>(acc, vv, fin))) break;
                        u0 = n0;
                        u1 = n1;
                        u2 = n2;
                        u3 = n3;
                        n0 = n1 = n2 = n3 = -1;
                        if (j + 4 < D) {
                            n0 = __ldg(col + 32 * (j + 4));
                            n1 = j + 5 < D ? __ldg(col + 32 * (j + 5)) : -1;
                            n2 = j + 6 < D ? __ldg(col + 32 * (j + 6)) : -1;
                            n3 = j + 7 < D ? __ldg(col + 32 * (j + 7)) : -1;
                        }
                        if (need) {
                            if (u0 >= 0) gor<W>(vp + (long long)u0 * W, acc);
                            if (u1 >= 0) gor<W>(vp + (long long)u1 * W, acc);
                            if (u2 >= 0) gor<W>(vp + (long long)u2 * W, acc);
                            if (u3 >= 0) gor<W>(vp + (long long)u3 * W, acc);
                        }
                    }
                    if (!need) {
#pragma unroll
                        for (int w = 0; w < W; ++w) acc[w] = 0ull;
                    }
                    settle_it = v >= 0;
                }
                if (settle_it) settle<W>(a, p, vn, t, sv, vv, acc, fin, grow);
                if (lane == 0 && li < kTaskSmem) s_cov[li] = covered ? s_cov[li] + 1 : 0;
            }
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const unsigned long long x = warp_or_redux(grow[w]);
                if (lane == 0 && x) atomicOr(&s_newmask[w], x);
            }
            __syncthreads();  // every warp has left the task loop
            if (threadIdx.x == 0) s_next = tbeg;
            if (threadIdx.x < W && s_newmask[threadIdx.x]) {
                atomicOr(&ctl->lanes_new[t % 3][threadIdx.x], s_newmask[threadIdx.x]);
                s_newmask[threadIdx.x] = 0ull;
            }
            if (blockIdx.x == 0 && threadIdx.x >= 32 && threadIdx.x < 32 + W)
                ctl->lanes_new[(t + 1) % 3][threadIdx.x - 32] = 0ull;
            if (!ms_barrier(ctl, bar, bar_target, a.spin_limit, ctl->lanes_new[t % 3], W, s_lanes)) return;
            finished = level_end<W>(a, b, t, s_lanes, s_fin, tlast, tslot);
            const uint64_t* tmp = vn;
            vn = const_cast<uint64_t*>(vp);
            vp = tmp;
        }
        // ---- read-out.  One item = 32 consecutive vertices (lane = vertex) x
        // 32 lanes of sources; a CTA's items cover its vertex range.  vp holds
        // the final visited words; bit p of the level at which source s
        // reached v is bit s of level plane p, OR-ed from the level arrays
        // (and from the stored planes of deeper levels).
        const int np = tlast ? 32 - __clz(tlast) : 0;
        const int tnb = min(tlast, p.nb_levels);
        const bool deep = tlast > p.nb_levels;
        constexpr int H = 2 * W;  // 32-lane halves of a vertex's words
        for (int it = gA * H + warp; it < gB * H; it += kMsWarps) {
            const int gi = it / H, hw = it - gi * H;
            const int sb = hw * 32;
            if (sb >= kb) continue;
            const int v = gi * 32 + lane;
            const bool valid = v < n;
            const int vr = valid ? v : n;  // the zero row stands in for lanes past n
            const unsigned* r32p = reinterpret_cast<const unsigned*>(vp + (long long)vr * W) + hw;
            const unsigned* nb32 = reinterpret_cast<const unsigned*>(p.nbl + (long long)vr * W) + hw;
            const unsigned r32 = __ldcg(r32p);
            // levels below 16 (bits 0..3) from the level arrays, all loads at once
            unsigned x[kNbLevelsMax];
#pragma unroll
            for (int t = 1; t <= kNbLevelsMax; ++t) x[t - 1] = t <= tnb ? __ldcg(nb32 + 2 * (t - 1) * stride) : 0u;
            unsigned pl0 = 0u, pl1 = 0u, pl2 = 0u, pl3 = 0u;
#pragma unroll
            for (int t = 1; t <= kNbLevelsMax; ++t) {
                if (t & 1) pl0 |= x[t - 1];
                if (t & 2) pl1 |= x[t - 1];
                if (t & 4) pl2 |= x[t - 1];
                if (t & 8) pl3 |= x[t - 1];
            }
            const unsigned* pp = reinterpret_cast<const unsigned*>(p.planes + (long long)vr * W) + hw;
            unsigned vals[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) vals[i] = 0u;
            const unsigned rt = bit_transpose32(r32);  // lane = source sb + lane: reached vertices
            unsigned cand = rt;
            int ecc = 0;
            long long dsum = 0;
            unsigned dt0 = 0u, dt1 = 0u, dt2 = 0u, dt3 = 0u;  // the low planes, transposed (for p.hist)
            for (int q = np - 1; q >= 0; --q) {
                unsigned d = q == 0 ? pl0 : q == 1 ? pl1 : q == 2 ? pl2 : q == 3 ? pl3 : 0u;
                if (deep) d |= __ldcg(pp + 2 * q * stride);
                if (!a.nostore) {
                    // bit 2i of d to bit q of vals[i], bit 2i + 1 to bit 16 + q: (ehi:elo)
                    // is d << q in 64 bits, and a funnel shift picks any 32 of them
                    const unsigned elo = d << q, ehi = q ? d >> (32 - q) : 0u;
                    const unsigned m0 = 1u << q, m1 = 0x10000u << q;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        vals[i] |= __funnelshift_r(elo, ehi, 2 * i) & m0;
                        vals[i] |= (2 * i + 1 <= 16 ? elo << (15 - 2 * i) : __funnelshift_r(elo, ehi, 2 * i - 15)) & m1;
                    }
                }
                const unsigned dt = bit_transpose32(d);
                if (q == 0) dt0 = dt;
                else if (q == 1) dt1 = dt;
                else if (q == 2) dt2 = dt;
                else if (q == 3) dt3 = dt;
                dsum += (long long)__popc(dt) << q;
                const unsigned c = cand & dt;
                if (c) {
                    cand = c;
                    ecc |= 1 << q;
                }
            }
            if (sb + lane < kb) {
                atomicAdd(&s_reached[sb + lane], __popc(rt));
                atomicAdd(reinterpret_cast<unsigned long long*>(&s_dsum[sb + lane]), (unsigned long long)dsum);
                atomicMax(&s_ecc[sb + lane], ecc);
                if (p.hist) {
                    // vertices of this item at each level t >= 1: the reached ones
                    // whose level bits spell t (tlast <= nb_levels <= 15 here)
                    for (int t = 1; t <= tlast; ++t) {
                        const unsigned m = rt & ((t & 1) ? dt0 : ~dt0) & ((t & 2) ? dt1 : ~dt1) &
                                           ((t & 4) ? dt2 : ~dt2) & ((t & 8) ? dt3 : ~dt3);
                        if (m) atomicAdd(&s_hist[t * L + sb + lane], __popc(m));
                    }
                }
            }
            if (valid && !a.nostore) {
                // unreached cells read -1
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const unsigned rm = (((r32 >> (2 * i)) & 1u) ? 0x0000FFFFu : 0u) | (((r32 >> (2 * i + 1)) & 1u) ? 0xFFFF0000u : 0u);
                    vals[i] = (vals[i] & rm) | ~rm;
                }
                const int nsrc = min(32, kb - sb);
                char* cell;
                long long step;
                if (a.layout == DAWN_SOURCE_MAJOR) {
                    const long long row0 = a.per_pass ? sb : s0 + sb;
                    cell = static_cast<char*>(a.out) + (row0 * a.out_row_stride + v) * a.dist_bytes;
                    step = a.out_row_stride * a.dist_bytes;
                } else {
                    cell = static_cast<char*>(a.out) + ((long long)v * a.out_row_stride + s0 + sb) * a.dist_bytes;
                    step = a.dist_bytes;
                }
                if (a.dist_bytes == 2) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i >= nsrc) break;
                        *reinterpret_cast<unsigned short*>(cell) = (unsigned short)(vals[i >> 1] >> (16 * (i & 1)));
                        cell += step;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (i >= nsrc) break;
                        *reinterpret_cast<int32_t*>(cell) = (int32_t)(short)(vals[i >> 1] >> (16 * (i & 1)));
                        cell += step;
                    }
                }
            }
        }
        __syncthreads();  // every item of this CTA has read its visited words and summed
        // both visited buffers back to zero over this CTA's vertices
        {
            const long long w0 = (long long)gA * 32 * W, w1 = (long long)min(gB * 32, n) * W;
            for (long long i = w0 + threadIdx.x; i < w1; i += kMsThreads) {
                a.V0[i] = 0ull;
                a.V1[i] = 0ull;
                p.nbl[i] = 0ull;  // NB[1]: the next pass's level-1 push ORs into it
            }
        }
        // the level slots start the next pass at zero (every CTA has read them)
        if (blockIdx.x == 0 && threadIdx.x < 3 * W) ctl->lanes_new[threadIdx.x / W][threadIdx.x % W] = 0ull;
        // per-source sums into the outputs (zeroed at the pass's start)
        for (int s = threadIdx.x; s < kb; s += kMsThreads) {
            if (s_reached[s]) atomicAdd(&a.reached[s0 + s], s_reached[s]);
            if (s_dsum[s]) atomicAdd(reinterpret_cast<unsigned long long*>(&a.dsum[s0 + s]), (unsigned long long)s_dsum[s]);
            if (s_ecc[s]) atomicMax(&a.ecc[s0 + s], s_ecc[s]);
            s_reached[s] = 0;
            s_ecc[s] = 0;
            s_dsum[s] = 0;
        }
        if (p.hist) {
            for (int i = threadIdx.x; i < (tlast + 1) * L; i += kMsThreads) {
                if (s_hist[i]) atomicAdd(&p.hist[(i / L) * kMsMaxLanes + (i % L)], s_hist[i]);
                s_hist[i] = 0;
            }
        }
        // the next pass seeds the visited buffers this pass has just cleared;
        // centrality products read every CTA's sums
        const bool products = p.hist || a.clos;
        if ((b + 1 < nbatches || products) && !ms_barrier(ctl, bar, bar_target, a.spin_limit)) return;
        if (products && blockIdx.x == 0) {
            for (int s = threadIdx.x; s < kb; s += kMsThreads) {
                if (p.hist) {
                    // sum over distances t = 1, 2, ... of (vertices at distance t) / t, ascending
                    double h = 0.0;
                    for (int t = 1; t <= tlast; ++t) {
                        int32_t* c = p.hist + t * kMsMaxLanes + s;
                        const int cnt = __ldcg(c);
                        if (cnt) {
                            h += (double)cnt / (double)t;
                            *c = 0;
                        }
                    }
                    a.harm[s0 + s] = h;
                }
                if (a.clos) {
                    const int r = __ldcg(a.reached + s0 + s);
                    const long long sum = __ldcg(a.dsum + s0 + s);
                    a.clos[s0 + s] = r > 1 ? (double)(r - 1) / (double)sum : 0.0;
                }
            }
        }
    }
    if (gtid == 0) ctl->bar[a.bar_parity ^ 1].count = 0;
}

__global__ void ms_sell_fill_kernel(const int4* __restrict__ slices, int32_t ns, const int2* __restrict__ vd,
                                    const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ in_idx,
                                    int32_t* __restrict__ sell) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < ns; s += nw) {
        const int4 tk = slices[s];
        const int2 x = vd[s * 32 + lane];
        const int b = x.x >= 0 ? in_ptr[x.x] : 0;
        for (int j = 0; j < tk.z; ++j) sell[(long long)tk.y + 32LL * j + lane] = j < x.y ? in_idx[b + j] : -1;
    }
}

// Cut the in-arc rows into the sliced kernel's tasks (once per graph).
int ms_plan_build(dawn_graph* g, cudaStream_t st) {
    if (g->ms_plan && static_cast<MsPlan*>(g->ms_plan)->sms == g->sms) return DAWN_OK;
    ms_release(g);
    const int n = g->n, sms = g->sms;
    std::vector<int32_t> ip((size_t)n + 1);
    DAWN_CUDA_TRY(cudaMemcpyAsync(ip.data(), g->in_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost, st));
    DAWN_CUDA_TRY(cudaStreamSynchronize(st));
    auto deg = [&](int v) { return ip[(size_t)v + 1] - ip[v]; };
    // Short rows of vertices outside the largest component go last: lanes of
    // the large component never reach them, so their slices stay uncovered
    // all pass, and grouped they keep few slices busy.
    int32_t big = 0;
    for (int32_t c : g->csize_host) big = std::max(big, c);
    auto minor = [&](int v) { return !g->csize_host.empty() && g->csize_host[(size_t)v] < big ? 1 : 0; };
    std::vector<int32_t> order;
    order.reserve((size_t)n);
    for (int v = 0; v < n; ++v)
        if (deg(v) > 0) order.push_back(v);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int dx = deg(x), dy = deg(y);
        if ((dx > kSellDeg) != (dy > kSellDeg)) return dx > kSellDeg;
        if (dx <= kSellDeg && minor(x) != minor(y)) return minor(x) < minor(y);
        return dx > dy;
    });
    const long long M = ip[(size_t)n];
    const long long nwarps = (long long)sms * kMsWarps;

    // Estimated warp time: the dependent memory round trips (kTrip each;
    // levels are latency bound) plus one per warp step of 32 arcs.
    auto piece_cost = [](int len) -> long long {
        const int rounds = (len + 127) / 128, steps = (len + 31) / 32;
        return (long long)kTrip * (2 + rounds) + steps;
    };
    auto slice_cost = [](int D) -> long long {
        const int rounds = (D + 3) / 4;
        return (long long)kTrip * (2 + std::max(0, rounds - 1) + (rounds > 2 ? rounds - 2 : 0)) + D;
    };
    struct Unit {
        int first, count;  // tasks
        long long cost;    // piece_cost / slice_cost of its tasks
        int split;         // a row cut into several pieces
    };
    std::vector<int4> tasks;
    std::vector<Unit> units;
    std::vector<int2> vd;
    std::vector<int32_t> cta_task((size_t)sms + 1), cta_hub((size_t)sms + 1), hub_v;
    long long piece = std::max<long long>(kPieceMin, ((M / (2 * nwarps)) + 31) / 32 * 32);
    long long sell_len = 0;
    int nslices = 0, max_hubs = 0, max_tasks = 0, first_slice = 0;
    std::vector<int4> slice_tasks;  // the slice tasks in slice-id order (for filling sell_idx)
    for (;; piece *= 2) {
        tasks.clear();
        units.clear();
        vd.clear();
        hub_v.clear();
        size_t i = 0;
        for (; i < order.size() && deg(order[i]) > kSellDeg; ++i) {
            const int v = order[i], d = deg(v), b = ip[v];
            if (d <= piece) {
                units.push_back({(int)tasks.size(), 1, piece_cost(d), 0});
                tasks.push_back(make_int4(v, b, b + d, -1));
            } else {
                const long long np0 = (d + piece - 1) / piece;
                const int ps = (int)(((d + np0 - 1) / np0 + 31) / 32 * 32);
                Unit u{(int)tasks.size(), 0, kTrip, 1};
                for (int j0 = b; j0 < b + d; j0 += ps) {
                    const int j1 = std::min(b + d, j0 + ps);
                    tasks.push_back(make_int4(v, j0, j1, 0));
                    u.count += 1;
                    u.cost += piece_cost(j1 - j0);
                }
                units.push_back(u);
            }
        }
        first_slice = (int)tasks.size();
        sell_len = 0;
        nslices = 0;
        for (; i < order.size(); i += 32) {
            int D = 0;
            for (size_t l = 0; l < 32; ++l) {
                const size_t idx = i + l;
                vd.push_back(idx < order.size() ? make_int2(order[idx], deg(order[idx])) : make_int2(-1, 0));
                if (idx < order.size()) D = std::max(D, deg(order[idx]));
            }
            units.push_back({(int)tasks.size(), 1, slice_cost(D), 0});
            tasks.push_back(make_int4(-1 - nslices, (int)sell_len, D, 0));
            sell_len += 32LL * D;
            ++nslices;
            if (sell_len >= (1LL << 31)) return fail(DAWN_E_INVALID, "graph too large for the sliced batched kernel");
        }
        // Units to CTAs, largest first, each to the least loaded CTA so far:
        // every CTA gets a mix of row lengths, and the rows that stay
        // uncovered longest (the short ones) are spread over the grid.
        std::vector<std::vector<int>> mine((size_t)sms);
        {
            using Load = std::pair<long long, int>;
            std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
            for (int c = 0; c < sms; ++c) heap.push({0, c});
            for (size_t x = 0; x < units.size(); ++x) {
                Load l = heap.top();
                heap.pop();
                mine[(size_t)l.second].push_back((int)x);
                l.first += units[x].cost;
                heap.push(l);
            }
        }
        std::vector<int4> by_cta;
        by_cta.reserve(tasks.size());
        max_hubs = 0;
        max_tasks = 0;
        for (int c = 0; c < sms; ++c) {
            cta_task[(size_t)c] = (int)by_cta.size();
            cta_hub[(size_t)c] = (int)hub_v.size();
            int local = 0;
            for (int x : mine[(size_t)c]) {
                const Unit& u = units[(size_t)x];
                for (int t = u.first; t < u.first + u.count; ++t) {
                    int4 tk = tasks[(size_t)t];
                    if (u.split) tk.w = local | (u.count << 8);  // CTA slot, pieces of the row
                    by_cta.push_back(tk);
                }
                if (u.split) {
                    hub_v.push_back(tasks[(size_t)u.first].x);
                    ++local;
                }
            }
            max_hubs = std::max(max_hubs, local);
            max_tasks = std::max(max_tasks, (int)by_cta.size() - cta_task[(size_t)c]);
        }
        cta_task[(size_t)sms] = (int)by_cta.size();
        cta_hub[(size_t)sms] = (int)hub_v.size();
        slice_tasks.assign(tasks.begin() + first_slice, tasks.end());
        tasks.swap(by_cta);
        if (max_hubs <= kHubMax) break;
    }

    auto* pl = new MsPlan();
    pl->sms = sms;
    pl->ntasks = (int)tasks.size();
    pl->nhubs = (int)hub_v.size();
    pl->nslices = nslices;
    pl->piece = (int)piece;
    pl->max_hubs = max_hubs;
    pl->max_tasks = max_tasks;
    pl->sell_len = sell_len;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t o_tasks = 0, o_ct = o_tasks + al(sizeof(int4) * tasks.size() + 16);
    const size_t o_ch = o_ct + al(sizeof(int32_t) * ((size_t)sms + 1));
    const size_t o_hv = o_ch + al(sizeof(int32_t) * ((size_t)sms + 1));
    const size_t o_vd = o_hv + al(sizeof(int32_t) * hub_v.size() + 4);
    const size_t o_si = o_vd + al(sizeof(int2) * vd.size() + 8);
    const size_t bytes = o_si + al(sizeof(int32_t) * (size_t)sell_len + 4);
    cudaError_t e = cudaMalloc(&pl->blob, bytes);
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "cudaMalloc (batched plan)", __FILE__, __LINE__);
    }
    g->ms_plan = pl;
    char* base = static_cast<char*>(pl->blob);
    pl->tasks = reinterpret_cast<int4*>(base + o_tasks);
    pl->cta_task = reinterpret_cast<int32_t*>(base + o_ct);
    pl->cta_hub = reinterpret_cast<int32_t*>(base + o_ch);
    pl->hub_v = reinterpret_cast<int32_t*>(base + o_hv);
    pl->sell_vd = reinterpret_cast<int2*>(base + o_vd);
    pl->sell_idx = reinterpret_cast<int32_t*>(base + o_si);
    if (!tasks.empty())
        DAWN_CUDA_TRY(cudaMemcpyAsync(pl->tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice, st));
    DAWN_CUDA_TRY(cudaMemcpyAsync(pl->cta_task, cta_task.data(), sizeof(int32_t) * cta_task.size(), cudaMemcpyHostToDevice, st));
    DAWN_CUDA_TRY(cudaMemcpyAsync(pl->cta_hub, cta_hub.data(), sizeof(int32_t) * cta_hub.size(), cudaMemcpyHostToDevice, st));
    if (!hub_v.empty())
        DAWN_CUDA_TRY(cudaMemcpyAsync(pl->hub_v, hub_v.data(), sizeof(int32_t) * hub_v.size(), cudaMemcpyHostToDevice, st));
    if (nslices > 0) {
        int4* sl = nullptr;  // slice descriptors in slice-id order
        DAWN_CUDA_TRY(cudaMallocAsync((void**)&sl, sizeof(int4) * slice_tasks.size(), st));
        DAWN_CUDA_TRY(cudaMemcpyAsync(sl, slice_tasks.data(), sizeof(int4) * slice_tasks.size(), cudaMemcpyHostToDevice, st));
        DAWN_CUDA_TRY(cudaMemcpyAsync(pl->sell_vd, vd.data(), sizeof(int2) * vd.size(), cudaMemcpyHostToDevice, st));
        ms_sell_fill_kernel<<<sms * 4, 256, 0, st>>>(sl, nslices, pl->sell_vd, g->in_ptr, g->in_idx, pl->sell_idx);
        DAWN_CUDA_TRY(cudaGetLastError());
        DAWN_CUDA_TRY(cudaFreeAsync(sl, st));
    }
    DAWN_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors go out of scope
    return DAWN_OK;
}

// The per-level new-bit arrays (levels 1 .. ms_nb_levels, sized for W = 4):
// as many as kNbBudget holds, at least 4, at most kNbLevelsMax.
int ms_nb_alloc(dawn_graph* g) {
    if (g->ms_nb) return DAWN_OK;
    const size_t per = sizeof(uint64_t) * 4 * ((size_t)g->n + 1);
    const int levels = (int)std::max<size_t>(4, std::min<size_t>(kNbLevelsMax, kNbBudget / per));
    DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_nb, per * (size_t)levels));
    DAWN_CUDA_TRY(cudaMemset(g->ms_nb, 0, per));  // NB[1] starts zero; later levels are zeroed ahead
    g->ms_nb_levels = levels;
    return DAWN_OK;
}

// Level planes for levels past the new-bit arrays (sized for W = 4).
int ms_planes_alloc(dawn_graph* g, int planes) {
    if (g->ms_planes && g->ms_planes_cap >= planes) return DAWN_OK;
    if (g->ms_planes) cudaFree(g->ms_planes);
    g->ms_planes = nullptr;
    g->ms_planes_cap = 0;
    DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_planes, sizeof(uint64_t) * 4 * ((size_t)g->n + 1) * (size_t)planes));
    g->ms_planes_cap = planes;
    return DAWN_OK;
}

template <int W>
int ms_launch_sliced_w(dawn_graph* g, MsArgs& a, MsSliced& p, cudaStream_t st) {
    dim3 grid(g->sms), block(kMsThreads);
    void* args[] = {&a, &p};
    const int hist_bytes = (int)sizeof(int) * (kNbLevelsMax + 1) * 64 * W;
    DAWN_CUDA_TRY(cudaFuncSetAttribute((const void*)msbfs_sliced_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       hist_bytes));
    DAWN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)msbfs_sliced_kernel<W>, grid, block, args,
                                              p.hist ? hist_bytes : 0, st));
    return DAWN_OK;
}

// Whole-run figures over the listed sources: {largest ecc, smallest ecc among
// sources that reach another vertex (-1 if none), pairs, distance total}.
__global__ void apsp_summary_kernel(const int32_t* __restrict__ ecc, const long long* __restrict__ dsum,
                                    const int32_t* __restrict__ reached, int32_t k, long long* out) {
    __shared__ int s_max, s_min;
    __shared__ unsigned long long s_pairs, s_total;
    if (threadIdx.x == 0) {
        s_max = 0;
        s_min = INT_MAX;
        s_pairs = 0ull;
        s_total = 0ull;
    }
    __syncthreads();
    int mx = 0, mn = INT_MAX;
    unsigned long long pairs = 0ull, total = 0ull;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        mx = max(mx, ecc[i]);
        if (reached[i] > 1) mn = min(mn, ecc[i]);
        pairs += (unsigned long long)(reached[i] - 1);
        total += (unsigned long long)dsum[i];
    }
    atomicMax(&s_max, mx);
    atomicMin(&s_min, mn);
    atomicAdd(&s_pairs, pairs);
    atomicAdd(&s_total, total);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = s_max;
        out[1] = s_min == INT_MAX ? -1 : s_min;
        out[2] = (long long)s_pairs;
        out[3] = (long long)s_total;
    }
}

int msbfs_run(dawn_graph* g, const int32_t* sources, int32_t k, void* dist_block, int dist_bytes, int layout,
              int32_t* ecc, int64_t* dsum, int32_t* reached, const dawn_msbfs_opts* opts, cudaStream_t st,
              double* closeness = nullptr, double* harmonic = nullptr, dawn_apsp_summary* summary = nullptr,
              bool nostore = false) {
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!sources || k < 1) return fail(DAWN_E_INVALID, "need k >= 1 sources (k = %d)", k);
    if (dist_bytes != 2 && dist_bytes != 4) return fail(DAWN_E_INVALID, "dist_bytes = %d: need 2 or 4", dist_bytes);
    if (layout != DAWN_SOURCE_MAJOR && layout != DAWN_VERTEX_MAJOR)
        return fail(DAWN_E_INVALID, "unknown layout %d", layout);
    int lanes = opts && opts->lanes ? opts->lanes : 0;
    if (lanes != 0 && lanes != 64 && lanes != 128 && lanes != 256)
        return fail(DAWN_E_INVALID, "lanes = %d: need 64, 128 or 256", lanes);
    if (lanes == 0 && g->tuning.lanes > 0) lanes = g->tuning.lanes;
    if (lanes == 0) lanes = k <= 64 ? 64 : (k <= 128 ? 128 : 256);
    const int W = lanes / 64;
    const long long spin = (opts && opts->spin_limit > 0) ? opts->spin_limit : kDefaultSpin;
    const int want = opts ? opts->kernel : 0;
    if (want != 0 && want != DAWN_MSBFS_SLICED && want != DAWN_MSBFS_PER_LEVEL)
        return fail(DAWN_E_INVALID, "kernel = %d: need 0, DAWN_MSBFS_SLICED or DAWN_MSBFS_PER_LEVEL", want);
    const size_t plane_bytes = sizeof(uint64_t) * 4 * ((size_t)g->n + 1);  // one level array or plane
    // harmonic centrality on the sliced kernel counts levels in its level arrays
    // only; a graph on which a pass went deeper keeps the per-level kernel for it
    const bool sliced = want == DAWN_MSBFS_SLICED ||
                        (want == 0 && !g->ms_sliced_off && !(harmonic && g->ms_harm_deep));

    // sources: checked on the host whatever memory they live in
    std::vector<int32_t> hsrc((size_t)k);
    DAWN_CUDA_TRY(cudaMemcpy(hsrc.data(), sources, sizeof(int32_t) * (size_t)k, cudaMemcpyDefault));
    for (int32_t i = 0; i < k; ++i)
        if (hsrc[i] < 0 || hsrc[i] >= g->n) return fail(DAWN_E_INVALID, "sources[%d] = %d outside [0, %d)", i, hsrc[i], g->n);

    int rc = ms_workspace(g, W);
    if (rc != DAWN_OK) return rc;
    if (sliced) {
        if ((rc = ms_plan_build(g, st)) != DAWN_OK) return rc;
        if ((rc = ms_nb_alloc(g)) != DAWN_OK) return rc;
    }

    const size_t cell = (size_t)dist_bytes;
    const bool out_dev = dist_block && is_device_ptr(dist_block);
    const bool ecc_dev = ecc && is_device_ptr(ecc), dsum_dev = dsum && is_device_ptr(dsum),
               reached_dev = reached && is_device_ptr(reached);
    const bool clos_dev = closeness && is_device_ptr(closeness), harm_dev = harmonic && is_device_ptr(harmonic);
    // temporaries: device sources, reductions, distance staging
    void* tmp = nullptr;
    size_t off_src = 0, off_ecc = 256 * (((size_t)k * 4 + 255) / 256);
    size_t off_dsum = off_ecc + 256 * (((size_t)k * 4 + 255) / 256);
    size_t off_reached = off_dsum + 256 * (((size_t)k * 8 + 255) / 256);
    size_t off_clos = off_reached + 256 * (((size_t)k * 4 + 255) / 256);
    size_t off_harm = off_clos + 256 * (((size_t)k * 8 + 255) / 256);
    size_t off_ring = off_harm + 256 * (((size_t)k * 8 + 255) / 256);
    size_t off_sum = off_ring + 256 * ((3 * kMsMaxLanes * sizeof(int32_t) + 255) / 256);
    size_t off_hist = off_sum + 256;
    size_t off_dist = off_hist + 256 * (((size_t)(kNbLevelsMax + 1) * kMsMaxLanes * sizeof(int32_t) + 255) / 256);
    size_t dist_cells = 0;
    if (nostore) dist_cells = 0;                               // reductions only
    else if (!dist_block) dist_cells = (size_t)lanes * g->n;   // one pass's block, kept on the device
    else if (!out_dev) dist_cells = (size_t)k * g->n;          // staging for a host block
    const size_t tmp_bytes = off_dist + dist_cells * cell + 256;
    DAWN_CUDA_TRY(cudaMallocAsync(&tmp, tmp_bytes, st));
    char* t8 = static_cast<char*>(tmp);
    int32_t* d_src = reinterpret_cast<int32_t*>(t8 + off_src);
    int32_t* d_ecc = ecc_dev ? ecc : reinterpret_cast<int32_t*>(t8 + off_ecc);
    long long* d_dsum = dsum_dev ? reinterpret_cast<long long*>(dsum) : reinterpret_cast<long long*>(t8 + off_dsum);
    int32_t* d_reached = reached_dev ? reached : reinterpret_cast<int32_t*>(t8 + off_reached);
    void* d_out = out_dev ? dist_block : static_cast<void*>(t8 + off_dist);
    double* d_clos = closeness ? (clos_dev ? closeness : reinterpret_cast<double*>(t8 + off_clos)) : nullptr;
    double* d_harm = harmonic ? (harm_dev ? harmonic : reinterpret_cast<double*>(t8 + off_harm)) : nullptr;
    int32_t* d_ring = reinterpret_cast<int32_t*>(t8 + off_ring);
    long long* d_sum = reinterpret_cast<long long*>(t8 + off_sum);
    int32_t* d_hist = reinterpret_cast<int32_t*>(t8 + off_hist);
    cudaError_t e = cudaMemcpyAsync(d_src, hsrc.data(), sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_harm) e = cudaMemsetAsync(d_ring, 0, 3 * kMsMaxLanes * sizeof(int32_t), st);
    if (e == cudaSuccess && d_harm && sliced)
        e = cudaMemsetAsync(d_hist, 0, (size_t)(kNbLevelsMax + 1) * kMsMaxLanes * sizeof(int32_t), st);

    MsArgs a;
    a.in_ptr = g->in_ptr;
    a.in_idx = g->in_idx;
    a.excl = g->excl;
    a.sources = d_src;
    a.V0 = g->ms_vis[0];
    a.V1 = g->ms_vis[1];
    a.acc = reinterpret_cast<unsigned long long*>(g->ms_acc);
    a.ecc = d_ecc;
    a.dsum = d_dsum;
    a.reached = d_reached;
    char* cbase = reinterpret_cast<char*>(g->ms_counts);
    a.part_i = reinterpret_cast<int32_t*>(cbase);
    a.part_l = reinterpret_cast<long long*>(cbase + (size_t)g->sms * kMsMaxLanes * 2 * sizeof(int32_t));
    MsCtl* ctl = reinterpret_cast<MsCtl*>(
        (reinterpret_cast<uintptr_t>(cbase + (size_t)g->sms * kMsMaxLanes * (2 * sizeof(int32_t) + sizeof(long long))) + 255) &
        ~(uintptr_t)255);
    a.ctl = ctl;
    // NB[1] of another lane width overlaps that width's NB[2], which is not
    // cleared after a run
    if (sliced && g->ms_sliced_w != W) g->ms_vis_dirty = 1;
    if (e == cudaSuccess && sliced && g->ms_vis_dirty) {
        // the sliced kernel starts from zero visited words, a zero NB[1] and
        // zero level slots; the per-level kernel or a failed run left others
        e = cudaMemsetAsync(g->ms_vis[0], 0, plane_bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->ms_vis[1], 0, plane_bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->ms_nb, 0, plane_bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->lanes_new[0][0], 0, sizeof(ctl->lanes_new), st);
        if (e == cudaSuccess) {
            g->ms_vis_dirty = 0;
            g->ms_sliced_w = W;
        }
    }
    a.spin_limit = spin;
    a.n = g->n;
    a.k = k;
    a.dist_bytes = dist_bytes;
    a.bar_parity = (int)(g->ms_launches & 1u);
    a.trace = opts ? reinterpret_cast<long long*>(opts->trace) : nullptr;
    a.trace_cap = (opts && opts->trace) ? opts->trace_cap : 0;
    if (a.trace && (a.trace_cap < 0 || !is_device_ptr(a.trace))) {
        cudaFreeAsync(tmp, st);
        return fail(DAWN_E_INVALID, "trace must be device memory with trace_cap >= 0");
    }
    a.out = d_out;
    a.nostore = nostore ? 1 : 0;
    a.ring = d_harm ? d_ring : nullptr;
    a.harm = d_harm;
    a.clos = d_clos;
    if (nostore) a.dist_bytes = 4;  // nothing is stored: no int16 limit
    if (!dist_block) {
        // no caller block: every pass writes its rows into one device block of `lanes` rows
        a.layout = DAWN_SOURCE_MAJOR;
        a.per_pass = 1;
        a.out_row_stride = g->n;
    } else {
        a.layout = layout;
        a.per_pass = 0;
        a.out_row_stride = layout == DAWN_SOURCE_MAJOR ? (long long)g->n : (long long)k;
    }
    int lrc = DAWN_OK;
    if (e == cudaSuccess && sliced) {
        const MsPlan* pl = static_cast<const MsPlan*>(g->ms_plan);
        MsSliced sp;
        sp.out_ptr = g->row_ptr;
        sp.out_idx = g->col_idx;
        sp.tasks = pl->tasks;
        sp.cta_task = pl->cta_task;
        sp.cta_hub = pl->cta_hub;
        sp.hub_v = pl->hub_v;
        sp.sell_vd = pl->sell_vd;
        sp.sell_idx = pl->sell_idx;
        sp.nbl = g->ms_nb;
        sp.nb_levels = std::min(kNbLevelsMax, g->ms_nb_levels * 4 / W);
        sp.planes = g->ms_planes;
        sp.planes_cap = g->ms_planes ? std::min(kPlanesMax, g->ms_planes_cap * 4 / W) : 0;
        sp.hist = d_harm ? d_hist : nullptr;
        if (W == 1) lrc = ms_launch_sliced_w<1>(g, a, sp, st);
        else if (W == 2) lrc = ms_launch_sliced_w<2>(g, a, sp, st);
        else lrc = ms_launch_sliced_w<4>(g, a, sp, st);
        if (lrc == DAWN_OK) g->ms_launches += 1;
    } else if (e == cudaSuccess) {
        if (W == 1) lrc = ms_launch_w<1>(g, a, st);
        else if (W == 2) lrc = ms_launch_w<2>(g, a, st);
        else lrc = ms_launch_w<4>(g, a, st);
        if (lrc == DAWN_OK) g->ms_launches += 1;
        g->ms_vis_dirty = 1;  // the per-level kernel leaves its last pass's words behind
    }
    if (e == cudaSuccess && lrc == DAWN_OK && dist_block && !out_dev)
        e = cudaMemcpyAsync(dist_block, d_out, (size_t)k * g->n * cell, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && lrc == DAWN_OK && ecc && !ecc_dev)
        e = cudaMemcpyAsync(ecc, d_ecc, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && lrc == DAWN_OK && dsum && !dsum_dev)
        e = cudaMemcpyAsync(dsum, d_dsum, sizeof(long long) * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && lrc == DAWN_OK && reached && !reached_dev)
        e = cudaMemcpyAsync(reached, d_reached, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && lrc == DAWN_OK && closeness && !clos_dev)
        e = cudaMemcpyAsync(closeness, d_clos, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && lrc == DAWN_OK && harmonic && !harm_dev)
        e = cudaMemcpyAsync(harmonic, d_harm, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, st);
    long long hsum[4] = {0, 0, 0, 0};
    if (e == cudaSuccess && lrc == DAWN_OK && summary) {
        apsp_summary_kernel<<<1, 1024, 0, st>>>(d_ecc, d_dsum, d_reached, k, d_sum);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hsum, d_sum, sizeof(hsum), cudaMemcpyDeviceToHost, st);
    }
    int status = 0;
    if (e == cudaSuccess && lrc == DAWN_OK)
        e = cudaMemcpyAsync(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (lrc != DAWN_OK) return lrc;
    if (e != cudaSuccess) return cuda_fail(e, "dawn_msbfs", __FILE__, __LINE__);
    if (status != DEV_OK) {
        DAWN_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(MsCtl), st));
        // a pass cut short can leave accumulator slots and visited words set
        DAWN_CUDA_TRY(cudaMemsetAsync(g->ms_acc, 0, sizeof(uint64_t) * (size_t)g->n * 4, st));
        g->ms_vis_dirty = 1;
        DAWN_CUDA_TRY(cudaStreamSynchronize(st));
        if (status == DEV_PLANES) {
            // more levels than the level arrays hold: 15 planes, else the per-level kernel
            // (harmonic centrality: the per-level kernel, which sums the levels as they end)
            if (harmonic && want != DAWN_MSBFS_SLICED) {
                g->ms_harm_deep = 1;
            } else if (harmonic) {
                return fail(DAWN_E_INVALID, "harmonic centrality on the sliced kernel needs at most %d levels; "
                                            "use DAWN_MSBFS_PER_LEVEL", kNbLevelsMax);
            } else if (g->ms_planes_cap < kPlanesMax && (size_t)kPlanesMax * plane_bytes <= kPlanesBudget) {
                if ((rc = ms_planes_alloc(g, kPlanesMax)) != DAWN_OK) return rc;
            } else if (want == DAWN_MSBFS_SLICED) {
                return fail(DAWN_E_INVALID, "a pass needs more levels than the sliced kernel's planes hold "
                                            "(%d); use DAWN_MSBFS_PER_LEVEL", (1 << kPlanesMax) - 1);
            } else {
                g->ms_sliced_off = 1;
            }
            return msbfs_run(g, sources, k, dist_block, dist_bytes, layout, ecc, dsum, reached, opts, st,
                             closeness, harmonic, summary, nostore);
        }
        if (status == DEV_OVERFLOW) return fail(DAWN_E_OVERFLOW, "a distance exceeded the int16 range (32767)");
        if (status == DEV_TIMEOUT) return fail(DAWN_E_TIMEOUT, "a grid-barrier wait on the device ran out of its spin budget");
        return fail(DAWN_E_CUDA, "unknown device status %d", status);
    }
    if (summary) {
        summary->diameter = (int32_t)hsum[0];
        summary->radius = (int32_t)hsum[1];
        summary->pairs = hsum[2];
        summary->dist_total = hsum[3];
    }
    return DAWN_OK;
}

}  // namespace

void ms_release(dawn_graph* g) {
    if (g->ms_plan) {
        auto* pl = static_cast<MsPlan*>(g->ms_plan);
        if (pl->blob) cudaFree(pl->blob);
        delete pl;
        g->ms_plan = nullptr;
    }
    if (g->ms_planes) cudaFree(g->ms_planes);
    g->ms_planes = nullptr;
    g->ms_planes_cap = 0;
    if (g->ms_nb) cudaFree(g->ms_nb);
    g->ms_nb = nullptr;
    g->ms_nb_levels = 0;
}

}  // namespace dawn

extern "C" {

DAWN_API int dawn_msbfs_ex(dawn_graph_t g, const int32_t* sources, int32_t k, void* dist_block,
                           int dist_bytes, int layout, int32_t* ecc, int64_t* dsum, int32_t* reached,
                           const dawn_msbfs_opts* opts, void* stream) {
    return dawn::msbfs_run(g, sources, k, dist_block, dist_bytes, layout, ecc, dsum, reached, opts,
                           (cudaStream_t)stream);
}

DAWN_API int dawn_centrality(dawn_graph_t g, const int32_t* sources, int32_t k, int32_t* ecc, int64_t* dsum,
                             int32_t* reached, double* closeness, double* harmonic, dawn_apsp_summary* summary,
                             const dawn_msbfs_opts* opts, void* stream) {
    return dawn::msbfs_run(g, sources, k, nullptr, 4, DAWN_SOURCE_MAJOR, ecc, dsum, reached, opts,
                           (cudaStream_t)stream, closeness, harmonic, summary, true);
}

DAWN_API int dawn_msbfs(dawn_graph_t g, const int32_t* sources, int32_t k, void* dist_block,
                        int dist_bytes, int layout, int32_t* ecc, int64_t* dsum, void* stream) {
    return dawn_msbfs_ex(g, sources, k, dist_block, dist_bytes, layout, ecc, dsum, nullptr, nullptr, stream);
}

}  // extern "C"
