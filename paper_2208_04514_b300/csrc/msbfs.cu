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
// covered for every running lane is skipped.  The kernel is persistent and
// cooperative: batches, their levels and the per-batch reductions
// (eccentricity = largest finite distance, distance sum, reached count, from
// per-level counts) all run in one launch, separated by the bounded grid
// barrier.
#include <climits>
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
        const size_t bytes = sizeof(uint64_t) * (size_t)g->n * 4;  // room for W = 4
        DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_vis[0], bytes));
        DAWN_CUDA_TRY(cudaMalloc((void**)&g->ms_vis[1], bytes));
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

    // sources: checked on the host whatever memory they live in
    std::vector<int32_t> hsrc((size_t)k);
    DAWN_CUDA_TRY(cudaMemcpy(hsrc.data(), sources, sizeof(int32_t) * (size_t)k, cudaMemcpyDefault));
    for (int32_t i = 0; i < k; ++i)
        if (hsrc[i] < 0 || hsrc[i] >= g->n) return fail(DAWN_E_INVALID, "sources[%d] = %d outside [0, %d)", i, hsrc[i], g->n);

    int rc = ms_workspace(g, W);
    if (rc != DAWN_OK) return rc;

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
    size_t off_dist = off_sum + 256;
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
    cudaError_t e = cudaMemcpyAsync(d_src, hsrc.data(), sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_harm) e = cudaMemsetAsync(d_ring, 0, 3 * kMsMaxLanes * sizeof(int32_t), st);

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
    if (e == cudaSuccess) {
        if (W == 1) lrc = ms_launch_w<1>(g, a, st);
        else if (W == 2) lrc = ms_launch_w<2>(g, a, st);
        else lrc = ms_launch_w<4>(g, a, st);
        if (lrc == DAWN_OK) g->ms_launches += 1;
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
        // a pass cut short can leave accumulator slots set
        DAWN_CUDA_TRY(cudaMemsetAsync(g->ms_acc, 0, sizeof(uint64_t) * (size_t)g->n * 4, st));
        DAWN_CUDA_TRY(cudaStreamSynchronize(st));
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
