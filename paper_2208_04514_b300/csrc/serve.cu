// Continuous-batching DAWN server: a device-resident request loop over several
// resident graphs.
//
// Every source of every request becomes one bit lane of its graph (64 * W
// lanes per graph).  One persistent cooperative kernel runs "iterations": in
// each, every occupied lane of every graph advances its own BFS by one level
// with the bit-lane BOVM pull of Alg. 1 / Eq. 4 (new = OR over in-neighbours
// of the step-start visited words, AND NOT the vertex's own).  A lane admitted
// at iteration t0 writes dist = t - t0 for the vertices it reaches at
// iteration t, so its row is exactly the single-source result whatever else
// shares the device (Thm 1: the first level at which a vertex is reached).
//
// Host <-> device protocol (device-mapped pinned memory):
//   * admission slot: the host thread writes one sorted batch of
//     {graph, lane, source, row address, element size, token} entries and
//     bumps batch_seq; at the end of an iteration CTA 0 copies it into device
//     memory, acknowledges it, and the lanes start at the next iteration.
//   * completion ring: when a lane's level reaches nothing, its row is final;
//     CTA 0 appends {token, levels, status} and bumps done_tail.
// Lanes are assigned only by the host, only from lanes whose completion it has
// seen, so a re-admitted lane is never still running.  A re-admitted lane's
// stale bits are masked off during its first iteration (and written back
// cleared).  Every wait is bounded; the kernel leaves when it has been idle
// for a while or when the host asks it to stop, and the host relaunches it on
// the next admission.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

constexpr int kSvThreads = 1024;
constexpr int kSvWarps = kSvThreads / 32;
constexpr int kSvMaxGraphs = 16;
constexpr int kSvMaxLanes = 256;
constexpr int kSvMaxAdmit = 1024;          // entries per admission batch
constexpr int kSvDoneRing = 1 << 16;       // completion records
constexpr int kSvSerial = 8;
constexpr int kSvHeavy = 512;
constexpr int kSvHeavyMax = 32;
constexpr long long kSvSegBytes = 1 << 16; // row-fill work item
constexpr unsigned kFull = 0xffffffffu;

struct AdmitEntry {
    int32_t graph;
    int32_t lane;
    int32_t src;
    int32_t bytes;          // 2 or 4
    unsigned long long row; // device address of the lane's distance row
    unsigned long long token;
};

struct DoneRec {
    unsigned long long token;
    int32_t levels;
    int32_t status;         // DEV_OK or DEV_OVERFLOW
};

// Device-mapped pinned memory shared with the host thread.
struct HostShared {
    volatile unsigned int batch_seq;   // host: bumped after a batch is written
    volatile unsigned int batch_ack;   // device: last batch consumed
    volatile unsigned int stop;        // host: leave the loop
    volatile unsigned int pad0;
    volatile unsigned long long done_tail;  // device: records appended
    volatile unsigned long long done_head;  // host: records consumed
    unsigned int count;
    unsigned int pad1;
    AdmitEntry entries[kSvMaxAdmit];
    DoneRec done[kSvDoneRing];
};

// Per graph, device memory.
struct SvGraph {
    const int32_t* in_ptr;
    const int32_t* in_idx;
    const uint32_t* excl;
    uint64_t* V[2];
    int32_t n;
    int32_t pad;
    int32_t lane_start[kSvMaxLanes];
    int32_t lane_bytes[kSvMaxLanes];
    unsigned long long lane_row[kSvMaxLanes];
    unsigned long long lane_token[kSvMaxLanes];
};

struct alignas(128) SvCtl {
    BarCounter bar[2];
    int status;
    int pad[31];
    unsigned long long lanes_new[3][kSvMaxGraphs][4];
    // published by CTA 0 for iteration t into pub[t & 1]: {admitted entries,
    // exit flag, first entry of each graph (kSvMaxGraphs + 1 values)}
    int pub[2][32];
    AdmitEntry admit[2][kSvMaxAdmit];     // sorted by (graph, src)
    long long seg_prefix[2][kSvMaxAdmit + 1];  // row-fill work items before each entry
};

struct SvArgs {
    SvGraph* graphs;
    SvCtl* ctl;
    HostShared* hs;       // device pointer of the mapped block
    long long spin_limit;
    long long idle_ns;
    int ngraphs;
    int bar_parity;
};

__device__ __forceinline__ unsigned sv_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned sv_ld_acquire_sys(const volatile unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int sv_ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long sv_ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long sv_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Admission entries and lane tables are rewritten by CTA 0 between
// iterations; every other CTA reads them through L2 (ld.global.cg).
__device__ __forceinline__ AdmitEntry ld_entry(const AdmitEntry* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 x = __ldcg(q), y = __ldcg(q + 1);
    AdmitEntry e;
    e.graph = (int32_t)(x.x & 0xffffffffull);
    e.lane = (int32_t)(x.x >> 32);
    e.src = (int32_t)(x.y & 0xffffffffull);
    e.bytes = (int32_t)(x.y >> 32);
    e.row = y.x;
    e.token = y.y;
    return e;
}

// With `snap`, thread 0 copies nsnap ints after the acquire into s_snap
// for the whole CTA (one L2 request per CTA, not one per warp).
__device__ bool sv_barrier(SvCtl* ctl, unsigned* count, unsigned& target, long long spin_limit,
                           const int* snap = nullptr, int nsnap = 0, int* s_snap = nullptr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const long long t0 = clock64();
        unsigned polls = 0;
        while ((int)(sv_ld_acquire(count) - target) < 0) {
            if (clock64() - t0 > spin_limit) {
                atomicCAS(&ctl->status, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
            if ((++polls & 15u) == 0 && sv_ld_relaxed_s32(&ctl->status) != DEV_OK) { ok = 0; break; }
        }
        if (ok)
            for (int i = 0; i < nsnap; ++i) s_snap[i] = sv_ld_relaxed_s32(snap + i);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ unsigned long long sv_warp_or64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ void sv_store(unsigned long long row, int bytes, long long v, int value) {
    if (bytes == 2) reinterpret_cast<int16_t*>(row)[v] = (int16_t)value;
    else reinterpret_cast<int32_t*>(row)[v] = value;
}

template <int W>
__global__ void __launch_bounds__(kSvThreads, 1) serve_kernel(SvArgs a) {
    constexpr int L = 64 * W;
    __shared__ int s_start[kSvMaxLanes];
    __shared__ int s_bytes[kSvMaxLanes];
    __shared__ unsigned long long s_row[kSvMaxLanes];
    __shared__ int s_asrc[kSvMaxAdmit];      // this graph's admitted sources (sorted)
    __shared__ int s_alane[kSvMaxAdmit];
    __shared__ unsigned long long s_newmask[4];
    __shared__ int s_hcount;
    __shared__ int s_hv[kSvHeavyMax], s_hj[kSvHeavyMax], s_hie[kSvHeavyMax];
    __shared__ unsigned long long s_hvv[kSvHeavyMax][W], s_hacc[kSvHeavyMax][W], s_hseed[kSvHeavyMax][W];
    __shared__ int s_exit;

    SvCtl* ctl = a.ctl;
    HostShared* hs = a.hs;
    __shared__ int s_pub[32];  // this iteration's {entries, exit flag, first entry per graph}
    __shared__ int s_status;
    if (threadIdx.x == 0) s_status = sv_ld_relaxed_s32(&ctl->status);
    __syncthreads();
    if (s_status != DEV_OK) return;
    unsigned* bar = &ctl->bar[a.bar_parity].count;
    unsigned bar_target = 0;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kSvWarps + (threadIdx.x >> 5);
    const int nw = gridDim.x * kSvWarps;
    const long long gtid = (long long)blockIdx.x * kSvThreads + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * kSvThreads;

    // lanes holding a BFS, per graph (the same in every CTA)
    __shared__ unsigned long long occ[kSvMaxGraphs][W];
    for (int i = threadIdx.x; i < kSvMaxGraphs * W; i += kSvThreads) (&occ[0][0])[i] = 0ull;
    unsigned long long last_busy = sv_globaltimer();
    unsigned int seen_seq = 0;  // CTA 0, thread 0: last admission batch taken

    if (threadIdx.x == 0) s_hcount = 0;
    if (threadIdx.x < 4) s_newmask[threadIdx.x] = 0;

    // iteration -1: CTA 0 picks up a batch that is already waiting
    if (blockIdx.x == 0) {
        __shared__ int s_take;
        if (threadIdx.x == 0) {
            seen_seq = sv_ld_acquire_sys(&hs->batch_ack);
            const unsigned seq = sv_ld_acquire_sys(&hs->batch_seq);
            s_take = seq != seen_seq ? (int)min(hs->count, (unsigned)kSvMaxAdmit) : -1;
            if (s_take >= 0) seen_seq = seq;
            for (int i = 0; i < 32; ++i) ctl->pub[0][i] = ctl->pub[1][i] = 0;
        }
        __syncthreads();
        const int take = s_take;
        if (take > 0) {
            for (int i = threadIdx.x; i < take; i += kSvThreads) ctl->admit[0][i] = hs->entries[i];
            __syncthreads();
            if (threadIdx.x == 0) {
                long long acc = 0;
                for (int i = 0; i < take; ++i) {
                    const AdmitEntry e = ctl->admit[0][i];
                    const long long rb = (long long)a.graphs[e.graph].n * e.bytes;
                    ctl->seg_prefix[0][i] = acc;
                    acc += (rb + kSvSegBytes - 1) / kSvSegBytes;
                    SvGraph* G = &a.graphs[e.graph];
                    G->lane_start[e.lane] = 0;
                    G->lane_bytes[e.lane] = e.bytes;
                    G->lane_row[e.lane] = e.row;
                    G->lane_token[e.lane] = e.token;
                }
                ctl->seg_prefix[0][take] = acc;
                ctl->pub[0][0] = take;
                int gi = 0;
                for (int g = 0; g <= kSvMaxGraphs; ++g) {
                    while (gi < take && ctl->admit[0][gi].graph < g) ++gi;
                    ctl->pub[0][2 + g] = gi;
                }
                __threadfence_system();
                *(volatile unsigned*)&hs->batch_ack = seen_seq;
            }
        }
        if (threadIdx.x < 3 * kSvMaxGraphs * 4) (&ctl->lanes_new[0][0][0])[threadIdx.x] = 0ull;
    }
    if (!sv_barrier(ctl, bar, bar_target, a.spin_limit, ctl->pub[0], 2 + kSvMaxGraphs + 1, s_pub)) return;

    for (int t = 0;; ++t) {
        const int par = t & 1;
        const int na = s_pub[0];
        const long long* seg = ctl->seg_prefix[par];
        // ---- (1) fill the rows of lanes admitted now: -1, and 0 at the source
        if (na > 0) {
            const long long items = __ldcg(seg + na);
            for (long long it = blockIdx.x; it < items; it += gridDim.x) {
                int lo = 0, hi = na;  // entry with seg_prefix[e] <= it < seg_prefix[e + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldcg(seg + mid) <= it) lo = mid; else hi = mid;
                }
                const AdmitEntry e = ld_entry(&ctl->admit[par][lo]);
                const long long rb = (long long)a.graphs[e.graph].n * e.bytes;
                const long long off = (it - __ldcg(seg + lo)) * kSvSegBytes;
                const long long len = min(kSvSegBytes, rb - off);
                char* p = reinterpret_cast<char*>(e.row) + off;
                if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (len & 15) == 0) {
                    for (long long i = threadIdx.x; i < len / 16; i += kSvThreads)
                        reinterpret_cast<int4*>(p)[i] = make_int4(-1, -1, -1, -1);
                } else {
                    for (long long i = threadIdx.x; i < len / e.bytes; i += kSvThreads)
                        sv_store((unsigned long long)p, e.bytes, i, -1);
                }
                __syncthreads();
                const long long srcoff = (long long)e.src * e.bytes;
                if (threadIdx.x == 0 && srcoff >= off && srcoff < off + len) sv_store(e.row, e.bytes, e.src, 0);
            }
        }
        // ---- (2) one level for every graph with occupied or admitted lanes
        for (int g = 0; g < a.ngraphs; ++g) {
            const int a0 = s_pub[2 + g];  // admitted entries are sorted by graph
            const int ai = s_pub[2 + g + 1];
            const int nag = ai - a0;
            unsigned long long adm[W];
            bool any = false;
#pragma unroll
            for (int w = 0; w < W; ++w) { adm[w] = 0ull; any |= occ[g][w] != 0ull; }
            for (int i = a0; i < ai; ++i) {
                const int ln = ld_entry(&ctl->admit[par][i]).lane;
                adm[ln >> 6] |= 1ull << (ln & 63);
            }
            if (!any && nag == 0) continue;
            SvGraph* G = &a.graphs[g];
            const int n = G->n;
            uint64_t* vcur = G->V[t & 1];
            uint64_t* vnext = G->V[(t & 1) ^ 1];
            // lanes that expand this iteration: occupied before now
            unsigned long long fin[W];
#pragma unroll
            for (int w = 0; w < W; ++w) fin[w] = ~occ[g][w];
            __syncthreads();
            for (int i = threadIdx.x; i < L; i += kSvThreads) {
                s_start[i] = __ldcg(G->lane_start + i);
                s_bytes[i] = __ldcg(G->lane_bytes + i);
                s_row[i] = __ldcg(G->lane_row + i);
            }
            for (int i = threadIdx.x; i < nag; i += kSvThreads) {
                const AdmitEntry e = ld_entry(&ctl->admit[par][a0 + i]);
                s_asrc[i] = e.src;
                s_alane[i] = e.lane;
            }
            __syncthreads();
            for (int vb = gw << 5; vb < n; vb += nw << 5) {
                const int v = vb + lane;
                const bool valid = v < n;
                unsigned long long vv[W], acc[W], seed[W];
                bool need = false;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    vv[w] = valid ? (__ldcg(vcur + (long long)v * W + w) & ~adm[w]) : ~0ull;
                    acc[w] = 0ull;
                    seed[w] = 0ull;
                    need |= (vv[w] | fin[w]) != ~0ull;
                }
                // admitted sources inside [vb, vb + 32)
                if (nag > 0 && valid) {
                    int lo = 0, hi = nag;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (s_asrc[mid] < v) lo = mid + 1; else hi = mid;
                    }
                    for (int i = lo; i < nag && s_asrc[i] == v; ++i) seed[s_alane[i] >> 6] |= 1ull << (s_alane[i] & 63);
                }
                if (valid && need && ((__ldg(G->excl + (v >> 5)) >> (v & 31)) & 1u)) need = false;
                int j = 0, ie = 0;
                if (need) {
                    const int ib = __ldg(G->in_ptr + v);
                    ie = __ldg(G->in_ptr + v + 1);
                    j = ib;
                    const int jl = min(ie, ib + kSvSerial);
                    for (; j < jl; ++j) {
                        const int u = __ldg(G->in_idx + j);
                        bool all = true;
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            acc[w] |= __ldcg(vcur + (long long)u * W + w) & ~adm[w];
                            all &= (acc[w] | vv[w] | fin[w]) == ~0ull;
                        }
                        if (all) { j = ie; break; }
                    }
                }
                bool deferred = false;
                if (need && ie - j > kSvHeavy) {
                    const int slot = atomicAdd(&s_hcount, 1);
                    if (slot < kSvHeavyMax) {
                        deferred = true;
                        s_hv[slot] = v;
                        s_hj[slot] = j;
                        s_hie[slot] = ie;
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            s_hvv[slot][w] = vv[w];
                            s_hacc[slot][w] = acc[w];
                            s_hseed[slot][w] = seed[w];
                        }
                    }
                }
                unsigned rest = __ballot_sync(kFull, need && !deferred && j < ie);
                while (rest) {
                    const int sl = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const int jb = __shfl_sync(kFull, j, sl);
                    const int je = __shfl_sync(kFull, ie, sl);
                    unsigned long long accL[W], vvL[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        accL[w] = __shfl_sync(kFull, acc[w], sl);
                        vvL[w] = __shfl_sync(kFull, vv[w], sl);
                    }
                    for (int base = jb; base < je; base += 32) {
                        const int jj = base + lane;
                        const int u = jj < je ? __ldg(G->in_idx + jj) : -1;
                        bool all = true;
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            const unsigned long long x = u >= 0 ? (__ldcg(vcur + (long long)u * W + w) & ~adm[w]) : 0ull;
                            accL[w] |= sv_warp_or64(x);
                            all &= (accL[w] | vvL[w] | fin[w]) == ~0ull;
                        }
                        if (all) break;
                    }
                    if (lane == sl) {
#pragma unroll
                        for (int w = 0; w < W; ++w) acc[w] = accL[w];
                    }
                }
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const unsigned long long nb = (need && !deferred) ? (acc[w] & ~vv[w] & ~fin[w]) : 0ull;
                    if (valid && !deferred) vnext[(long long)v * W + w] = vv[w] | nb | seed[w];
                    unsigned long long uni = sv_warp_or64(nb);
                    if (lane == 0 && uni) atomicOr(&s_newmask[w], uni);
                    while (uni) {
                        const int bit = __ffsll((long long)uni) - 1;
                        uni &= uni - 1;
                        const int s = w * 64 + bit;
                        if ((nb >> bit) & 1ull) sv_store(s_row[s], s_bytes[s], v, t - s_start[s]);
                    }
                }
            }
            __syncthreads();
            const int nh = min(s_hcount, kSvHeavyMax);
            for (int h = 0; h < nh; ++h) {
                unsigned long long part[W];
#pragma unroll
                for (int w = 0; w < W; ++w) part[w] = 0ull;
                const int hie = s_hie[h];
                for (int jj = s_hj[h] + threadIdx.x; jj < hie; jj += kSvThreads) {
                    const int u = __ldg(G->in_idx + jj);
#pragma unroll
                    for (int w = 0; w < W; ++w) part[w] |= __ldcg(vcur + (long long)u * W + w) & ~adm[w];
                }
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    part[w] = sv_warp_or64(part[w]);
                    if (lane == 0 && part[w]) atomicOr(&s_hacc[h][w], part[w]);
                }
            }
            __syncthreads();
            for (int h = threadIdx.x >> 5; h < nh; h += kSvWarps) {
                const int v = s_hv[h];
                unsigned long long nbw[W];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    nbw[w] = s_hacc[h][w] & ~s_hvv[h][w] & ~fin[w];
                    if (lane == w) vnext[(long long)v * W + w] = s_hvv[h][w] | nbw[w] | s_hseed[h][w];
                    if (lane == 0 && nbw[w]) atomicOr(&s_newmask[w], nbw[w]);
                }
                for (int i = lane; i < L; i += 32)
                    if ((nbw[i >> 6] >> (i & 63)) & 1ull) sv_store(s_row[i], s_bytes[i], v, t - s_start[i]);
            }
            __syncthreads();
            if (threadIdx.x == 0) s_hcount = 0;
            if (threadIdx.x < W) {
                if (s_newmask[threadIdx.x]) atomicOr(&ctl->lanes_new[t % 3][g][threadIdx.x], s_newmask[threadIdx.x]);
                s_newmask[threadIdx.x] = 0;
            }
            // lanes admitted now start counting at this iteration (all threads
            // have read occ[g] above; the next graph's first barrier orders this)
            if (threadIdx.x == 0) {
#pragma unroll
                for (int w = 0; w < W; ++w) occ[g][w] |= adm[w];
            }
        }
        // ---- (3) CTA 0: next batch from the host, idle / stop decision
        if (blockIdx.x == 0) {
            __shared__ int s_take;
            const int npar = par ^ 1;
            if (threadIdx.x == 0) {
                const unsigned seq = sv_ld_acquire_sys(&hs->batch_seq);
                s_take = (seq != seen_seq) ? (int)min(hs->count, (unsigned)kSvMaxAdmit) : 0;
                if (seq != seen_seq) seen_seq = seq;
            }
            if (threadIdx.x < kSvMaxGraphs * 4) (&ctl->lanes_new[(t + 1) % 3][0][0])[threadIdx.x] = 0ull;
            __syncthreads();
            const int take = min(s_take, kSvMaxAdmit);
            for (int i = threadIdx.x; i < take; i += kSvThreads) ctl->admit[npar][i] = hs->entries[i];
            __syncthreads();
            if (threadIdx.x == 0) {
                long long acc = 0;
                for (int i = 0; i < take; ++i) {
                    const AdmitEntry e = ctl->admit[npar][i];
                    const long long rb = (long long)a.graphs[e.graph].n * e.bytes;
                    ctl->seg_prefix[npar][i] = acc;
                    acc += (rb + kSvSegBytes - 1) / kSvSegBytes;
                    SvGraph* G = &a.graphs[e.graph];
                    G->lane_start[e.lane] = t + 1;
                    G->lane_bytes[e.lane] = e.bytes;
                    G->lane_row[e.lane] = e.row;
                    G->lane_token[e.lane] = e.token;
                }
                ctl->seg_prefix[npar][take] = acc;
                ctl->pub[npar][0] = take;
                int gi = 0;
                for (int g = 0; g <= kSvMaxGraphs; ++g) {
                    while (gi < take && ctl->admit[npar][gi].graph < g) ++gi;
                    ctl->pub[npar][2 + g] = gi;
                }
                if (take > 0) {
                    __threadfence_system();
                    *(volatile unsigned*)&hs->batch_ack = seen_seq;
                }
                bool busy = take > 0;
                for (int g = 0; g < a.ngraphs; ++g)
                    for (int w = 0; w < W; ++w) busy |= occ[g][w] != 0ull;
                const unsigned long long now = sv_globaltimer();
                if (busy) last_busy = now;
                ctl->pub[npar][1] = (*(volatile unsigned*)&hs->stop != 0u) ||
                                    (!busy && (long long)(now - last_busy) > a.idle_ns);
            }
        }
        if (!sv_barrier(ctl, bar, bar_target, a.spin_limit, ctl->pub[par ^ 1], 2 + kSvMaxGraphs + 1, s_pub)) return;
        // ---- (4) lanes whose level reached nothing are done (thread 0 of every
        //      CTA computes the same masks; CTA 0 reports them to the host)
        if (threadIdx.x == 0) {
            for (int g = 0; g < a.ngraphs; ++g) {
                SvGraph* G = &a.graphs[g];
                for (int w = 0; w < W; ++w) {
                    if (!occ[g][w]) continue;
                    const unsigned long long got = sv_ld_relaxed_u64(&ctl->lanes_new[t % 3][g][w]);
                    unsigned long long started_now = 0ull, over = 0ull;
                    unsigned long long m = occ[g][w];
                    while (m) {
                        const int b = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        const int s = w * 64 + b;
                        const int st = __ldcg(G->lane_start + s);
                        if (st == t) started_now |= 1ull << b;  // admitted now: has not expanded yet
                        else if (__ldcg(G->lane_bytes + s) == 2 && t + 1 - st > 32767) over |= 1ull << b;
                    }
                    const unsigned long long fin = ((occ[g][w] & ~got) & ~started_now) | over;
                    if (fin && blockIdx.x == 0) {
                        unsigned long long f = fin;
                        while (f) {
                            const int b = __ffsll((long long)f) - 1;
                            f &= f - 1;
                            const int s = w * 64 + b;
                            const unsigned long long tail = hs->done_tail;
                            const bool ov = (over >> b) & 1ull;
                            volatile DoneRec* dst = &hs->done[tail % kSvDoneRing];
                            dst->token = __ldcg(G->lane_token + s);
                            dst->levels = ov ? -1 : t - 1 - __ldcg(G->lane_start + s);
                            dst->status = ov ? DEV_OVERFLOW : DEV_OK;
                            __threadfence_system();
                            hs->done_tail = tail + 1;
                        }
                    }
                    occ[g][w] &= ~fin;
                }
            }
        }
        __syncthreads();
        if (s_pub[1]) break;
    }
    if (gtid == 0) ctl->bar[a.bar_parity ^ 1].count = 0;
}

// ------------------------------------------------------------------ host side

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    int graph = 0;
    std::vector<int32_t> sources;
    int dist_bytes = 2;
    void* dist_out = nullptr;
    bool out_dev = false;
    char* block = nullptr;        // device rows (the caller's block, or staging in the arena)
    size_t block_bytes = 0;
    size_t arena_off = 0;
    bool staged = false;
    int next = 0;                 // next source to admit
    int rows_done = 0;
    int state = DAWN_REQ_PENDING;
    int err = DAWN_OK;
    double t_submit = 0, t_done = 0;
    cudaEvent_t copied = nullptr;
};

}  // namespace
}  // namespace dawn

struct dawn_server {
    std::vector<dawn_graph*> graphs;
    int lanes = 256;
    int W = 4;
    int sms = 0;
    size_t budget = 0;
    char* arena = nullptr;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    size_t arena_used = 0;
    dawn::SvGraph* d_graphs = nullptr;
    dawn::SvCtl* d_ctl = nullptr;
    dawn::HostShared* hs = nullptr;       // host view (mapped)
    dawn::HostShared* hs_dev = nullptr;   // device view
    std::vector<std::vector<int>> free_lanes;                       // per graph
    std::vector<std::vector<std::pair<uint64_t, int>>> lane_owner;  // per graph: (request, row)
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool kernel_live = false;
    unsigned launches = 0;
    unsigned batch_seq = 0;
    uint64_t next_id = 1;
    unsigned long long token_next = 1;
    std::map<unsigned long long, std::pair<uint64_t, int>> tokens;  // token -> (request, graph lane)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;                    // submitted, not fully admitted
    std::map<uint64_t, dawn::Request*> reqs;
    std::atomic<bool> stop{false};
    std::thread worker;
    int fatal = DAWN_OK;
    int device = 0;
};

namespace dawn {
namespace {

bool arena_alloc(dawn_server* s, size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t noff = it->first + bytes;
            s->free_blocks.erase(it);
            if (rest) s->free_blocks[noff] = rest;
            s->arena_used += bytes;
            return true;
        }
    }
    return false;
}

void arena_free(dawn_server* s, size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    s->arena_used -= bytes;
    auto it = s->free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blocks.erase(nx);
    }
    if (it != s->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blocks.erase(it);
        }
    }
}

int launch_kernel(dawn_server* s) {
    SvArgs a;
    a.graphs = s->d_graphs;
    a.ctl = s->d_ctl;
    a.hs = s->hs_dev;
    a.spin_limit = kDefaultSpin;
    a.idle_ns = 2000000;  // leave after 2 ms without work
    a.ngraphs = (int)s->graphs.size();
    a.bar_parity = (int)(s->launches & 1u);
    void* args[] = {&a};
    dim3 grid(s->sms), block(kSvThreads);
    cudaError_t e;
    if (s->W == 1) e = cudaLaunchCooperativeKernel((const void*)serve_kernel<1>, grid, block, args, 0, s->kstream);
    else if (s->W == 2) e = cudaLaunchCooperativeKernel((const void*)serve_kernel<2>, grid, block, args, 0, s->kstream);
    else e = cudaLaunchCooperativeKernel((const void*)serve_kernel<4>, grid, block, args, 0, s->kstream);
    if (e != cudaSuccess) return cuda_fail(e, "serve kernel launch", __FILE__, __LINE__);
    s->launches += 1;
    cudaEventRecord(s->kdone, s->kstream);
    s->kernel_live = true;
    return DAWN_OK;
}

void fail_all(dawn_server* s, int code) {
    for (auto& kv : s->reqs) {
        Request* r = kv.second;
        if (r->state == DAWN_REQ_PENDING || r->state == DAWN_REQ_RUNNING) {
            r->state = DAWN_REQ_FAILED;
            r->err = code;
            r->t_done = now_s();
        }
    }
    s->queue.clear();
}

// One pass of the host side of the loop.  Called with s->mu held.
bool service(dawn_server* s) {
    bool progress = false;
    // ---- completions
    const unsigned long long tail = s->hs->done_tail;
    unsigned long long head = s->hs->done_head;
    std::atomic_thread_fence(std::memory_order_acquire);
    while (head < tail) {
        const DoneRec r = *const_cast<const DoneRec*>(&s->hs->done[head % kSvDoneRing]);
        ++head;
        progress = true;
        auto it = s->tokens.find(r.token);
        if (it == s->tokens.end()) continue;
        const uint64_t rid = it->second.first;
        const int glane = it->second.second;
        s->tokens.erase(it);
        Request* q = s->reqs.count(rid) ? s->reqs[rid] : nullptr;
        const int g = glane / kSvMaxLanes, ln = glane % kSvMaxLanes;
        s->free_lanes[g].push_back(ln);
        if (!q) continue;
        if (r.status == DEV_OVERFLOW) q->err = DAWN_E_OVERFLOW;
        q->rows_done += 1;
        if (q->rows_done == (int)q->sources.size()) {
            if (!q->out_dev && q->err == DAWN_OK) {
                cudaMemcpyAsync(q->dist_out, q->block, q->block_bytes, cudaMemcpyDeviceToHost, s->cstream);
                cudaEventRecord(q->copied, s->cstream);
            } else {
                q->state = q->err == DAWN_OK ? DAWN_REQ_DONE : DAWN_REQ_FAILED;
                q->t_done = now_s();
                if (q->staged) { arena_free(s, q->arena_off, q->block_bytes); q->staged = false; }
            }
        }
    }
    s->hs->done_head = head;
    // ---- finished host copies
    for (auto& kv : s->reqs) {
        Request* q = kv.second;
        if (q->state == DAWN_REQ_RUNNING && q->rows_done == (int)q->sources.size() && !q->out_dev && q->err == DAWN_OK) {
            if (cudaEventQuery(q->copied) == cudaSuccess) {
                q->state = DAWN_REQ_DONE;
                q->t_done = now_s();
                if (q->staged) { arena_free(s, q->arena_off, q->block_bytes); q->staged = false; }
                progress = true;
            }
        }
    }
    // ---- admissions: one batch at a time, the device acknowledges it
    if (s->hs->batch_ack == s->batch_seq && !s->queue.empty()) {
        std::vector<AdmitEntry> batch;
        for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < kSvMaxAdmit;) {
            Request* q = s->reqs[*it];
            if (q->state == DAWN_REQ_FAILED) { it = s->queue.erase(it); continue; }
            if (!q->block) {
                // admission by device memory: a host-output request needs its staging block
                if (!arena_alloc(s, q->block_bytes, &q->arena_off)) { ++it; continue; }
                q->block = s->arena + q->arena_off;
                q->staged = true;
            }
            auto& fl = s->free_lanes[q->graph];
            while (q->next < (int)q->sources.size() && !fl.empty() && (int)batch.size() < kSvMaxAdmit) {
                const int ln = fl.back();
                fl.pop_back();
                AdmitEntry e;
                e.graph = q->graph;
                e.lane = ln;
                e.src = q->sources[q->next];
                e.bytes = q->dist_bytes;
                e.row = reinterpret_cast<unsigned long long>(q->block + (size_t)q->next * s->graphs[q->graph]->n * q->dist_bytes);
                e.token = s->token_next++;
                s->tokens[e.token] = {q->id, q->graph * kSvMaxLanes + ln};
                batch.push_back(e);
                q->next += 1;
                q->state = DAWN_REQ_RUNNING;
            }
            if (q->next == (int)q->sources.size()) it = s->queue.erase(it);
            else ++it;
        }
        if (!batch.empty()) {
            std::sort(batch.begin(), batch.end(), [](const AdmitEntry& x, const AdmitEntry& y) {
                return x.graph != y.graph ? x.graph < y.graph : x.src < y.src;
            });
            std::memcpy(s->hs->entries, batch.data(), batch.size() * sizeof(AdmitEntry));
            s->hs->count = (unsigned)batch.size();
            std::atomic_thread_fence(std::memory_order_seq_cst);
            s->batch_seq += 1;
            s->hs->batch_seq = s->batch_seq;
            progress = true;
        }
    }
    // ---- the device loop: relaunch when work is waiting and the last launch left
    if (s->kernel_live && cudaEventQuery(s->kdone) == cudaSuccess) {
        s->kernel_live = false;
        int status = 0;
        cudaMemcpy(&status, &s->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (status != DEV_OK) {
            s->fatal = status == DEV_TIMEOUT ? DAWN_E_TIMEOUT : DAWN_E_CUDA;
            cudaMemset(s->d_ctl, 0, sizeof(SvCtl));
            fail_all(s, s->fatal);
        }
    }
    const bool waiting = s->hs->batch_ack != s->batch_seq;
    bool lanes_busy = false;
    for (size_t g = 0; g < s->graphs.size(); ++g) lanes_busy |= (int)s->free_lanes[g].size() < s->lanes;
    if (!s->kernel_live && (waiting || lanes_busy) && !s->stop.load()) {
        if (launch_kernel(s) != DAWN_OK) {
            s->fatal = DAWN_E_CUDA;
            fail_all(s, s->fatal);
        }
        progress = true;
    }
    return progress;
}

void worker_main(dawn_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop.load()) {
        const bool progress = service(s);
        if (!progress) {
            s->cv.wait_for(lock, std::chrono::microseconds(20));
        }
        s->cv.notify_all();
    }
}

void server_release(dawn_server* s) {
    if (!s) return;
    for (auto& kv : s->reqs) {
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
        delete kv.second;
    }
    if (s->kstream) cudaStreamSynchronize(s->kstream);
    if (s->cstream) cudaStreamSynchronize(s->cstream);
    for (int g = 0; g < (int)s->graphs.size() && s->d_graphs; ++g) {
        SvGraph hg;
        if (cudaMemcpy(&hg, s->d_graphs + g, sizeof(SvGraph), cudaMemcpyDeviceToHost) == cudaSuccess) {
            cudaFree(hg.V[0]);
            cudaFree(hg.V[1]);
        }
    }
    if (s->d_graphs) cudaFree(s->d_graphs);
    if (s->d_ctl) cudaFree(s->d_ctl);
    if (s->arena) cudaFree(s->arena);
    if (s->hs) cudaFreeHost(s->hs);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    delete s;
}

}  // namespace
}  // namespace dawn

extern "C" {

DAWN_API int dawn_serve_create(const dawn_graph_t* graphs, int ngraphs, size_t mem_budget_bytes, int max_lanes,
                               dawn_server_t* out) {
    using namespace dawn;
    if (!out) return fail(DAWN_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs < 1 || ngraphs > kSvMaxGraphs)
        return fail(DAWN_E_INVALID, "ngraphs = %d: need 1..%d", ngraphs, kSvMaxGraphs);
    if (max_lanes != 64 && max_lanes != 128 && max_lanes != 256)
        return fail(DAWN_E_INVALID, "max_lanes = %d: need 64, 128 or 256", max_lanes);
    for (int i = 0; i < ngraphs; ++i)
        if (!graphs[i]) return fail(DAWN_E_INVALID, "graphs[%d] is NULL", i);
    dawn_server* s = new dawn_server();
    s->lanes = max_lanes;
    s->W = max_lanes / 64;
    s->graphs.assign(graphs, graphs + ngraphs);
    s->budget = mem_budget_bytes ? mem_budget_bytes : ((size_t)1 << 30);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->arena, s->budget);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_ctl, sizeof(SvCtl));
    if (e == cudaSuccess) e = cudaMemset(s->d_ctl, 0, sizeof(SvCtl));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->hs, sizeof(HostShared), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->hs_dev, s->hs, 0);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_graphs, sizeof(SvGraph) * ngraphs);
    if (e != cudaSuccess) {
        server_release(s);
        return cuda_fail(e, "dawn_serve_create", __FILE__, __LINE__);
    }
    std::memset(s->hs, 0, sizeof(HostShared));
    s->free_blocks[0] = s->budget;
    std::vector<SvGraph> hg((size_t)ngraphs);
    for (int i = 0; i < ngraphs; ++i) {
        std::memset(&hg[i], 0, sizeof(SvGraph));
        hg[i].in_ptr = graphs[i]->in_ptr;
        hg[i].in_idx = graphs[i]->in_idx;
        hg[i].excl = graphs[i]->excl;
        hg[i].n = graphs[i]->n;
        const size_t vb = sizeof(uint64_t) * (size_t)graphs[i]->n * s->W;
        if ((e = cudaMalloc((void**)&hg[i].V[0], vb)) != cudaSuccess ||
            (e = cudaMalloc((void**)&hg[i].V[1], vb)) != cudaSuccess ||
            (e = cudaMemset(hg[i].V[0], 0, vb)) != cudaSuccess || (e = cudaMemset(hg[i].V[1], 0, vb)) != cudaSuccess) {
            for (int j = 0; j <= i; ++j) { cudaFree(hg[j].V[0]); cudaFree(hg[j].V[1]); }
            cudaFree(s->d_graphs);
            s->d_graphs = nullptr;
            server_release(s);
            return cuda_fail(e, "dawn_serve_create (visited words)", __FILE__, __LINE__);
        }
        std::vector<int> fl;
        for (int l = max_lanes - 1; l >= 0; --l) fl.push_back(l);
        s->free_lanes.push_back(fl);
    }
    e = cudaMemcpy(s->d_graphs, hg.data(), sizeof(SvGraph) * ngraphs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        server_release(s);
        return cuda_fail(e, "dawn_serve_create", __FILE__, __LINE__);
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return DAWN_OK;
}

DAWN_API int dawn_serve_submit(dawn_server_t s, int graph_idx, const int32_t* sources, int32_t k, int dist_bytes,
                               void* dist_out, uint64_t* req_id) {
    using namespace dawn;
    if (!s) return fail(DAWN_E_INVALID, "server is NULL");
    if (graph_idx < 0 || graph_idx >= (int)s->graphs.size()) return fail(DAWN_E_INVALID, "graph_idx %d out of range", graph_idx);
    if (!sources || k < 1) return fail(DAWN_E_INVALID, "need k >= 1 sources");
    if (dist_bytes != 2 && dist_bytes != 4) return fail(DAWN_E_INVALID, "dist_bytes = %d: need 2 or 4", dist_bytes);
    if (!dist_out || !req_id) return fail(DAWN_E_INVALID, "dist_out / req_id is NULL");
    const int n = s->graphs[graph_idx]->n;
    Request* q = new Request();
    q->graph = graph_idx;
    q->sources.resize((size_t)k);
    cudaError_t e = cudaMemcpy(q->sources.data(), sources, sizeof(int32_t) * (size_t)k, cudaMemcpyDefault);
    if (e != cudaSuccess) { delete q; return cuda_fail(e, "dawn_serve_submit (sources)", __FILE__, __LINE__); }
    for (int i = 0; i < k; ++i)
        if (q->sources[i] < 0 || q->sources[i] >= n) {
            const int bad = q->sources[i];
            delete q;
            return fail(DAWN_E_INVALID, "sources[%d] = %d outside [0, %d)", i, bad, n);
        }
    q->dist_bytes = dist_bytes;
    q->dist_out = dist_out;
    q->out_dev = is_device_ptr(dist_out);
    q->block_bytes = (size_t)k * n * dist_bytes;
    if (q->out_dev) q->block = static_cast<char*>(dist_out);
    else if ((q->block_bytes + 255) / 256 * 256 > s->budget) {
        delete q;
        return fail(DAWN_E_NOMEM, "request block of %zu bytes can never fit the %zu-byte budget", (size_t)k * n * dist_bytes,
                    s->budget);
    }
    if ((e = cudaEventCreateWithFlags(&q->copied, cudaEventDisableTiming)) != cudaSuccess) {
        delete q;
        return cuda_fail(e, "dawn_serve_submit (event)", __FILE__, __LINE__);
    }
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->fatal != DAWN_OK) {
            cudaEventDestroy(q->copied);
            delete q;
            return fail(s->fatal, "the server stopped after a device failure");
        }
        q->id = s->next_id++;
        s->reqs[q->id] = q;
        s->queue.push_back(q->id);
        *req_id = q->id;
    }
    s->cv.notify_all();
    return DAWN_OK;
}

DAWN_API int dawn_serve_poll(dawn_server_t s, uint64_t req_id, int* state) {
    using namespace dawn;
    if (!s || !state) return fail(DAWN_E_INVALID, "server / state is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(DAWN_E_STATE, "unknown request id %llu", (unsigned long long)req_id);
    *state = it->second->state;
    if (it->second->state == DAWN_REQ_FAILED) return fail(it->second->err, "request %llu failed", (unsigned long long)req_id);
    return DAWN_OK;
}

DAWN_API int dawn_serve_times(dawn_server_t s, uint64_t req_id, double* submit_s, double* done_s) {
    using namespace dawn;
    if (!s) return fail(DAWN_E_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(DAWN_E_STATE, "unknown request id %llu", (unsigned long long)req_id);
    if (submit_s) *submit_s = it->second->t_submit;
    if (done_s) *done_s = it->second->t_done;
    return DAWN_OK;
}

DAWN_API int dawn_serve_drain(dawn_server_t s, int64_t timeout_ms) {
    using namespace dawn;
    if (!s) return fail(DAWN_E_INVALID, "server is NULL");
    const double t0 = now_s();
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        bool open = false;
        for (auto& kv : s->reqs) open |= kv.second->state == DAWN_REQ_PENDING || kv.second->state == DAWN_REQ_RUNNING;
        if (!open) return s->fatal == DAWN_OK ? DAWN_OK : fail(s->fatal, "the server stopped after a device failure");
        if (timeout_ms >= 0 && (now_s() - t0) * 1e3 > (double)timeout_ms)
            return fail(DAWN_E_TIMEOUT, "requests still open after %lld ms", (long long)timeout_ms);
        s->cv.wait_for(lock, std::chrono::microseconds(200));
    }
}

DAWN_API int dawn_serve_destroy(dawn_server_t s) {
    using namespace dawn;
    if (!s) return DAWN_OK;
    dawn_serve_drain(s, 60000);
    s->stop.store(true);
    s->hs->stop = 1;
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    server_release(s);
    return DAWN_OK;
}

}  // extern "C"
