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
// Graphs of low average degree (many levels, small frontiers) take the
// frontier step instead: the bit-lane push of Alg. 3 (Eq. 5-7) from only the
// (vertex, lane word) pairs that gained lanes in the previous iteration,
// along their CSR rows.  New lanes are set in one visited array in place by
// atomic OR, so each new (vertex, lane) is claimed by exactly one arc and
// gets the same level as in the pull; the arrivals form the next frontier.
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
constexpr int kSvPushCap = 4096;           // next-frontier keys staged per CTA round
constexpr int kSvPushWarpDeg = 32;         // longer rows are pushed by the whole warp
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

// Per graph, device memory.  Dense graphs keep two vertex-major visited arrays
// (V[0], V[1], ping-pong; W words per vertex).  Frontier graphs are stored
// word-major, one n-word array per lane word, indexed by the key w * n + v:
// the visited words VS (updated in place), per iteration parity the frontier
// words F[p] (lanes that reached (v, w) in the last iteration) and the list
// Q[p] of the keys whose frontier word is nonzero (each key once: its first
// writer appends it).
struct SvGraph {
    const int32_t* in_ptr;
    const int32_t* in_idx;
    const uint32_t* excl;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    uint64_t* V[2];
    uint64_t* VS;
    uint64_t* F[2];
    uint32_t* Q[2];
    int32_t n;
    int32_t frontier;
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
    unsigned long long lanes_over[3][kSvMaxGraphs][4];  // lanes whose next distance overflowed an int16 row
    // published by CTA 0 for iteration t into pub[t & 1]: {admitted entries,
    // exit flag, first entry of each graph (kSvMaxGraphs + 1 values)}
    int pub[2][32];
    // frontier graphs: keys appended to Q during iteration t are counted in
    // qn[(t + 1) % 3][g]; slot (t + 2) % 3 is cleared during iteration t
    int qn[3][kSvMaxGraphs];
    AdmitEntry admit[2][kSvMaxAdmit];     // sorted by (graph, src)
    long long seg_prefix[2][kSvMaxAdmit + 1];  // row-fill work items before each entry
    // the host mailbox {batch_seq, stop} as the last CTA read it during
    // iteration t, in mbox[t & 1] (CTA 0 decides with it one iteration later)
    alignas(128) unsigned mbox[2][32];
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
__device__ __forceinline__ unsigned sv_ld_relaxed_sys(const volatile unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
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

constexpr int kSvSnapMax = 2 + kSvMaxGraphs + 1;  // ints a barrier snapshot copies at most (per array)

// With `snap`, thread 0 copies nsnap ints (and nsnap2 from snap2) after the
// acquire into shared memory for the whole CTA (one L2 request per CTA, not
// one per warp).
__device__ bool sv_barrier(SvCtl* ctl, unsigned* count, unsigned& target, long long spin_limit,
                           const int* snap = nullptr, int nsnap = 0, int* s_snap = nullptr,
                           const int* snap2 = nullptr, int nsnap2 = 0, int* s_snap2 = nullptr) {
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
        if (ok) {
            // every load issued before the first store: one round trip, not one per word
            int v[kSvSnapMax], v2[kSvSnapMax];
#pragma unroll
            for (int i = 0; i < kSvSnapMax; ++i) {
                v[i] = i < nsnap ? sv_ld_relaxed_s32(snap + i) : 0;
                v2[i] = i < nsnap2 ? sv_ld_relaxed_s32(snap2 + i) : 0;
            }
#pragma unroll
            for (int i = 0; i < kSvSnapMax; ++i) {
                if (i < nsnap) s_snap[i] = v[i];
                if (i < nsnap2) s_snap2[i] = v2[i];
            }
        }
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

// One distance of a lane; false (nothing stored) when it does not fit the
// lane's int16 row, which retires the lane with an overflow report.
__device__ __forceinline__ bool sv_put(unsigned long long row, int bytes, long long v, int value) {
    if (bytes == 2) {
        if (value > 32767) return false;
        reinterpret_cast<int16_t*>(row)[v] = (int16_t)value;
    } else {
        reinterpret_cast<int32_t*>(row)[v] = value;
    }
    return true;
}

// Frontier push of lane word w along up to four arcs (u -> x[q]) of one row:
// f holds the lanes that reached u in the last iteration; Vw / Fw are the
// word-w visited words and next-parity frontier words.  The arcs' loads and
// atomics are issued together.  Lanes new at x are set in Vw[x] in place by
// atomic OR (so every new (x, lane) is claimed by exactly one arc), their
// distances stored, and OR-ed into Fw[x].  Bit q of the result: arc q made
// Fw[x[q]] nonzero, so its key joins the next list.  nm / om collect the
// lanes that grew / overflowed their rows.
template <int W>
__device__ __forceinline__ unsigned sv_push_arcs(uint64_t* Vw, uint64_t* Fw, const int32_t* __restrict__ ci, int j,
                                                 int cnt, int w, unsigned long long f, int t,
                                                 const unsigned long long* s_row, const int* s_bytes, const int* s_start,
                                                 unsigned long long (&nm)[W], unsigned long long (&om)[W], int (&x)[4]) {
    unsigned long long have[4], nb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = q < cnt ? __ldg(ci + j + q) : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) have[q] = q < cnt ? __ldcg(Vw + x[q]) : ~0ull;
    // The lanes of x not visited at the start of the iteration (have is read
    // after the last barrier, so it holds every earlier iteration's bits) are
    // new at this iteration, whichever thread sets them first: the visited and
    // frontier words take them together (the visited word's old value is not
    // needed, which spares a round trip), and a repeated claim of the same
    // lane by another thread writes the same distance.  The key is queued by
    // the claim that finds its frontier word empty.
#pragma unroll
    for (int q = 0; q < 4; ++q) nb[q] = f & ~have[q];
    unsigned app = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (nb[q]) {
            atomicOr(reinterpret_cast<unsigned long long*>(Vw + x[q]), nb[q]);
            if (atomicOr(reinterpret_cast<unsigned long long*>(Fw + x[q]), nb[q]) == 0ull) app |= 1u << q;
        }
    }
    unsigned long long grew = 0ull, over = 0ull;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned long long m = nb[q];
        grew |= m;
        while (m) {
            const int b = __ffsll((long long)m) - 1;
            m &= m - 1;
            const int s = w * 64 + b;
            if (!sv_put(s_row[s], s_bytes[s], x[q], t - s_start[s])) over |= 1ull << b;
        }
    }
#pragma unroll
    for (int q = 0; q < W; ++q)
        if (q == w) {
            nm[q] |= grew;
            om[q] |= over;
        }
    return app;
}

// Warp-wide append of the lanes' keys with app set: one shared-memory
// reservation per warp into the CTA's staging buffer; what does not fit goes
// straight to the list with one global reservation.
__device__ __forceinline__ void sv_append(bool app, uint32_t key, uint32_t* s_pbuf, int* s_pcount, uint32_t* Qn,
                                          int* qnext, int lane) {
    const unsigned b = __ballot_sync(kFull, app);
    if (!b) return;
    const int leader = __ffs(b) - 1;
    const int cnt = __popc(b);
    int slot0 = 0, gbase = 0;
    if (lane == leader) {
        slot0 = atomicAdd(s_pcount, cnt);
        const int spill = slot0 + cnt - max(kSvPushCap, slot0);
        if (spill > 0) gbase = atomicAdd(qnext, spill);
    }
    slot0 = __shfl_sync(kFull, slot0, leader);
    gbase = __shfl_sync(kFull, gbase, leader);
    if (app) {
        const int slot = slot0 + __popc(b & ((1u << lane) - 1u));
        if (slot < kSvPushCap) s_pbuf[slot] = key;
        else Qn[gbase + slot - max(kSvPushCap, slot0)] = key;
    }
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
    __shared__ int s_front[kSvMaxGraphs];    // 1: frontier graph
    __shared__ int s_qn[kSvMaxGraphs];       // frontier entries to expand this iteration
    __shared__ unsigned long long s_adm[kSvMaxGraphs][W];
    __shared__ uint32_t s_pbuf[kSvPushCap];  // next-frontier keys staged by this CTA
    __shared__ int s_pcount, s_pc, s_pbase;
    __shared__ unsigned long long s_overmask[4];
    __shared__ unsigned long long s_fin[kSvMaxGraphs * 4], s_ovr[kSvMaxGraphs * 4];
    __shared__ int s_recoff[kSvMaxGraphs * 4 + 1];
    __shared__ unsigned long long s_done_tail;  // CTA 0: completion records written so far

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
    if (threadIdx.x == 0) s_pcount = 0;
    if (threadIdx.x < 4) s_newmask[threadIdx.x] = 0;
    if (threadIdx.x < 4) s_overmask[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) s_done_tail = hs->done_tail;
    for (int g = threadIdx.x; g < kSvMaxGraphs; g += kSvThreads) s_front[g] = g < a.ngraphs ? a.graphs[g].frontier : 0;

    // iteration -1: CTA 0 picks up a batch that is already waiting
    if (blockIdx.x == 0) {
        __shared__ int s_take;
        if (threadIdx.x == 0) {
            seen_seq = sv_ld_acquire_sys(&hs->batch_ack);
            const unsigned seq = sv_ld_acquire_sys(&hs->batch_seq);
            s_take = seq != seen_seq ? (int)min(hs->count, (unsigned)kSvMaxAdmit) : -1;
            if (s_take >= 0) seen_seq = seq;
            for (int i = 0; i < 32; ++i) ctl->pub[0][i] = ctl->pub[1][i] = 0;
            ctl->mbox[1][0] = seen_seq;  // what iteration 0 decides with: nothing new yet
            ctl->mbox[1][1] = 0u;
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
        if (threadIdx.x < 3 * kSvMaxGraphs * 4) (&ctl->lanes_over[0][0][0])[threadIdx.x] = 0ull;
    }
    if (!sv_barrier(ctl, bar, bar_target, a.spin_limit, ctl->pub[0], 2 + kSvMaxGraphs + 1, s_pub, ctl->qn[0],
                    kSvMaxGraphs, s_qn))
        return;

    for (int t = 0;; ++t) {
        const int par = t & 1;
        const int na = s_pub[0];
        const long long* seg = ctl->seg_prefix[par];
        // The host mailbox is read over PCIe (~2 us, during which the reading
        // thread stalls) by the last CTA, which has the least work when the
        // frontiers are small; CTA 0 decides with what it read during the
        // iteration before (ordered by that iteration's barrier), so a batch or
        // a stop is taken one iteration later.  The load of that copy is
        // issued now and used at the end of the iteration.
        unsigned seq_early = 0u, stop_early = 0u;
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
            const unsigned sq = sv_ld_relaxed_sys(&hs->batch_seq);
            const unsigned sp = *(volatile unsigned*)&hs->stop;
            ctl->mbox[par][0] = sq;
            ctl->mbox[par][1] = sp;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            seq_early = __ldcg(&ctl->mbox[par ^ 1][0]);
            stop_early = __ldcg(&ctl->mbox[par ^ 1][1]);
        }
        // lanes admitted now, per graph
        if (na > 0) {
            for (int i = threadIdx.x; i < kSvMaxGraphs * W; i += kSvThreads) (&s_adm[0][0])[i] = 0ull;
            __syncthreads();
            for (int i = threadIdx.x; i < na; i += kSvThreads) {
                const AdmitEntry e = ld_entry(&ctl->admit[par][i]);
                atomicOr(&s_adm[e.graph][e.lane >> 6], 1ull << (e.lane & 63));
            }
            __syncthreads();
        }
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
        // ---- (1b) frontier graphs that receive lanes now: clear those lanes'
        //      visited bits left by earlier requests (dense graphs mask them
        //      on read instead), then one barrier before any push reads V
        {
            bool clear = false;
            for (int g = 0; g < a.ngraphs; ++g) clear |= s_front[g] && s_pub[2 + g + 1] > s_pub[2 + g];
            if (clear) {
                for (int g = 0; g < a.ngraphs; ++g) {
                    if (!s_front[g] || s_pub[2 + g + 1] == s_pub[2 + g]) continue;
                    const long long ng = a.graphs[g].n;
                    for (int w = 0; w < W; ++w) {
                        const unsigned long long m = s_adm[g][w];
                        if (!m) continue;
                        uint64_t* Vw = a.graphs[g].VS + w * ng;
                        for (long long v = gtid; v < ng; v += gthreads) {
                            const unsigned long long x = __ldcg(Vw + v);
                            if (x & m) Vw[v] = x & ~m;
                        }
                    }
                }
                if (!sv_barrier(ctl, bar, bar_target, a.spin_limit)) return;
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
            for (int w = 0; w < W; ++w) {
                adm[w] = nag > 0 ? s_adm[g][w] : 0ull;
                any |= occ[g][w] != 0ull;
            }
            const bool front = s_front[g] != 0;
            if (front ? (s_qn[g] == 0 && nag == 0) : (!any && nag == 0)) continue;
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
            for (int i = threadIdx.x; i < nag && !front; i += kSvThreads) {
                const AdmitEntry e = ld_entry(&ctl->admit[par][a0 + i]);
                s_asrc[i] = e.src;
                s_alane[i] = e.lane;
            }
            __syncthreads();
            if (front) {
                // ---- frontier graph: push the lanes that reached each listed
                //      (vertex, word) in the last iteration along its CSR row
                const int pq = t & 1;
                uint64_t* VS = G->VS;
                uint64_t* Fc = G->F[pq];
                uint64_t* Fn = G->F[pq ^ 1];
                const uint32_t* Qc = G->Q[pq];
                uint32_t* Qn = G->Q[pq ^ 1];
                const int32_t* rp = G->row_ptr;
                const int32_t* ci = G->col_idx;
                int* qnext = &ctl->qn[(t + 1) % 3][g];
                // sources of the lanes admitted now: visited, and in the next frontier
                for (long long i = gtid; i < nag; i += gthreads) {
                    const AdmitEntry e = ld_entry(&ctl->admit[par][a0 + i]);
                    const unsigned long long bit = 1ull << (e.lane & 63);
                    const long long key = (long long)(e.lane >> 6) * n + e.src;
                    atomicOr(reinterpret_cast<unsigned long long*>(VS + key), bit);
                    if (atomicOr(reinterpret_cast<unsigned long long*>(Fn + key), bit) == 0ull)
                        Qn[atomicAdd(qnext, 1)] = (uint32_t)key;
                }
                unsigned long long nm[W], om[W];
#pragma unroll
                for (int w = 0; w < W; ++w) nm[w] = om[w] = 0ull;
                const int nq = s_qn[g];
                // one listed key per thread and round (the loop bound is the
                // same for the whole CTA); appends are staged in shared memory
                for (long long base = (long long)blockIdx.x * kSvThreads; base < nq; base += gthreads) {
                    const long long i = base + threadIdx.x;
                    int w = 0;
                    unsigned long long f = 0ull;
                    int rb = 0, re = 0;
                    if (i < nq) {
                        const uint32_t key = __ldcg(Qc + i);
                        w = (int)(key / (uint32_t)n);
                        const int u = (int)(key - (uint32_t)w * (uint32_t)n);
                        f = __ldcg(Fc + key);
                        rb = __ldg(rp + u);
                        re = __ldg(rp + u + 1);
                        Fc[key] = 0ull;
                        f &= occ[g][w];  // lanes retired since: dropped
                        if (!f) re = rb;
                    }
                    uint64_t* Vw = VS + (long long)w * n;
                    uint64_t* Fw = Fn + (long long)w * n;
                    const bool wide = re - rb > kSvPushWarpDeg;
                    const int deg = wide ? 0 : re - rb;
                    const int dmax = (int)__reduce_max_sync(kFull, (unsigned)deg);
                    for (int d0 = 0; d0 < dmax; d0 += 4) {
                        int x[4] = {0, 0, 0, 0};
                        const int cnt = min(4, deg - d0);
                        const unsigned app = cnt > 0 ? sv_push_arcs<W>(Vw, Fw, ci, rb + d0, cnt, w, f, t, s_row,
                                                                       s_bytes, s_start, nm, om, x)
                                                     : 0u;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            sv_append((app >> q) & 1u, (uint32_t)w * (uint32_t)n + (uint32_t)x[q], s_pbuf, &s_pcount,
                                      Qn, qnext, lane);
                    }
                    unsigned wl = __ballot_sync(kFull, wide);
                    while (wl) {  // long rows: the whole warp, one arc per thread
                        const int sl = __ffs(wl) - 1;
                        wl &= wl - 1;
                        const int jb = __shfl_sync(kFull, rb, sl);
                        const int je = __shfl_sync(kFull, re, sl);
                        const unsigned long long fs = __shfl_sync(kFull, f, sl);
                        const int ws = __shfl_sync(kFull, w, sl);
                        uint64_t* Vws = VS + (long long)ws * n;
                        uint64_t* Fws = Fn + (long long)ws * n;
                        for (int j0 = jb; j0 < je; j0 += 32) {
                            int x[4] = {0, 0, 0, 0};
                            const int j = j0 + lane;
                            const unsigned app = j < je ? sv_push_arcs<W>(Vws, Fws, ci, j, 1, ws, fs, t, s_row, s_bytes,
                                                                          s_start, nm, om, x)
                                                        : 0u;
                            sv_append(app & 1u, (uint32_t)ws * (uint32_t)n + (uint32_t)x[0], s_pbuf, &s_pcount, Qn,
                                      qnext, lane);
                        }
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        const int c = min(s_pcount, kSvPushCap);
                        s_pcount = 0;
                        s_pc = c;
                        s_pbase = c > 0 ? atomicAdd(qnext, c) : 0;
                    }
                    __syncthreads();
                    for (int k = threadIdx.x; k < s_pc; k += kSvThreads) Qn[s_pbase + k] = s_pbuf[k];
                    __syncthreads();
                }
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const unsigned long long m = sv_warp_or64(nm[w]);
                    if (lane == 0 && m) atomicOr(&s_newmask[w], m);
                    const unsigned long long o = sv_warp_or64(om[w]);
                    if (lane == 0 && o) atomicOr(&s_overmask[w], o);
                }
            }
            for (int vb = front ? n : gw << 5; vb < n; vb += nw << 5) {
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
                        if (((nb >> bit) & 1ull) && !sv_put(s_row[s], s_bytes[s], v, t - s_start[s]))
                            atomicOr(&s_overmask[w], 1ull << bit);
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
                    if (((nbw[i >> 6] >> (i & 63)) & 1ull) && !sv_put(s_row[i], s_bytes[i], v, t - s_start[i]))
                        atomicOr(&s_overmask[i >> 6], 1ull << (i & 63));
            }
            __syncthreads();
            if (threadIdx.x == 0) s_hcount = 0;
            if (threadIdx.x < W) {
                if (s_newmask[threadIdx.x]) atomicOr(&ctl->lanes_new[t % 3][g][threadIdx.x], s_newmask[threadIdx.x]);
                if (s_overmask[threadIdx.x]) atomicOr(&ctl->lanes_over[t % 3][g][threadIdx.x], s_overmask[threadIdx.x]);
                s_newmask[threadIdx.x] = 0;
                s_overmask[threadIdx.x] = 0;
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
                s_take = 0;
                if (seq_early != seen_seq) {
                    // a new batch: read its sequence number here too, so that this
                    // thread's own read orders its reads of the batch
                    const unsigned seq = sv_ld_acquire_sys(&hs->batch_seq);
                    __threadfence_system();  // the batch was written before its sequence number
                    s_take = (int)min(hs->count, (unsigned)kSvMaxAdmit);
                    seen_seq = seq;
                }
            }
            if (threadIdx.x < kSvMaxGraphs * 4) (&ctl->lanes_new[(t + 1) % 3][0][0])[threadIdx.x] = 0ull;
            if (threadIdx.x < kSvMaxGraphs * 4) (&ctl->lanes_over[(t + 1) % 3][0][0])[threadIdx.x] = 0ull;
            if (threadIdx.x < kSvMaxGraphs) ctl->qn[(t + 2) % 3][threadIdx.x] = 0;
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
                ctl->pub[npar][1] = (stop_early != 0u) ||
                                    (!busy && (long long)(now - last_busy) > a.idle_ns);
            }
        }
        if (!sv_barrier(ctl, bar, bar_target, a.spin_limit, ctl->pub[par ^ 1], 2 + kSvMaxGraphs + 1, s_pub,
                        ctl->qn[(t + 1) % 3], kSvMaxGraphs, s_qn))
            return;
        // ---- (4) lanes whose level reached nothing, or whose distances no
        //      longer fit their int16 rows, are done: every CTA updates its
        //      occupancy the same way; CTA 0 reports them to the host
        if (threadIdx.x < a.ngraphs * W) {
            const int g = threadIdx.x / W, w = threadIdx.x % W;
            const unsigned long long o = occ[g][w];
            unsigned long long fin = 0ull, ovr = 0ull;
            if (o) {
                const unsigned long long got = sv_ld_relaxed_u64(&ctl->lanes_new[t % 3][g][w]);
                ovr = sv_ld_relaxed_u64(&ctl->lanes_over[t % 3][g][w]) & o;
                const unsigned long long started_now = na > 0 ? s_adm[g][w] : 0ull;  // not expanded yet
                fin = (o & ~got & ~started_now) | ovr;
            }
            s_fin[threadIdx.x] = fin;
            s_ovr[threadIdx.x] = ovr;
            occ[g][w] = o & ~fin;
        }
        __syncthreads();
        if (blockIdx.x == 0) {
            const int nwords = a.ngraphs * W;
            if (threadIdx.x == 0) {
                int acc = 0;
                for (int i = 0; i < nwords; ++i) {
                    s_recoff[i] = acc;
                    acc += __popcll(s_fin[i]);
                }
                s_recoff[nwords] = acc;
            }
            __syncthreads();
            if (s_recoff[nwords] > 0) {
                const unsigned long long tail = s_done_tail;
                for (int i = threadIdx.x; i < nwords * 64; i += kSvThreads) {
                    const int wi = i >> 6, b = i & 63;
                    const unsigned long long fw = s_fin[wi];
                    if (!((fw >> b) & 1ull)) continue;
                    const int g = wi / W, s = (wi % W) * 64 + b;
                    const SvGraph* G = &a.graphs[g];
                    const bool ov = (s_ovr[wi] >> b) & 1ull;
                    const unsigned long long r = tail + s_recoff[wi] + __popcll(fw & ((1ull << b) - 1ull));
                    volatile DoneRec* dst = &hs->done[r % kSvDoneRing];
                    dst->token = __ldcg(G->lane_token + s);
                    dst->levels = ov ? -1 : t - 1 - __ldcg(G->lane_start + s);
                    dst->status = ov ? DEV_OVERFLOW : DEV_OK;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence_system();  // records before the tail that publishes them
                    s_done_tail = tail + s_recoff[nwords];
                    hs->done_tail = s_done_tail;
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
    std::vector<dawn::SvGraph> host_graphs;  // device pointers of each graph's server state
    int fatal = DAWN_OK;
    int device = 0;
    // the idle fast path (see start_fast): a lone small request on an AUTO
    // low-degree graph runs on the single-source cluster engine
    std::vector<char> fast_ok;      // per graph
    cudaStream_t fstream = nullptr;
    cudaEvent_t fdone = nullptr;
    uint64_t fast_req = 0;          // the request running there (0: none)
    int32_t* fstage = nullptr;      // int32 rows when the request wants int16 rows
    size_t fstage_bytes = 0;
    int32_t* fsrc = nullptr;        // its sources on the device
    int* fovf_dev = nullptr;        // set when a distance does not fit int16
    int* fovf_host = nullptr;       // pinned copy
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

// Every row of request q is in its block: copy a staged block out to the
// host, or finish the request.  Called with s->mu held.
void rows_complete(dawn_server* s, Request* q) {
    if (!q->out_dev && q->err == DAWN_OK) {
        cudaMemcpyAsync(q->dist_out, q->block, q->block_bytes, cudaMemcpyDeviceToHost, s->cstream);
        cudaEventRecord(q->copied, s->cstream);
    } else {
        q->state = q->err == DAWN_OK ? DAWN_REQ_DONE : DAWN_REQ_FAILED;
        q->t_done = now_s();
        if (q->staged) { arena_free(s, q->arena_off, q->block_bytes); q->staged = false; }
    }
}

// int32 distance rows to int16 rows; *ovf = 1 when a distance does not fit
// (the request then fails with DAWN_E_OVERFLOW, as a lane of the loop does).
__global__ void fast_rows16_kernel(const int32_t* __restrict__ d, long long total, int16_t* out, int* ovf) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int v = d[i];
        if (v > 32767) *ovf = 1;
        out[i] = (int16_t)(v > 32767 ? 32767 : v);
    }
}

// The idle fast path.  A request of at most kFastMaxK sources on a graph
// served in AUTO mode, arriving while the server has nothing else queued or on
// the device, runs as single-source searches on a stream of its own instead of
// one bit lane each in the serving loop: on a low-degree graph (average
// out-degree below 8: lattices, road-like graphs) on thread-block clusters
// side by side (cluster_launch_many), else one launch per source with the
// single-source AUTO engine.  A lone search in the loop advances one level per
// loop iteration, several times slower than a cluster level or a grid level
// of the single-source kernel.  The distances are the same (every engine is
// exact).  Requests that arrive meanwhile queue for the loop, whose kernel
// starts when the fast path's kernels release their SMs.  Returns DAWN_OK
// when it started; otherwise the request stays in the queue (and a graph
// whose engine could not be launched leaves the fast path).
constexpr int kFastMaxK = 4;

int start_fast(dawn_server* s, Request* q) {
    dawn_graph* g = s->graphs[q->graph];
    const int k = (int)q->sources.size();
    const long long n = g->n;
    if (!q->block) {
        if (!arena_alloc(s, q->block_bytes, &q->arena_off)) return DAWN_E_NOMEM;
        q->block = s->arena + q->arena_off;
        q->staged = true;
    }
    int32_t* rows = reinterpret_cast<int32_t*>(q->block);
    if (q->dist_bytes == 2) {
        const size_t need = sizeof(int32_t) * (size_t)k * (size_t)n;
        if (need > s->fstage_bytes) {
            if (s->fstage) cudaFree(s->fstage);
            s->fstage = nullptr;
            s->fstage_bytes = 0;
            if (cudaMalloc((void**)&s->fstage, need) != cudaSuccess) return DAWN_E_NOMEM;
            s->fstage_bytes = need;
        }
        rows = s->fstage;
    }
    cudaError_t e = cudaMemcpyAsync(s->fsrc, q->sources.data(), sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice,
                                    s->fstream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->fovf_dev, 0, sizeof(int), s->fstream);
    if (e != cudaSuccess) return cuda_fail(e, "serving fast path", __FILE__, __LINE__);
    int rc = DAWN_OK;
    if (g->m < 8 * (int64_t)g->n && g->cl_size >= 0) {
        rc = cluster_launch_many(g, s->fsrc, k, rows, n, nullptr, nullptr, s->fstream);
    } else {
        for (int i = 0; i < k && rc == DAWN_OK; ++i)
            rc = sssp_launch(g, q->sources[(size_t)i], rows + (size_t)i * (size_t)n, nullptr, nullptr, s->fstream);
    }
    if (rc != DAWN_OK) {
        s->fast_ok[q->graph] = 0;
        if (q->staged) { arena_free(s, q->arena_off, q->block_bytes); q->staged = false; q->block = nullptr; }
        return rc;
    }
    if (q->dist_bytes == 2) {
        const long long total = (long long)k * n;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 4LL * s->sms);
        fast_rows16_kernel<<<blocks, 256, 0, s->fstream>>>(rows, total, reinterpret_cast<int16_t*>(q->block), s->fovf_dev);
    }
    cudaMemcpyAsync(s->fovf_host, s->fovf_dev, sizeof(int), cudaMemcpyDeviceToHost, s->fstream);
    cudaEventRecord(s->fdone, s->fstream);
    q->next = k;
    q->state = DAWN_REQ_RUNNING;
    s->fast_req = q->id;
    return DAWN_OK;
}

// The fast path's request once its stream reached fdone.
void finish_fast(dawn_server* s) {
    Request* q = s->reqs.count(s->fast_req) ? s->reqs[s->fast_req] : nullptr;
    const int rc = graph_sync_status(s->graphs[q ? q->graph : 0], s->fstream);
    s->fast_req = 0;
    if (!q) return;
    if (rc != DAWN_OK) q->err = rc;
    else if (*s->fovf_host) q->err = DAWN_E_OVERFLOW;
    q->rows_done = (int)q->sources.size();
    rows_complete(s, q);
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
        if (q->rows_done == (int)q->sources.size()) rows_complete(s, q);
    }
    s->hs->done_head = head;
    // ---- the idle fast path: its request, once its stream is through
    if (s->fast_req && cudaEventQuery(s->fdone) != cudaErrorNotReady) {
        finish_fast(s);
        progress = true;
    }
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
    // ---- the idle fast path: a lone small request on a low-degree AUTO graph
    //      while the loop has nothing queued, admitted or running
    if (!s->fast_req && !s->kernel_live && s->hs->batch_ack == s->batch_seq && s->queue.size() == 1) {
        Request* q = s->reqs[s->queue.front()];
        bool idle = true;
        for (size_t g = 0; g < s->graphs.size(); ++g) idle &= (int)s->free_lanes[g].size() == s->lanes;
        if (idle && q->state == DAWN_REQ_PENDING && q->next == 0 && s->fast_ok[q->graph] &&
            (int)q->sources.size() <= kFastMaxK && start_fast(s, q) == DAWN_OK) {
            s->queue.pop_front();
            progress = true;
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

void free_graph_state(SvGraph& hg) {
    for (int p = 0; p < 2; ++p) {
        cudaFree(hg.V[p]);
        cudaFree(hg.F[p]);
        cudaFree(hg.Q[p]);
        hg.V[p] = nullptr;
        hg.F[p] = nullptr;
        hg.Q[p] = nullptr;
    }
    cudaFree(hg.VS);
    hg.VS = nullptr;
}

void server_release(dawn_server* s) {
    if (!s) return;
    for (auto& kv : s->reqs) {
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
        delete kv.second;
    }
    if (s->kstream) cudaStreamSynchronize(s->kstream);
    if (s->cstream) cudaStreamSynchronize(s->cstream);
    if (s->fstream) cudaStreamSynchronize(s->fstream);
    if (s->fstage) cudaFree(s->fstage);
    if (s->fsrc) cudaFree(s->fsrc);
    if (s->fovf_dev) cudaFree(s->fovf_dev);
    if (s->fovf_host) cudaFreeHost(s->fovf_host);
    if (s->fdone) cudaEventDestroy(s->fdone);
    if (s->fstream) cudaStreamDestroy(s->fstream);
    for (auto& hg : s->host_graphs) free_graph_state(hg);
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

DAWN_API int dawn_serve_create_ex(const dawn_graph_t* graphs, int ngraphs, size_t mem_budget_bytes, int max_lanes,
                                  const int32_t* modes, dawn_server_t* out) {
    using namespace dawn;
    if (!out) return fail(DAWN_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs < 1 || ngraphs > kSvMaxGraphs)
        return fail(DAWN_E_INVALID, "ngraphs = %d: need 1..%d", ngraphs, kSvMaxGraphs);
    if (max_lanes != 64 && max_lanes != 128 && max_lanes != 256)
        return fail(DAWN_E_INVALID, "max_lanes = %d: need 64, 128 or 256", max_lanes);
    for (int i = 0; i < ngraphs; ++i) {
        if (!graphs[i]) return fail(DAWN_E_INVALID, "graphs[%d] is NULL", i);
        const int md = modes ? modes[i] : DAWN_SERVE_AUTO;
        if (md != DAWN_SERVE_AUTO && md != DAWN_SERVE_DENSE && md != DAWN_SERVE_FRONTIER)
            return fail(DAWN_E_INVALID, "modes[%d] = %d: need DAWN_SERVE_AUTO, _DENSE or _FRONTIER", i, md);
    }
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
    std::vector<SvGraph>& hg = s->host_graphs;
    hg.resize((size_t)ngraphs);
    for (int i = 0; i < ngraphs; ++i) {
        std::memset(&hg[i], 0, sizeof(SvGraph));
        const dawn_graph* gi = graphs[i];
        hg[i].in_ptr = gi->in_ptr;
        hg[i].in_idx = gi->in_idx;
        hg[i].excl = gi->excl;
        hg[i].row_ptr = gi->row_ptr;
        hg[i].col_idx = gi->col_idx;
        hg[i].n = gi->n;
        const int md = modes ? modes[i] : DAWN_SERVE_AUTO;
        // auto: low average degree (lattices, road-like graphs) means many
        // levels with small frontiers, where a full pass per level is waste
        hg[i].frontier = md == DAWN_SERVE_FRONTIER || (md == DAWN_SERVE_AUTO && gi->m < 8 * (int64_t)gi->n);
        if (hg[i].frontier && (int64_t)gi->n * s->W >= ((int64_t)1 << 32)) {
            if (md == DAWN_SERVE_FRONTIER) {
                server_release(s);
                return fail(DAWN_E_INVALID, "graphs[%d]: the frontier step needs n * max_lanes / 64 < 2^32", i);
            }
            hg[i].frontier = 0;
        }
        const size_t nk = (size_t)gi->n * s->W;
        const size_t vb = sizeof(uint64_t) * nk;
        if (hg[i].frontier) {
            e = cudaMalloc((void**)&hg[i].VS, vb);
            if (e == cudaSuccess) e = cudaMemset(hg[i].VS, 0, vb);
            for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
                e = cudaMalloc((void**)&hg[i].F[p], vb);
                if (e == cudaSuccess) e = cudaMemset(hg[i].F[p], 0, vb);
                if (e == cudaSuccess) e = cudaMalloc((void**)&hg[i].Q[p], sizeof(uint32_t) * nk);
            }
        } else {
            for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
                e = cudaMalloc((void**)&hg[i].V[p], vb);
                if (e == cudaSuccess) e = cudaMemset(hg[i].V[p], 0, vb);
            }
        }
        if (e != cudaSuccess) {
            server_release(s);
            return cuda_fail(e, "dawn_serve_create (per-graph state)", __FILE__, __LINE__);
        }
        std::vector<int> fl;
        for (int l = max_lanes - 1; l >= 0; --l) fl.push_back(l);
        s->free_lanes.push_back(fl);
        // the idle fast path: graphs served in AUTO mode
        s->fast_ok.push_back(md == DAWN_SERVE_AUTO ? 1 : 0);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->fstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->fsrc, sizeof(int32_t) * kFastMaxK);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->fovf_dev, sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->fovf_host, sizeof(int), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        server_release(s);
        return cuda_fail(e, "dawn_serve_create (fast path)", __FILE__, __LINE__);
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

DAWN_API int dawn_serve_create(const dawn_graph_t* graphs, int ngraphs, size_t mem_budget_bytes, int max_lanes,
                               dawn_server_t* out) {
    return dawn_serve_create_ex(graphs, ngraphs, mem_budget_bytes, max_lanes, nullptr, out);
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
