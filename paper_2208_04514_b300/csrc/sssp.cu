// Single-source DAWN on sm_103a: the whole level loop in one persistent
// cooperative kernel.
//
// One level ("step") of DAWN is the Boolean vector-matrix product of the
// frontier alpha with the adjacency over (OR, AND), masked by the vertices
// already reached; every newly reached vertex gets dist = step (Sec. 3.3,
// Eq. 5-7 and Alg. 3; Sec. 3.2, Eq. 2-4 and Alg. 1).  The kernel evaluates a
// level in one of two directions:
//
//  * push (SOVM, Alg. 3): the union of the CSR rows of the frontier
//    vertices (Eq. 7).  The frontier is a queue of row records
//    {first arc, arc count} with their offsets in the level's concatenated
//    arc list; the arcs are cut into equal ranges, one per warp, which walks
//    its range 32 arcs at a time, so every load of col_idx is a coalesced
//    run.  A target is claimed with atomicOr on the visited bitmap; the lane
//    whose atomicOr flipped the bit writes dist and appends the target's own
//    row to the next queue (one atomic per warp).
//  * pull (BOVM, Alg. 1): every vertex not yet reached evaluates the
//    compressed inner product of Eq. 4 over its in-neighbours and stops at
//    the first in-neighbour already reached.  The test reads the visited
//    bitmap as it was at the start of the step (the merge of alpha and beta
//    happens after the whole vertex loop), so a vertex found in this step
//    never certifies another one in the same step.  New bits go to a second
//    bitmap which becomes the current one after the grid barrier.  Testing
//    against all reached vertices rather than the frontier alone is exact:
//    an unreached v has d(v) >= step and a reached u has d(u) <= step - 1, so
//    an arc u -> v gives d(v) = step.
//
// The direction is chosen per level from device counters with Beamer's rule
// (push -> pull when m_f * alpha > m_u; pull -> push when n_f * beta < n and
// the frontier shrank).  Levels are separated by a grid barrier whose spin is
// bounded; on expiry the kernel records DEV_TIMEOUT and every CTA returns.
#include <climits>
#include <mutex>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

#ifndef DAWN_SSSP_MIN_CTAS
#define DAWN_SSSP_MIN_CTAS 1  // CTAs per SM the register budget is sized for
#endif
#ifndef DAWN_CTL_PREFETCH
#define DAWN_CTL_PREFETCH 1
#endif
#ifndef DAWN_LOOKAHEAD
#define DAWN_LOOKAHEAD 1  // list pulls look one level ahead for the stop at the component's size
#endif
#ifndef DAWN_LOOKAHEAD_DEEP
#define DAWN_LOOKAHEAD_DEEP 1  // and two levels ahead for vertices with short rows
#endif
#ifndef DAWN_SSSP_SMEM_BITMAP_MAX
#define DAWN_SSSP_SMEM_BITMAP_MAX (200 * 1024)
#endif
constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// Only the graph arrays, which no launch writes, are marked __restrict__ (and
// may take the read-only cache path).  The bitmaps and queues are rewritten
// by other CTAs from level to level inside one launch, and an SM's L1 may
// still hold a line of them from an earlier level, so every load of them is
// ld.global.cg (cached in L2 only, the point of coherence).
struct SsspArgs {
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col_idx;
    const int32_t* __restrict__ in_ptr;
    const int32_t* __restrict__ in_idx;
    const uint32_t* __restrict__ excl;
    uint32_t* vis0;
    uint32_t* vis1;
    int2* q0;
    int2* q1;
    int32_t* q0off;          // arc offset of each entry of q0 / q1
    int32_t* q1off;
    int32_t* dist;
    Ctl* ctl;
    dawn_sssp_stats* stats;  // device, may be null
    long long* trace;        // device, may be null: 4 int64 per grid barrier
    long long m;
    long long spin_limit;
    int32_t n;
    int32_t nwords;
    int32_t src;
    int32_t srb, sre;        // the source row [srb, sre) of col_idx; srb < 0: read from row_ptr
    long long reach_target;  // vertices reachable from src when known (symmetric graph: src's
                             // connected component), else past n: the loop stops on reaching them
    int32_t mode;
    int32_t alpha;
    int32_t beta;
    int32_t trace_cap;
    int32_t pull_serial;     // in-neighbours a lane tests alone in a pull level
    int32_t bar_parity;      // which of the two barrier counters this launch uses
    int32_t smem_words;      // > 0: pull levels copy the bitmap (this many words) to shared memory
    const int32_t* __restrict__ pull_idx;  // in-adjacency rows ordered by out-degree, largest first
    const int2* __restrict__ first2;       // the first two entries of each pull_idx row (-1 past its end)
    int32_t* cand0;          // per-CTA lists of unreached pull candidates (null: none)
    int32_t* cand1;
    long long cand_cap;      // entries per list
};

// A frontier queue: entries {first arc, arc count} and, in a parallel array,
// each entry's offset in the level's concatenated arc list.
struct Queue {
    int2* ent;
    int32_t* off;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One trace record {kind, step, count, time}; called by one thread.
__device__ __forceinline__ void trace_rec(const SsspArgs& a, int& slot, long long kind, long long step,
                                          long long count) {
    if (a.trace && slot < a.trace_cap) {
        long long* r = a.trace + 4 * (long long)slot;
        r[0] = kind;
        r[1] = step;
        r[2] = count;
        r[3] = (long long)globaltimer_ns();
    }
    ++slot;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier with a bounded spin.  Every CTA adds one to the launch's
// arrival counter with a release reduction and spins (acquire loads) until
// the counter reaches its own running target, gridDim.x more per barrier.
// Returns false (in every thread of the CTA) when the wait ran out or
// another CTA reported a failure.  `target` lives in thread 0.  With `snap`,
// thread 0 also reads that counter slot after the acquire and leaves
// {qpack, nf, mf, nc, lr} in s_snap for the whole CTA: one L2 request per CTA
// instead of one per warp on a single hot line (and likewise snap2 into
// s_snap2, read with it).
struct NoStep {
    __device__ void operator()() const {}
};

// after: run by thread 0 once the snapshot is taken, before the CTA is
// released (the level loop's bookkeeping, published through shared memory).
template <typename After = NoStep>
__device__ bool grid_barrier(Ctl* ctl, unsigned* count, unsigned& target, long long spin_limit,
                             const CtrSlot* snap = nullptr, unsigned long long* s_snap = nullptr,
                             After after = After(), const CtrSlot* snap2 = nullptr,
                             unsigned long long* s_snap2 = nullptr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        red_release_add(count, 1u);
        const long long t0 = clock64();
        unsigned polls = 0;
        while ((int)(ld_acquire(count) - target) < 0) {
            if (clock64() - t0 > spin_limit) {
                atomicCAS(&ctl->status, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
            if ((++polls & 15u) == 0 && ld_relaxed_s32(&ctl->status) != DEV_OK) { ok = 0; break; }
        }
        if (ok && snap) {
            s_snap[0] = ld_relaxed_u64(&snap->qpack);
            s_snap[1] = ld_relaxed_u64(&snap->nf);
            s_snap[2] = ld_relaxed_u64(&snap->mf);
            s_snap[3] = ld_relaxed_u64(&snap->nc);
            s_snap[4] = ld_relaxed_u64(&snap->lr);
            if (snap2) {  // a second level's slot (the fused levels 1 and 2)
                s_snap2[0] = ld_relaxed_u64(&snap2->qpack);
                s_snap2[1] = ld_relaxed_u64(&snap2->nf);
                s_snap2[2] = ld_relaxed_u64(&snap2->mf);
                s_snap2[3] = ld_relaxed_u64(&snap2->nc);
                s_snap2[4] = ld_relaxed_u64(&snap2->lr);
            }
            after();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int warp_inclusive_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Append the CSR row [rb, re) of each lane with `has` set to the queue as one
// record {first arc, arc count} (empty rows are left out), with the record's
// offset in the level's concatenated arc list.  One 64-bit atomic reserves
// the warp's records (high word) and arcs (low word) together, so offsets
// grow with the slot index.  The low word cannot carry into the high one: a
// level's arcs total at most m < 2^31.  A row of more than kEntryArcs arcs
// sets the level's long-row flag, which keeps the next push from splitting
// its work by record index.  Must be reached by the full warp.
__device__ __forceinline__ void warp_enqueue(bool has, int rb, int re, int lane, Queue q, CtrSlot* out) {
    const int deg = has ? re - rb : 0;
    const unsigned rows = __ballot_sync(kFull, deg > 0);
    if (!rows) return;
    const int dincl = warp_inclusive_scan(deg, lane);
    const int dtot = __shfl_sync(kFull, dincl, 31);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&out->qpack, ((unsigned long long)__popc(rows) << 32) | (unsigned)dtot);
    base = __shfl_sync(kFull, base, 0);
    if (__any_sync(kFull, deg > kEntryArcs) && lane == 0) atomicOr(&out->lr, 1ull);
    if (deg > 0) {
        const int pos = (int)(base >> 32) + __popc(rows & ((1u << lane) - 1u));
        q.ent[pos] = make_int2(rb, deg);
        q.off[pos] = (int)(base & 0xffffffffu) + dincl - deg;
    }
}

// Sum (nf, mf) over the CTA and add them to the level's counters (and the
// CTA's count of candidates left for the next pull, when given).
__device__ __forceinline__ void flush_counts(long long nf, long long mf, CtrSlot* out, const int* s_cn = nullptr) {
    __shared__ long long s_nf[kWarps], s_mf[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nf += __shfl_down_sync(kFull, nf, o);
        mf += __shfl_down_sync(kFull, mf, o);
    }
    if (lane == 0) { s_nf[w] = nf; s_mf[w] = mf; }
    __syncthreads();
    if (w == 0) {  // warp 0 sums the warps' partial counts
        long long a = lane < kWarps ? s_nf[lane] : 0, b = lane < kWarps ? s_mf[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(kFull, a, o);
            b += __shfl_down_sync(kFull, b, o);
        }
        if (lane == 0) {
            if (a) atomicAdd(&out->nf, (unsigned long long)a);
            if (b) atomicAdd(&out->mf, (unsigned long long)b);
            if (s_cn && *s_cn) atomicAdd(&out->nc, (unsigned long long)*s_cn);
        }
    }
}

// flush_counts for two levels at once (the fused levels 1 and 2).
__device__ __forceinline__ void flush_counts_two(long long nf1, long long mf1, CtrSlot* out1, long long nf2,
                                                 long long mf2, CtrSlot* out2) {
    __shared__ long long s_c[4][kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long v[4] = {nf1, mf1, nf2, mf2};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
        if (lane == 0) s_c[k][w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
        unsigned long long* dst[4] = {&out1->nf, &out1->mf, &out2->nf, &out2->mf};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            long long x = s_c[k][lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
            if (lane == 0 && x) atomicAdd(dst[k], (unsigned long long)x);
        }
    }
}

// Append v (lanes with `keep`) to this CTA's candidate list: one shared
// reservation per warp.  Must be reached by the full warp.
__device__ __forceinline__ void warp_keep(bool keep, int v, int lane, int32_t* list, int* s_cn) {
    const unsigned b = __ballot_sync(kFull, keep);
    if (!b) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(s_cn, __popc(b));
    base = __shfl_sync(kFull, base, 0);
    if (keep) list[base + __popc(b & ((1u << lane) - 1u))] = v;
}

// Vertices first reached by a level and the sum of their out-degrees (the
// values the out-of-line level functions return in registers).
struct LevelCount {
    long long nf, mf;
};

// Load the 32 queue entries starting at slot b (one per lane).
__device__ __forceinline__ void load_batch(const Queue& q, int qn, int b, int lane, int2& e, int& eoff) {
    const int i = b + lane;
    e = i < qn ? __ldcg(q.ent + i) : make_int2(0, 0);
    eoff = i < qn ? __ldcg(q.off + i) : INT_MAX;
}

// The rows left in every warp's buffer at the end of a push level, queued
// with one reservation for the whole CTA: the level's counter is a single
// address, and with one reservation per warp the last warps of a heavy
// level waited microseconds in line for it.  Reached by every warp of the
// CTA (nbuf = 0 for a warp without work).
__device__ __noinline__ void push_final_flush(const int2* buf, int nbuf, int lane, Queue q, CtrSlot* out) {
    __shared__ int s_fr[kWarps], s_fa[kWarps], s_fl[kWarps];
    const int warp = threadIdx.x >> 5;
    int arcs = 0;
    bool lng = false;
    for (int i = lane; i < nbuf; i += 32) {
        const int d = buf[i].y;
        arcs += d;
        lng |= d > kEntryArcs;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arcs += __shfl_xor_sync(kFull, arcs, o);
    lng = __any_sync(kFull, lng);
    if (lane == 0) {
        s_fr[warp] = nbuf;
        s_fa[warp] = arcs;
        s_fl[warp] = lng ? 1 : 0;
    }
    __syncthreads();
    if (warp == 0) {  // kWarps == 32: one lane per warp
        const int r = s_fr[lane], ar = s_fa[lane];
        const int ri = warp_inclusive_scan(r, lane), ai = warp_inclusive_scan(ar, lane);
        const int rows = __shfl_sync(kFull, ri, 31), tarcs = __shfl_sync(kFull, ai, 31);
        const bool anylng = __any_sync(kFull, s_fl[lane] != 0);
        unsigned long long base = 0;
        if (lane == 0 && rows > 0) base = atomicAdd(&out->qpack, ((unsigned long long)rows << 32) | (unsigned)tarcs);
        base = __shfl_sync(kFull, base, 0);
        if (lane == 0 && anylng) atomicOr(&out->lr, 1ull);
        s_fr[lane] = (int)(base >> 32) + ri - r;            // this warp's first slot
        s_fa[lane] = (int)(base & 0xffffffffu) + ai - ar;  // and the arc offset of its first row
    }
    __syncthreads();
    const int slot0 = s_fr[warp];
    int carry = s_fa[warp];
    for (int i0 = 0; i0 < nbuf; i0 += 32) {
        const int i = i0 + lane;
        const int2 e = i < nbuf ? buf[i] : make_int2(0, 0);
        const int incl = warp_inclusive_scan(e.y, lane);
        if (i < nbuf) {
            q.ent[slot0 + i] = e;
            q.off[slot0 + i] = carry + incl - e.y;
        }
        carry += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();
}

// Windows of 32 arcs a push takes per group (see push_level).
constexpr int kPushGroup = 4;

// The rows a push level claims gather in a per-warp buffer in the kernel's
// dynamic shared memory (the pull levels' bitmap copy, idle during a push)
// and are reserved in the queue in batches: one atomic on the level's
// counter per batch of >= kPushFlush rows instead of one per group of
// windows, since every warp's reservations meet on that one counter.
extern __shared__ uint4 s_bitmap4[];  // the kernel's dynamic shared memory
constexpr int kPushBuf = 192;                          // rows a warp's buffer holds
constexpr int kPushFlush = kPushBuf - 32 * kPushGroup;  // a group adds at most 32 * kPushGroup
constexpr int kPushBufBytes = kWarps * kPushBuf * (int)sizeof(int2);

// Append the lanes' claimed non-empty rows {first arc, arc count} to the
// warp's buffer (nbuf rows, warp-uniform).  Full warp.
__device__ __forceinline__ void warp_buffer_group(unsigned has, const int* rb, const int* re, int lane, int2* buf,
                                                  int& nbuf) {
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < kPushGroup; ++i) cnt += ((has >> i) & 1u) && re[i] > rb[i];
    const int incl = warp_inclusive_scan(cnt, lane);
    int pos = nbuf + incl - cnt;
#pragma unroll
    for (int i = 0; i < kPushGroup; ++i) {
        if (((has >> i) & 1u) && re[i] > rb[i]) {
            buf[pos] = make_int2(rb[i], re[i] - rb[i]);
            ++pos;
        }
    }
    nbuf += __shfl_sync(kFull, incl, 31);
    __syncwarp();
}

// Reserve the warp's nbuf buffered rows in the queue (one atomic: records in
// the high word, arcs in the low word) and copy them with their arc offsets;
// a row of more than kEntryArcs arcs raises the level's long-row flag.
// Full warp.
__device__ __forceinline__ void warp_flush_rows(const int2* buf, int nbuf, int lane, Queue q, CtrSlot* out) {
    int arcs = 0;
    bool lng = false;
    for (int i = lane; i < nbuf; i += 32) {
        const int d = buf[i].y;
        arcs += d;
        lng |= d > kEntryArcs;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arcs += __shfl_xor_sync(kFull, arcs, o);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&out->qpack, ((unsigned long long)nbuf << 32) | (unsigned)arcs);
    base = __shfl_sync(kFull, base, 0);
    if (__any_sync(kFull, lng) && lane == 0) atomicOr(&out->lr, 1ull);
    const int slot0 = (int)(base >> 32);
    int carry = (int)(base & 0xffffffffu);
    for (int i0 = 0; i0 < nbuf; i0 += 32) {
        const int i = i0 + lane;
        const int2 e = i < nbuf ? buf[i] : make_int2(0, 0);
        const int incl = warp_inclusive_scan(e.y, lane);
        if (i < nbuf) {
            q.ent[slot0 + i] = e;
            q.off[slot0 + i] = carry + incl - e.y;
        }
        carry += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();
}

// SOVM push: expand the frontier's rows (Eq. 7: the new vector is the union
// of the CSR rows of the frontier).  The level's E arcs are cut into equal
// ranges, a multiple of 32 long, one per warp of the grid; a warp finds the
// record holding its first arc with a 32-ary search over the sorted record
// offsets, then walks its range in groups of kPushGroup windows of 32
// consecutive arcs.  Within a group the col_idx loads, the bitmap tests, the
// atomicOr claims and the row_ptr loads of all windows are issued back to back,
// so a warp waits for one chain of memory round trips per group, not per
// window.
//
// pretest: read each target's bitmap word before claiming it, to spare the
// atomics on targets already reached; off while few are reached (the read
// would only lengthen the chain of round trips).
__device__ void push_level(const SsspArgs& a, int step, uint32_t* vis, Queue qin, unsigned long long pack,
                           bool qlong, bool pretest, Queue qout, CtrSlot* out, long long& nf, long long& mf) {
    const int lane = threadIdx.x & 31;
    const int qn = (int)(pack >> 32);
    const long long E = (long long)(pack & 0xffffffffull);
    const long long nw = (long long)gridDim.x * kWarps;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    int2* buf = reinterpret_cast<int2*>(s_bitmap4) + (threadIdx.x >> 5) * kPushBuf;  // claimed rows
    int nbuf = 0;  // warp-uniform
    if (E == 0) return;
    // Light levels (rows of at most 8 arcs on average and none longer than
    // kEntryArcs, e.g. a lattice frontier): each warp takes whole records by
    // index, so its first record is known without a search, and claims
    // without a read-only pre-test.  Heavy levels (hub rows): equal arc
    // ranges found by a 32-ary search.
    const bool light = E <= 8LL * qn && !qlong;
    pretest = pretest && !light;
    long long a0, a1;
    int bstart;
    int2 e;
    int eoff;
    if (light) {
        const long long per = (qn + nw - 1) / nw;
        const long long s0 = gw * per;
        if (s0 >= qn) {
            push_final_flush(buf, 0, lane, qout, out);  // the CTA's reservation waits for every warp
            return;
        }
        const long long s1 = min((long long)qn, s0 + per);
        bstart = (int)s0;
        load_batch(qin, qn, bstart, lane, e, eoff);
        const int end_off = s1 < qn ? __ldcg(qin.off + s1) : (int)E;
        a0 = __shfl_sync(kFull, eoff, 0);
        a1 = end_off;
    } else {
        long long chunk = (E + nw - 1) / nw;
        chunk = (chunk + 31) & ~31LL;
        a0 = gw * chunk;
        if (a0 >= E) {
            push_final_flush(buf, 0, lane, qout, out);
            return;
        }
        a1 = min(E, a0 + chunk);
        // largest slot i with off[i] <= a0 (off[0] = 0, so one exists)
        int lo = 0, hi = qn;
        while (hi - lo > 32) {
            const int stp = (hi - lo + 31) >> 5;
            const int p = lo + lane * stp;
            const int v = p < hi ? __ldcg(qin.off + p) : INT_MAX;
            const unsigned b = __ballot_sync(kFull, (long long)v <= a0);
            const int k = 31 - __clz(b);
            lo += k * stp;
            hi = min(hi, lo + stp);
        }
        bstart = lo;
        load_batch(qin, qn, bstart, lane, e, eoff);
    }
    for (long long gb = a0; gb < a1; gb += 32 * kPushGroup) {
        int cidx[kPushGroup];
#pragma unroll
        for (int q = 0; q < kPushGroup; ++q) {
            const long long wb = gb + 32 * q;
            cidx[q] = -1;
            if (wb >= a1) continue;  // warp-uniform
            // keep the batch covering this window: if its last arc lies past
            // the batch's last entry, restart the batch at the entry holding wb
            const long long last = min(wb + 31, a1 - 1);
            const int off31 = __shfl_sync(kFull, eoff, 31);
            const int len31 = __shfl_sync(kFull, e.y, 31);
            if (bstart + 32 < qn && last >= (long long)off31 + len31) {
                int k;
                if (wb >= (long long)off31 + len31) k = 32;
                else k = 31 - __clz(__ballot_sync(kFull, (long long)eoff <= wb));
                bstart += k;
                load_batch(qin, qn, bstart, lane, e, eoff);
            }
            const long long t = wb + lane;
            int o = 0;
#pragma unroll
            for (int b = 16; b > 0; b >>= 1) {
                const int cand = o + b;
                const int pv = __shfl_sync(kFull, eoff, cand);
                if ((long long)pv <= t) o = cand;
            }
            const int ostart = __shfl_sync(kFull, e.x, o);
            const int ooff = __shfl_sync(kFull, eoff, o);
            if (t < a1) cidx[q] = ostart + (int)(t - ooff);
        }
        int c[kPushGroup];
#pragma unroll
        for (int q = 0; q < kPushGroup; ++q) c[q] = cidx[q] >= 0 ? __ldg(a.col_idx + cidx[q]) : -1;
        uint32_t wv[kPushGroup];
#pragma unroll
        for (int q = 0; q < kPushGroup; ++q) wv[q] = (c[q] >= 0 && pretest) ? __ldcg(vis + (c[q] >> 5)) : (c[q] >= 0 ? 0u : kFull);
        // targets that look unreached: claim them and fetch their rows together
        int rb[kPushGroup], re[kPushGroup];
        unsigned cand = 0;
#pragma unroll
        for (int q = 0; q < kPushGroup; ++q) {
            rb[q] = re[q] = 0;
            if (c[q] >= 0 && !((wv[q] >> (c[q] & 31)) & 1u)) {
                cand |= 1u << q;
                rb[q] = __ldg(a.row_ptr + c[q]);
                re[q] = __ldg(a.row_ptr + c[q] + 1);
            }
        }
        unsigned claimed = 0;
#pragma unroll
        for (int q = 0; q < kPushGroup; ++q) {
            if ((cand >> q) & 1u) {
                const uint32_t bit = 1u << (c[q] & 31);
                const uint32_t old = atomicOr(&vis[c[q] >> 5], bit);
                if (!(old & bit)) claimed |= 1u << q;
            }
        }
#pragma unroll
        for (int q = 0; q < kPushGroup; ++q) {
            if ((claimed >> q) & 1u) {
                a.dist[c[q]] = step;
                nf += 1;
                mf += re[q] - rb[q];
            }
        }
        warp_buffer_group(claimed, rb, re, lane, buf, nbuf);
        if (nbuf >= kPushFlush) {
            warp_flush_rows(buf, nbuf, lane, qout, out);
            nbuf = 0;
        }
    }
    push_final_flush(buf, nbuf, lane, qout, out);
}

// BOVM pull: every unreached vertex tests its in-neighbours against the
// step-start bitmap vcur, stopping at the first hit (Eq. 4); results go to
// vnext.  A lane first tests up to pull_serial in-neighbours of its own
// vertex; vertices with in-arcs left are then taken one at a time by the
// whole warp, 32 in-neighbours per round, so that one long row does not
// hold 31 idle lanes.

// kSmem: the CTA first copies the whole step-start bitmap into shared memory
// (it is read-only for the level), so every in-neighbour test is a shared
// memory load instead of an L2 round trip (s_bitmap4, the kernel's dynamic
// shared memory).

template <bool kSmem>
__device__ __forceinline__ uint32_t bm_word(const uint32_t* vcur, int w) {
    if (kSmem) return reinterpret_cast<const uint32_t*>(s_bitmap4)[w];
    return __ldcg(vcur + w);
}

// BOVM pull over the whole bitmap (Alg. 1 / Eq. 4).  With `keep` (this
// CTA's region of a candidate list) every candidate left unreached is
// appended to it, for list pulls at the following levels.
//
// A warp takes kPullChunk of its bitmap words at a time, in two passes.
// Pass 1: every candidate of the chunk tests its first two in-neighbours
// (the likeliest to be reached: rows are in descending degree order), all
// words' loads issued together and coalesced (first2 holds them densely);
// most found vertices are settled here.  Pass 2: the candidates still open,
// packed 32 to a round through a per-warp list in shared memory, test the rest
// of their rows: up to pull_serial in-neighbours each, in aligned 16-byte
// groups, then the rows left are packed end to end across the warp, 32
// in-arcs per round, so that one long row does not hold 31 idle lanes.
constexpr int kPullChunk = 4;
__shared__ int s_pull_open[kWarps][kPullChunk * 32];  // pass 2 work, per warp (both instantiations)

template <bool kSmem>
__device__ void pull_level(const SsspArgs& a, int step, const uint32_t* vcur, uint32_t* vnext,
                           long long& nf, long long& mf, int32_t* keep, int* s_cn) {
    const int lane = threadIdx.x & 31;
    const bool symmetric = a.in_ptr == a.row_ptr;
    const unsigned below = (1u << lane) - 1u;
    int* open = s_pull_open[threadIdx.x >> 5];
    // this CTA's words are a contiguous range; its warps take chunks of
    // kPullChunk words from a shared counter, so a warp whose chunks hold many
    // open candidates does not keep the others waiting for it
    __shared__ int s_chunk;
    const int R = (a.nwords + gridDim.x - 1) / gridDim.x;
    const int wbase = (int)min((long long)a.nwords, (long long)blockIdx.x * R);
    const int wend = min(a.nwords, wbase + R);
    // chunks of up to kPullChunk words, fewer when the range is short, so
    // that every warp of the CTA gets work
    const int kc = max(1, min(kPullChunk, R / kWarps));
    if (threadIdx.x == 0) s_chunk = 0;
    if (kSmem) {
        const uint4* src4 = reinterpret_cast<const uint4*>(vcur);
        for (int i = threadIdx.x; i < (a.smem_words >> 2); i += kThreads) s_bitmap4[i] = __ldcg(src4 + i);
    }
    __syncthreads();
    while (true) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&s_chunk, 1);
        c = __shfl_sync(kFull, c, 0);
        const int w0 = wbase + c * kc;
        if (w0 >= wend) break;  // warp-uniform
        const int wlim = min(wend, w0 + kc);  // this chunk's words: [w0, wlim)
        // ---- pass 1: the first two in-neighbours of every candidate
        uint32_t cur[kPullChunk];
        unsigned cmask = 0;  // bit k: this lane's vertex of word k is a candidate
#pragma unroll
        for (int k = 0; k < kPullChunk; ++k) {
            const int w = w0 + k;
            cur[k] = kFull;
            if (w < wlim) {
                cur[k] = bm_word<kSmem>(vcur, w);
                // candidates: not reached, and with at least one in-arc (excl
                // also covers the padding bits past n).  excl is kept out of
                // the visited set itself: a vertex without in-arcs may still
                // have out-arcs, and it must not look reached to them.
                const uint32_t skip = cur[k] | __ldg(a.excl + w);
                if (!((skip >> lane) & 1u)) cmask |= 1u << k;
            }
        }
        if (!__any_sync(kFull, cmask)) {  // nothing to test: carry the words over
#pragma unroll
            for (int k = 0; k < kPullChunk; ++k)
                if (lane == 0 && w0 + k < wlim) vnext[w0 + k] = cur[k];
            continue;
        }
        int2 f2[kPullChunk];
        int db[kPullChunk], de[kPullChunk];  // out-row bounds: m_f of the vertices found
#pragma unroll
        for (int k = 0; k < kPullChunk; ++k) {
            f2[k] = make_int2(-1, -1);
            db[k] = de[k] = 0;
            if ((cmask >> k) & 1u) {
                const int v = ((w0 + k) << 5) + lane;
                f2[k] = __ldg(a.first2 + v);
                db[k] = __ldg(a.row_ptr + v);
                de[k] = __ldg(a.row_ptr + v + 1);
            }
        }
        unsigned fmask = 0;
#pragma unroll
        for (int k = 0; k < kPullChunk; ++k) {
            uint32_t h = 0;
            if (f2[k].x >= 0) h |= (bm_word<kSmem>(vcur, f2[k].x >> 5) >> (f2[k].x & 31)) & 1u;
            if (f2[k].y >= 0) h |= (bm_word<kSmem>(vcur, f2[k].y >> 5) >> (f2[k].y & 31)) & 1u;
            if (h) fmask |= 1u << k;
        }
        int nopen = 0;  // warp-uniform
#pragma unroll
        for (int k = 0; k < kPullChunk; ++k) {
            const int w = w0 + k;
            if (w >= wlim) continue;  // warp-uniform
            const int v = (w << 5) + lane;
            const bool f = (fmask >> k) & 1u;
            const uint32_t newbits = __ballot_sync(kFull, f);
            if (f) {
                a.dist[v] = step;
                nf += 1;
                mf += de[k] - db[k];
            }
            // pass 2 may set more bits of w (atomicOr, in program order after this store)
            if (lane == 0) vnext[w] = cur[k] | newbits;
            const bool op = ((cmask & ~fmask) >> k) & 1u;
            const unsigned ob = __ballot_sync(kFull, op);
            if (op) open[nopen + __popc(ob & below)] = v;
            nopen += __popc(ob);
        }
        __syncwarp();
        // ---- pass 2: the rest of the open candidates' rows
        for (int b0 = 0; b0 < nopen; b0 += 32) {
            const bool has = b0 + lane < nopen;
            const int v = has ? open[b0 + lane] : 0;
            int ib = 0, ie = 0;
            if (has) {
                ib = __ldg(a.in_ptr + v);
                ie = __ldg(a.in_ptr + v + 1);
            }
            int j = min(ib + 2, ie);
            bool found = false;
            const int jl = min(ie, ib + a.pull_serial);
            while (!found && j < jl) {
                // the aligned group of 4 in-neighbours holding j, one 16-byte load
                const int g0 = j & ~3;
                const int4 q = __ldg(reinterpret_cast<const int4*>(a.pull_idx + g0));
                const int xs[4] = {q.x, q.y, q.z, q.w};
                uint32_t h = 0;
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    if (g0 + x >= j && g0 + x < jl) h |= (bm_word<kSmem>(vcur, xs[x] >> 5) >> (xs[x] & 31)) & 1u;
                found = h != 0;
                j = min(g0 + 4, jl);
            }
            // rows with in-arcs left: each round packs the unresolved rows of
            // the warp end to end, tests their next 32 in-arcs (one per lane)
            // and resolves every owner from one ballot; found rows drop out
            const bool left = __any_sync(kFull, has && !found && j < ie);
            while (left) {
                const int rem = (has && !found) ? ie - j : 0;
                const int incl = warp_inclusive_scan(rem, lane);
                const int total = __shfl_sync(kFull, incl, 31);
                if (total == 0) break;
                const int ex = incl - rem;
                int o = 0;
#pragma unroll
                for (int bb = 16; bb > 0; bb >>= 1) {
                    const int cidx = o + bb;
                    const int pv = __shfl_sync(kFull, ex, cidx);
                    if (pv <= lane) o = cidx;
                }
                const int oj = __shfl_sync(kFull, j, o);
                const int oex = __shfl_sync(kFull, ex, o);
                bool hh = false;
                if (lane < total) {
                    const int x = __ldg(a.pull_idx + oj + (lane - oex));
                    hh = (bm_word<kSmem>(vcur, x >> 5) >> (x & 31)) & 1u;
                }
                const unsigned hits = __ballot_sync(kFull, hh);
                if (rem > 0 && ex < 32) {
                    const int hi = min(32, ex + rem);
                    const unsigned seg = (hi >= 32 ? kFull : ((1u << hi) - 1u)) & ~((1u << ex) - 1u);
                    if (hits & seg) found = true;
                    j += hi - ex;
                }
            }
            if (found) {
                a.dist[v] = step;
                atomicOr(vnext + (v >> 5), 1u << (v & 31));
                nf += 1;
                mf += symmetric ? (ie - ib) : (__ldg(a.row_ptr + v + 1) - __ldg(a.row_ptr + v));
            }
            if (keep) warp_keep(has && !found, v, lane, keep, s_cn);
        }
        __syncwarp();  // the open list is refilled by the next chunk
    }
}

// The look-ahead's second hop: whether one of u's first two in-neighbours
// (h0 for u = f2.x, h1 for u = f2.y; -1 past a row's end) was reached before
// the level `step` (the same step-start test as the list pull's).
__device__ __forceinline__ bool two_hop_hit(const SsspArgs& a, int2 h0, int2 h1, int step) {
    const int ws[4] = {h0.x, h0.y, h1.x, h1.y};
    int dw[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) dw[x] = ws[x] >= 0 ? __ldcg(a.dist + ws[x]) : -1;
    bool hit = false;
#pragma unroll
    for (int x = 0; x < 4; ++x) hit |= dw[x] >= 0 && dw[x] < step;
    return hit;
}

// The look-ahead's third hop, for a vertex v whose in-degree and whose
// in-neighbours' in-degrees are at most two (so that h0 and h1 hold every
// in-neighbour w of each in-neighbour u of v): whether one of the first two
// in-neighbours x of some w (g[] = first2 of h0.x, h0.y, h1.x, h1.y) was
// reached before the level `step`.
__device__ __forceinline__ bool three_hop_hit(const SsspArgs& a, const int2 (&g)[4], int step) {
    int dx[8];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        dx[2 * x] = g[x].x >= 0 ? __ldcg(a.dist + g[x].x) : -1;
        dx[2 * x + 1] = g[x].y >= 0 ? __ldcg(a.dist + g[x].y) : -1;
    }
    bool hit = false;
#pragma unroll
    for (int x = 0; x < 8; ++x) hit |= dx[x] >= 0 && dx[x] < step;
    return hit;
}

// A vertex v the look-ahead placed at level step + 1 (lanes with `ahead`) or
// step + 2 (lanes with `ahead2`; the two exclude each other), called by the
// lanes that ran the test, possibly divergent: dist is written now, and the
// count and out-degrees go straight to the level's counter slot (step % 3,
// as the loop picks it) with one pair of atomics per warp: the count of
// both in nc's high word; in lr (a list pull queues nothing) the degrees in
// the low word and the count of step + 2 placements in the high word.
// indeg: v's in-degree (its out-degree on a symmetric graph).
__device__ __forceinline__ void look_ahead(const SsspArgs& a, bool ahead, bool ahead2, int v, int indeg, int lane,
                                           int step, bool symmetric) {
    const unsigned am = __activemask();
    const unsigned hb = __ballot_sync(am, ahead || ahead2);
    const unsigned hb2 = __ballot_sync(am, ahead2);
    if (!(ahead || ahead2)) return;
    a.dist[v] = ahead ? step + 1 : step + 2;
    const unsigned deg = (unsigned)(symmetric ? indeg : (__ldg(a.row_ptr + v + 1) - __ldg(a.row_ptr + v)));
    const unsigned dsum = __reduce_add_sync(hb, deg);  // < m < 2^31: row_ptr is int32
    if (lane == __ffs(hb) - 1) {
        CtrSlot* out = &a.ctl->ctr[a.bar_parity][step % 3];
        atomicAdd(&out->nc, (unsigned long long)__popc(hb) << 32);
        atomicAdd(&out->lr, ((unsigned long long)__popc(hb2) << 32) | dsum);
    }
}

// BOVM pull over this CTA's list of candidates (the vertices a pull left
// unreached), instead of the whole bitmap.  The step-start visited test reads
// the distances: 0 <= dist[u] < step exactly when u was reached before this
// level (vertices found now carry dist = step), so found vertices can be set
// in the visited bitmap in place.  Candidates still unreached move to `keep`.
// No push queue is written (a list pull is mostly followed by another one);
// a push after it expands the frontier straight from this level's list
// (list_push_level).
__device__ __noinline__ LevelCount list_pull_level(const SsspArgs& a, int step, uint32_t* vis, const int32_t* cand,
                                                  int ncand, int32_t* keep, int* s_cn) {
    const int lane = threadIdx.x & 31;
    // the look-ahead below serves the stop at the component's size (known on symmetric graphs)
    const bool look = DAWN_LOOKAHEAD && a.mode == DAWN_MODE_AUTO && a.reach_target <= a.n;
    long long nf = 0, mf = 0;
    const bool symmetric = a.in_ptr == a.row_ptr;
    // one candidate per thread and round; the loop bound is the same for the whole warp
    for (int base = threadIdx.x & ~31; base < ncand; base += kThreads) {
        const int i = base + lane;
        const bool has = i < ncand;
        const int v = has ? __ldcg(cand + i) : 0;
        int ib = 0, ie = 0;
        int2 f2 = make_int2(-1, -1);
        if (has) {
            ib = __ldg(a.in_ptr + v);
            ie = __ldg(a.in_ptr + v + 1);
            f2 = __ldg(a.first2 + v);  // in parallel with the row bounds
        }
        // the first two in-neighbours first (rows are in descending degree order)
        bool found = false;
        {
            const int d0 = f2.x >= 0 ? __ldcg(a.dist + f2.x) : -1;
            const int d1 = f2.y >= 0 ? __ldcg(a.dist + f2.y) : -1;
            found = (d0 >= 0 && d0 < step) || (d1 >= 0 && d1 < step);
        }
        int j = min(ib + 2, ie);
        const int jl = min(ie, ib + a.pull_serial);
        while (!found && j < jl) {
            // the aligned group of 4 in-neighbours holding j, one 16-byte load
            const int g0 = j & ~3;
            const int4 q = __ldg(reinterpret_cast<const int4*>(a.pull_idx + g0));
            const int uu[4] = {q.x, q.y, q.z, q.w};
            int du[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) du[x] = (g0 + x >= j && g0 + x < jl) ? __ldcg(a.dist + uu[x]) : -1;
#pragma unroll
            for (int x = 0; x < 4; ++x) found |= du[x] >= 0 && du[x] < step;
            j = min(g0 + 4, jl);
        }
        // rows with in-arcs left: packed 32 at a time across the warp, as in pull_level
        while (true) {
            const int rem = (has && !found) ? ie - j : 0;
            const int incl = warp_inclusive_scan(rem, lane);
            const int total = __shfl_sync(kFull, incl, 31);
            if (total == 0) break;
            const int ex = incl - rem;
            int o = 0;
#pragma unroll
            for (int bb = 16; bb > 0; bb >>= 1) {
                const int cidx = o + bb;
                const int pv = __shfl_sync(kFull, ex, cidx);
                if (pv <= lane) o = cidx;
            }
            const int oj = __shfl_sync(kFull, j, o);
            const int oex = __shfl_sync(kFull, ex, o);
            bool hh = false;
            if (lane < total) {
                const int x = __ldg(a.pull_idx + oj + (lane - oex));
                const int dx = __ldcg(a.dist + x);
                hh = dx >= 0 && dx < step;
            }
            const unsigned hits = __ballot_sync(kFull, hh);
            if (rem > 0 && ex < 32) {
                const int hi = min(32, ex + rem);
                const unsigned seg = (hi >= 32 ? kFull : ((1u << hi) - 1u)) & ~((1u << ex) - 1u);
                if (hits & seg) found = true;
                j += hi - ex;
            }
        }
        if (found) {
            a.dist[v] = step;
            atomicOr(vis + (v >> 5), 1u << (v & 31));
            nf += 1;
            mf += symmetric ? (ie - ib) : (__ldg(a.row_ptr + v + 1) - __ldg(a.row_ptr + v));
        } else if (look && has) {
            // Look one level ahead.  v has no in-neighbour reached before this
            // level, so d(v) >= step + 1, and each of its first two
            // in-neighbours u (its whole row when it has at most two in-arcs)
            // is unreached at step start too: an in-neighbour of u reached
            // before this level puts u at this level and v at the next one.
            // The two-hop test reads u's first two in-neighbours and their
            // distances (the same step-start test as above).  It feeds the
            // stop test only: when the vertices it shows are all that is
            // left of the source's component, the loop ends here and the next
            // level is not run.  Their dist is written now, and they stay in
            // the list and out of the bitmap, so that a next level, if it
            // runs, finds them again with the same value.
            const int2 h0 = f2.x >= 0 ? __ldg(a.first2 + f2.x) : make_int2(-1, -1);
            const int2 h1 = f2.y >= 0 ? __ldg(a.first2 + f2.y) : make_int2(-1, -1);
            // Two levels ahead, for short rows: when v has at most two in-arcs
            // and so has each of its in-neighbours u, the two-hop test reads
            // every in-neighbour w of every u; if none was reached before this
            // level, no u is found at it, so d(u) >= step + 1 for all of them
            // and d(v) >= step + 2.  A w with an in-neighbour x reached before
            // this level (x among w's first two) bounds d(w) <= step, so
            // d(v) <= step + 2: then v is placed at step + 2.  The first two
            // in-neighbours of the w are loaded beside their distances.
            bool deep = DAWN_LOOKAHEAD_DEEP && ie - ib <= 2;
            if (deep) {
                const int lu0 = f2.x >= 0 ? __ldg(a.in_ptr + f2.x + 1) - __ldg(a.in_ptr + f2.x) : 0;
                const int lu1 = f2.y >= 0 ? __ldg(a.in_ptr + f2.y + 1) - __ldg(a.in_ptr + f2.y) : 0;
                deep = lu0 <= 2 && lu1 <= 2;
            }
            int2 gw[4];
            {
                const int ws[4] = {h0.x, h0.y, h1.x, h1.y};
#pragma unroll
                for (int x = 0; x < 4; ++x) gw[x] = (deep && ws[x] >= 0) ? __ldg(a.first2 + ws[x]) : make_int2(-1, -1);
            }
            const bool hit = two_hop_hit(a, h0, h1, step);
            const bool hit2 = !hit && deep && three_hop_hit(a, gw, step);
            look_ahead(a, hit, hit2, v, ie - ib, lane, step, symmetric);
        }
        warp_keep(has && !found, v, lane, keep, s_cn);
    }
    return {nf, mf};
}

// SOVM push right after a list pull (Eq. 7), without a queue: the frontier
// is the entries of that pull's input list (this CTA's part) whose distance
// is the level just finished (step - 1).  Each warp packs the rows of its
// frontier vertices end to end and expands them 32 arcs per round; claims
// and the next queue are as in push_level.
__device__ __noinline__ LevelCount list_push_level(const SsspArgs& a, int step, uint32_t* vis, const int32_t* list,
                                                  int nlist, CtrSlot* out) {
    const int lane = threadIdx.x & 31;
    long long nf = 0, mf = 0;
    // the queue of the frontier this level finds: (step & 1) ? q1 : q0
    const Queue qout = (step & 1) ? Queue{a.q1, a.q1off} : Queue{a.q0, a.q0off};
    // one list entry per thread and round; the loop bound is the same for the whole warp
    for (int base = threadIdx.x & ~31; base < nlist; base += kThreads) {
        const int i = base + lane;
        const int v = i < nlist ? __ldcg(list + i) : -1;
        const bool fr = v >= 0 && __ldcg(a.dist + v) == step - 1;
        int j = 0, je = 0;
        if (fr) {
            j = __ldg(a.row_ptr + v);
            je = __ldg(a.row_ptr + v + 1);
        }
        while (__any_sync(kFull, j < je)) {
            const int rem = je - j;
            const int incl = warp_inclusive_scan(rem, lane);
            const int total = __shfl_sync(kFull, incl, 31);
            const int ex = incl - rem;
            int o = 0;
#pragma unroll
            for (int bb = 16; bb > 0; bb >>= 1) {
                const int cidx = o + bb;
                const int pv = __shfl_sync(kFull, ex, cidx);
                if (pv <= lane) o = cidx;
            }
            const int oj = __shfl_sync(kFull, j, o);
            const int oex = __shfl_sync(kFull, ex, o);
            bool claimed = false;
            int c = 0, rb = 0, re = 0;
            if (lane < total) {
                c = __ldg(a.col_idx + oj + (lane - oex));
                const uint32_t bit = 1u << (c & 31);
                if (!(__ldcg(vis + (c >> 5)) & bit)) claimed = !(atomicOr(vis + (c >> 5), bit) & bit);
            }
            if (claimed) {
                a.dist[c] = step;
                rb = __ldg(a.row_ptr + c);
                re = __ldg(a.row_ptr + c + 1);
                nf += 1;
                mf += re - rb;
            }
            warp_enqueue(claimed, rb, re, lane, qout, out);
            if (rem > 0 && ex < 32) j += min(32, ex + rem) - ex;
        }
    }
    return {nf, mf};
}

// After a pull level: queue the vertices it reached (bits of vnow not in vold).
__device__ void bitmap_to_queue(const SsspArgs& a, const uint32_t* vnow, const uint32_t* vold,
                                Queue qout, CtrSlot* out) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int nw = gridDim.x * kWarps;
    for (int base = gw << 5; base < a.nwords; base += nw << 5) {
        const int w = base + lane;
        uint32_t nb = w < a.nwords ? (__ldcg(vnow + w) & ~__ldcg(vold + w)) : 0u;
        int rounds = __popc(nb);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(kFull, rounds, o));
        for (int r = 0; r < rounds; ++r) {
            const bool has = nb != 0;
            int rb = 0, re = 0;
            if (has) {
                const int v = (w << 5) + (__ffs(nb) - 1);
                nb &= nb - 1;
                rb = __ldg(a.row_ptr + v);
                re = __ldg(a.row_ptr + v + 1);
            }
            warp_enqueue(has, rb, re, lane, qout, out);
        }
    }
}

// Largest arc total T of the source's out-neighbours' rows for which every
// CTA runs level 2 itself (fused_init_levels); 0 turns the fused level 2 off.
#ifndef DAWN_FUSE2_MAX_ARCS
#define DAWN_FUSE2_MAX_ARCS 16384
#endif
// Largest CTA vertex range (bitmap words) the fused level 2 keeps in shared memory.
constexpr int kFuse2Words = kWarps * kPullChunk * 32 - 2 * kThreads;
// Arcs of the level-1 rows a thread reads per round of the fused level 2.
#ifndef DAWN_FUSE2_UNROLL
#define DAWN_FUSE2_UNROLL 8
#endif
constexpr int kFuse2Unroll = DAWN_FUSE2_UNROLL;

// Init and the first levels together (see the kernel).  Every CTA clears a
// contiguous vertex range of its own, and meanwhile reads the whole source
// row (the level-1 vertices, one per thread) with each one's row bounds; the
// level-1 rows hold T arcs in all (a CTA-wide scan, the same in every CTA).
//
// T small (at most DAWN_FUSE2_MAX_ARCS, and the direction rule pushes level
// 2 anyway): every CTA runs level 2 for its own range as well.  A level-2
// vertex is a target of a level-1 row that is neither the source nor a
// level-1 vertex, which a CTA can decide for the vertices of its own range
// from the source row alone, so no grid barrier separates levels 1 and 2:
// the CTA claims its level-1 vertices in a shared-memory copy of its bitmap
// words, then reads all T arcs of the level-1 rows (the same lines in every
// CTA, from L2 after the first reader) and claims the targets in its range
// there too; the claim that sets a bit first reaches the vertex (dist = 2)
// and queues its row for level 3.  Returns 2.
//
// Otherwise: level 1 alone (the claims in the CTA's range, their rows queued
// for the level-2 push).  Returns 1.  Must be reached by the whole CTA.
__device__ __noinline__ int fused_init_levels(const SsspArgs& a, int srb, int sdeg, CtrSlot* out1, CtrSlot* out2) {
    __shared__ int s_wsum[kWarps];
    __shared__ int s_T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t src = a.src;
    const bool d16 = (((uintptr_t)a.dist) & 15u) == 0;
    // ranges of a multiple of 128 vertices: whole int4 groups and bitmap words
    const long long per = (((long long)a.n + gridDim.x - 1) / gridDim.x + 127) & ~127LL;
    const long long v0 = (long long)blockIdx.x * per;
    const long long v1 = min((long long)a.n, v0 + per);
    // this thread's arc of the source row, loaded while the range is cleared
    const int c = threadIdx.x < sdeg ? __ldg(a.col_idx + srb + threadIdx.x) : -1;
    if (v0 < v1) {
        if (d16) {
            int4* d4 = reinterpret_cast<int4*>(a.dist);
            const long long e4 = v1 >> 2;
            for (long long i = (v0 >> 2) + threadIdx.x; i < e4; i += kThreads) d4[i] = make_int4(-1, -1, -1, -1);
            for (long long i = (e4 << 2) + threadIdx.x; i < v1; i += kThreads) a.dist[i] = -1;
        } else {
            for (long long i = v0 + threadIdx.x; i < v1; i += kThreads) a.dist[i] = -1;
        }
        const long long w1 = min((long long)a.nwords, (v1 + 31) >> 5);
        for (long long w = (v0 >> 5) + threadIdx.x; w < w1; w += kThreads)
            a.vis0[w] = (w == (src >> 5)) ? (1u << (src & 31)) : 0u;
    }
    // the level-1 vertex's row bounds (the loads wait for c, not for the clearing)
    int rb = 0, re = 0;
    if (c >= 0) {
        rb = __ldg(a.row_ptr + c);
        re = __ldg(a.row_ptr + c + 1);
    }
    // exclusive scan of the level-1 row lengths over the CTA: arc offsets and T
    const int deg = re - rb;
    const int incl = warp_inclusive_scan(deg, lane);
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();  // also orders the clearing before the claims below
    if (warp == 0) {
        const int x = s_wsum[lane];
        const int xi = warp_inclusive_scan(x, lane);
        s_wsum[lane] = xi - x;
        if (lane == 31) s_T = xi;
    }
    __syncthreads();
    const int off = s_wsum[warp] + incl - deg;
    const int T = s_T;
    if (threadIdx.x == 0 && src >= v0 && src < v1) a.dist[src] = 0;
    // the direction rule pushes level 2 (T bounds the arcs of the level-1 rows)
    const bool push2 = a.mode == DAWN_MODE_PUSH || (long long)T * a.alpha <= a.m - sdeg - T;
    // (a CTA claims at most min(T, its range) vertices: the claim list's bound)
    const bool fuse2 = DAWN_FUSE2_MAX_ARCS > 0 && T >= 1 && T <= DAWN_FUSE2_MAX_ARCS && push2 &&
                       per <= 32LL * kFuse2Words && min((long long)T, per) <= kPushBufBytes / 4;
    if (!fuse2) {
        bool claimed = false;
        if (c >= v0 && c < v1 && c != src) {
            const uint32_t bit = 1u << (c & 31);
            claimed = !(atomicOr(&a.vis0[c >> 5], bit) & bit);
            if (claimed) a.dist[c] = 1;
        }
        warp_enqueue(claimed, rb, re, lane, Queue{a.q1, a.q1off}, out1);
        flush_counts(claimed ? 1 : 0, claimed ? re - rb : 0, out1);
        return 1;
    }
    // ---- levels 1 and 2 in this CTA's range.  Shared memory: the level-1
    // rows' arc offsets and first arcs, and the CTA's bitmap words (the
    // pull's per-warp lists, idle until the first pull); the push's per-warp
    // row buffers (the dynamic shared memory, idle until the first push).
    int* s_off = &s_pull_open[0][0];
    int* s_rb = s_off + kThreads;
    uint32_t* s_vis = reinterpret_cast<uint32_t*>(s_rb + kThreads);
    const long long wr0 = v0 >> 5;
    const int nwr = (int)((v1 - v0 + 31) >> 5);  // v0 is a multiple of 128
    for (int i = threadIdx.x; i < nwr; i += kThreads)
        s_vis[i] = (wr0 + i == (src >> 5)) ? (1u << (src & 31)) : 0u;
    s_off[threadIdx.x] = off;
    s_rb[threadIdx.x] = rb;
    __syncthreads();
    long long nf1 = 0, mf1 = 0;
    if (c >= v0 && c < v1) {
        const uint32_t bit = 1u << (c & 31);
        if (!(atomicOr(&s_vis[(c - v0) >> 5], bit) & bit)) {
            a.dist[c] = 1;
            nf1 = 1;
            mf1 = deg;
        }
    }
    __syncthreads();  // every level-1 vertex of the range is marked before level 2 tests it
    // level 2, first pass: every arc of the level-1 rows, kFuse2Unroll per
    // thread with their col_idx loads in flight together; the targets claimed
    // in this CTA's range go to a list (in the push's row buffers, idle until
    // the first push: at most T entries)
    __shared__ int s_nclaim;
    int* claims = reinterpret_cast<int*>(s_bitmap4);
    if (threadIdx.x == 0) s_nclaim = 0;
    for (int base = 0; base < T; base += kThreads * kFuse2Unroll) {  // CTA-uniform
        int t[kFuse2Unroll];
#pragma unroll
        for (int q = 0; q < kFuse2Unroll; ++q) {
            const int e = base + q * kThreads + threadIdx.x;
            t[q] = -1;
            if (e < T) {
                // the level-1 row holding arc e: the last entry whose offset is <= e
                int lo = 0, hi = sdeg;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_off[mid] <= e) lo = mid;
                    else hi = mid;
                }
                t[q] = s_rb[lo] + (e - s_off[lo]);
            }
        }
#pragma unroll
        for (int q = 0; q < kFuse2Unroll; ++q) t[q] = t[q] >= 0 ? __ldg(a.col_idx + t[q]) : -1;
#pragma unroll
        for (int q = 0; q < kFuse2Unroll; ++q) {
            if (t[q] >= v0 && t[q] < v1) {
                const uint32_t bit = 1u << (t[q] & 31);
                if (!(atomicOr(&s_vis[(t[q] - v0) >> 5], bit) & bit)) {
                    a.dist[t[q]] = 2;
                    claims[atomicAdd(&s_nclaim, 1)] = t[q];
                }
            }
        }
    }
    __syncthreads();
    // second pass: the claimed vertices' rows, queued for level 3
    long long nf2 = 0, mf2 = 0;
    const int ncl = s_nclaim;
    const Queue q2{a.q0, a.q0off};  // the frontier found at level 2 lives in queue 0
    for (int b = threadIdx.x & ~31; b < ncl; b += kThreads) {  // bound uniform over the warp
        const int i = b + lane;
        int rb2 = 0, re2 = 0;
        if (i < ncl) {
            const int t = claims[i];
            rb2 = __ldg(a.row_ptr + t);
            re2 = __ldg(a.row_ptr + t + 1);
            nf2 += 1;
            mf2 += re2 - rb2;
        }
        warp_enqueue(i < ncl, rb2, re2, lane, q2, out2);
    }
    __syncthreads();
    // the CTA's bitmap words with both levels' claims (the clearing above wrote zeros)
    for (int i = threadIdx.x; i < nwr; i += kThreads) a.vis0[wr0 + i] = s_vis[i];
    flush_counts_two(nf1, mf1, out1, nf2, mf2, out2);
    return 2;
}

// level kinds: push (SOVM), pull over the bitmap, pull over the candidate lists
enum LevelKind { kPush = 0, kBitmapPull = 1, kListPull = 2, kStop = 3 };
// how a push gets its frontier: the queue, a conversion of the bitmap
// difference a bitmap pull left (then a barrier), or a list pull's list
enum PushFrom { kFromQueue = 0, kFromBitmap = 1, kFromList = 2 };

// The level loop's bookkeeping, kept by thread 0 of each CTA in shared memory
// and advanced inside the grid barrier that ends a level, so the other threads
// hold only the level's kind in registers.
struct LoopState {
    long long mu;       // arcs out of vertices not yet reached
    long long prev_nf;  // vertices found by the level before the last one
    long long reached, edges;
    int pushes, pulls;
    int last;           // kind of the last level run
    int kind, from;     // the next level (kStop: the loop is over)
    int levels;         // when stopped: the last level that reached a vertex
};

// The parameters of the direction rule (copied out of the launch arguments, so
// that the barrier's callback captures a few scalars, not the whole struct).
struct RuleArgs {
    long long reach_target;
    int32_t n, mode, alpha, beta;
    bool lists;
};

// Thread 0, once the level `step` is over and its counters are in snap: add
// them up and choose the next level (Beamer's rule, list pulls while the
// candidates are few), or stop.
__device__ __forceinline__ void next_level(const RuleArgs& a, LoopState& L, const unsigned long long* snap, int step) {
    const bool lists = a.lists;
    const long long nf_cur = (long long)snap[1];
    const long long mf_cur = (long long)snap[2];
    const long long nc_cur = (long long)(snap[3] & 0xffffffffull);  // unreached candidates, after a pull (the
                                                                     // high word counts a list pull's look-ahead)
    if (nf_cur == 0 || step >= a.n) {
        L.kind = kStop;
        L.levels = step > 0 ? step - 1 : 0;
        return;
    }
    L.reached += nf_cur;
    L.edges += mf_cur;
    L.mu -= mf_cur;
    // every vertex src can reach has its distance: no level can find more
    // (the empty level that would show it is skipped)
    if (L.reached >= a.reach_target) {
        L.kind = kStop;
        L.levels = step;
        return;
    }
    int kind;
    if (a.mode == DAWN_MODE_PUSH) kind = kPush;
    else if (a.mode == DAWN_MODE_PULL)
        kind = (L.last != kPush && lists && nc_cur <= 4 * mf_cur && 4 * nc_cur <= a.n) ? kListPull : kBitmapPull;
    else if (L.last == kPush) kind = mf_cur * a.alpha > L.mu ? kBitmapPull : kPush;
    // after a pull: test only the candidates left while they are few (next to
    // the frontier's arcs, and at most a quarter of the vertices: a larger
    // list is cheaper as a bitmap pull with its tests in shared memory);
    // otherwise the push / pull rule
    else if (lists && nc_cur <= 4 * mf_cur && 4 * nc_cur <= a.n) kind = kListPull;
    else kind = (nf_cur * a.beta < a.n && nf_cur < L.prev_nf) ? kPush : kBitmapPull;
    L.from = kind != kPush ? kFromQueue : (L.last == kBitmapPull ? kFromBitmap : (L.last == kListPull ? kFromList : kFromQueue));
    L.prev_nf = nf_cur;
    L.kind = kind;
    L.last = kind;
    if (kind == kPush) ++L.pushes;
    else ++L.pulls;
}

__global__ void __launch_bounds__(kThreads, DAWN_SSSP_MIN_CTAS) sssp_kernel(SsspArgs a) {
    Ctl* ctl = a.ctl;
    __shared__ unsigned long long s_snap[5];  // {qpack, nf, mf, nc, lr} of the level just finished
    __shared__ int s_cn, s_cin, s_cprev;      // this CTA's candidates: being kept / to test / tested last
    __shared__ LoopState L;
    __shared__ int s_status;
    // an earlier call that failed leaves the barrier state inconsistent: this
    // launch then stops before its first barrier (its outputs are undefined,
    // and the host clears the control block when it reports the failure).
    // The status load overlaps the clearing below.
    if (threadIdx.x == 0) s_status = ld_relaxed_s32(&ctl->status);
    const int lane = threadIdx.x & 31;
    // the per-level trace: thread 0 of CTA 0, its record count kept in shared
    // memory (not a register carried through the level loop)
    const bool tracer = a.trace && blockIdx.x == 0 && threadIdx.x == 0;
    __shared__ int s_tslot;
    int& tslot = s_tslot;
    if (tracer) tslot = 0;
    unsigned* bar = &ctl->bar[a.bar_parity].count;
    unsigned bar_target = 0;
    if (tracer) trace_rec(a, tslot, 0, 0, 1);
#if DAWN_CTL_PREFETCH
    // The control block's lines (this launch's barrier counter and counter
    // slots) and the statistics record are touched first by the level-1
    // atomics, the first grid barrier and the last write; the L2 may have
    // lost them since the last launch, so bring them in now, off the chain.
    if (blockIdx.x == 0 && threadIdx.x < 6) {
        const void* p = threadIdx.x == 0 ? (const void*)&ctl->bar[a.bar_parity]
                      : threadIdx.x <= 3 ? (const void*)&ctl->ctr[a.bar_parity][threadIdx.x - 1]
                      : threadIdx.x == 4 ? (const void*)&ctl->status
                                         : (const void*)a.stats;
        if (p) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
#endif
    const long long gtid = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * kThreads;

    // candidate lists: this CTA's region is the vertices of the bitmap words its warps scan
    const int nwarps = gridDim.x * kWarps;
    const long long region = (long long)kWarps * ((a.nwords + nwarps - 1) / nwarps) * 32;
    const bool lists = a.cand0 != nullptr && region * gridDim.x <= a.cand_cap;
    // this launch's counter slots (zero on entry); zero the next launch's
    CtrSlot* ctr = ctl->ctr[a.bar_parity];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x < 3 * (int)(sizeof(CtrSlot) / 8))
        reinterpret_cast<unsigned long long*>(ctl->ctr[a.bar_parity ^ 1])[threadIdx.x] = 0;

    // ---- init: dist = -1 except dist[src] = 0; visited = {src}
    const int32_t src = a.src;
    const int srb = a.srb >= 0 ? a.srb : __ldg(a.row_ptr + src);
    const int sre = a.srb >= 0 ? a.sre : __ldg(a.row_ptr + src + 1);
    const int sdeg = sre - srb;
    // Level 1 (the push of the source row) joins the init when the rule would
    // push and the row fits one pass of the CTA: each CTA clears a contiguous
    // vertex range of its own and then claims the source's out-neighbours in
    // that range, so only __syncthreads orders the clearing before the claims
    // and the first grid barrier already ends level 1.  When the level-1 rows
    // are short, level 2 joins it too (fused_init_levels): the first grid
    // barrier then ends level 2.
    const bool fused = a.mode != DAWN_MODE_PULL && sdeg <= kThreads &&
                       (a.mode == DAWN_MODE_PUSH || (long long)sdeg * a.alpha <= a.m - sdeg);
    // the loop starts after level 0 (the source), or after level 1 (or 2) when fused
    int step = fused ? 1 : 0;
    if (threadIdx.x == 0) {
        L.mu = a.m - (fused ? sdeg : 0);
        L.prev_nf = fused ? 1 : 0;
        L.reached = fused ? 1 : 0;
        L.edges = fused ? sdeg : 0;
        L.pushes = fused ? 1 : 0;
        L.pulls = 0;
        L.last = kPush;
        L.kind = kStop;
        L.from = kFromQueue;
        L.levels = 0;
        s_cn = s_cin = s_cprev = 0;
    }
    const RuleArgs ra = {a.reach_target, a.n, a.mode, a.alpha, a.beta, lists};
    unsigned long long* const snap = s_snap;
    LoopState* const lp = &L;
    auto advance = [ra, snap, lp](int done_step) { next_level(ra, *lp, snap, done_step); };
    const bool d16 = (((uintptr_t)a.dist) & 15u) == 0;
    if (fused) {
        const int levels = fused_init_levels(a, srb, sdeg, &ctr[1], &ctr[2]);  // ends with __syncthreads
        if (s_status != DEV_OK) return;
        if (levels == 2) {
            // level 1's counts come with level 2's: the rule runs for both
            __shared__ unsigned long long s_snap1[5];
            unsigned long long* const snap1 = s_snap1;
            if (!grid_barrier(ctl, bar, bar_target, a.spin_limit, &ctr[2], s_snap, [ra, snap, snap1, lp]() {
                    next_level(ra, *lp, snap1, 1);
                    if (lp->kind != kStop) next_level(ra, *lp, snap, 2);
                }, &ctr[1], s_snap1))
                return;
            step = 2;
            if (tracer) {
                trace_rec(a, tslot, 1, 0, 1);
                trace_rec(a, tslot, 2, 1, (long long)s_snap1[1]);
                trace_rec(a, tslot, 2, 2, (long long)s_snap[1]);
            }
        } else {
            if (!grid_barrier(ctl, bar, bar_target, a.spin_limit, &ctr[1], s_snap, [advance]() { advance(1); })) return;
            if (tracer) {
                trace_rec(a, tslot, 1, 0, 1);
                trace_rec(a, tslot, 2, 1, (long long)s_snap[1]);
            }
        }
        if (gtid == 0) ctl->bar[a.bar_parity ^ 1].count = 0;  // the next launch's counter
    } else {
        if (d16) {
            int4* d4 = reinterpret_cast<int4*>(a.dist);
            const long long n4 = a.n >> 2;
            for (long long i = gtid; i < n4; i += gthreads) d4[i] = make_int4(-1, -1, -1, -1);
            for (long long i = (n4 << 2) + gtid; i < a.n; i += gthreads) a.dist[i] = -1;
        } else {
            for (long long i = gtid; i < a.n; i += gthreads) a.dist[i] = -1;
        }
        for (long long w = gtid; w < a.nwords; w += gthreads)
            a.vis0[w] = (w == (src >> 5)) ? (1u << (src & 31)) : 0u;
        if (blockIdx.x == 0 && threadIdx.x < 32) {  // level 0: the source, queue = {src}
            warp_enqueue(lane == 0, srb, sre, lane, Queue{a.q0, a.q0off}, &ctr[0]);
            if (lane == 0) {
                ctr[0].nf = 1;
                ctr[0].mf = (unsigned long long)sdeg;
            }
        }
        __syncthreads();
        if (s_status != DEV_OK) return;
        // dist[src] = 0 after the fill; the barrier orders it after every -1 store
        if (!grid_barrier(ctl, bar, bar_target, a.spin_limit, &ctr[0], s_snap, [advance]() { advance(0); })) return;
        if (gtid == 0) {
            a.dist[src] = 0;
            ctl->bar[a.bar_parity ^ 1].count = 0;  // the next launch's counter
        }
        if (tracer) trace_rec(a, tslot, 1, 0, 1);
    }

    int vpar = 0;  // the current visited bitmap: vis0 or vis1 (they swap after a bitmap pull)
    int cpar = 0;  // the list the next list pull reads
    while (true) {
        const int kind = L.kind;  // chosen by thread 0 inside the last barrier
        if (kind == kStop) break;
        const int from = L.from;
        uint32_t* const vcur = vpar ? a.vis1 : a.vis0;
        uint32_t* const vnext = vpar ? a.vis0 : a.vis1;
        // this CTA's two candidate lists
        int32_t* const cl0 = (cpar ? a.cand1 : a.cand0) + blockIdx.x * region;
        int32_t* const cl1 = (cpar ? a.cand0 : a.cand1) + blockIdx.x * region;
        CtrSlot* cur = &ctr[step % 3];
        // the frontier found at step s lives in queue (s & 1)
        const Queue qcur = (step & 1) ? Queue{a.q1, a.q1off} : Queue{a.q0, a.q0off};
        const Queue qnext = (step & 1) ? Queue{a.q0, a.q0off} : Queue{a.q1, a.q1off};
        unsigned long long qpack = s_snap[0];
        bool qlong = s_snap[4] != 0;  // the queue holds a row of more than kEntryArcs arcs
        const bool pull = kind != kPush;
        if (blockIdx.x == 0 && threadIdx.x < (int)(sizeof(CtrSlot) / 8))
            reinterpret_cast<unsigned long long*>(&ctr[(step + 2) % 3])[threadIdx.x] = 0;

        if (from == kFromBitmap) {
            // the frontier exists only as a bitmap difference: turn it into a queue
            bitmap_to_queue(a, vcur, vnext, qcur, cur);
            if (!grid_barrier(ctl, bar, bar_target, a.spin_limit, cur, s_snap)) return;
            qpack = s_snap[0];
            qlong = s_snap[4] != 0;
            if (tracer) trace_rec(a, tslot, 4, step, (long long)(qpack >> 32));
        }
        CtrSlot* out = &ctr[(step + 1) % 3];
        long long nf = 0, mf = 0;
        if (kind == kBitmapPull) {
            int32_t* keep = lists ? cl0 : nullptr;
            if (a.smem_words > 0) pull_level<true>(a, step + 1, vcur, vnext, nf, mf, keep, &s_cn);
            else pull_level<false>(a, step + 1, vcur, vnext, nf, mf, keep, &s_cn);
        } else if (kind == kListPull) {
            const LevelCount lc = list_pull_level(a, step + 1, vcur, cl0, s_cin, cl1, &s_cn);
            nf = lc.nf;
            mf = lc.mf;
            cpar ^= 1;
        } else if (from == kFromList) {
            // the frontier: entries of the last list pull's input list found by it
            const LevelCount lc = list_push_level(a, step + 1, vcur, cl1, s_cprev, out);
            nf = lc.nf;
            mf = lc.mf;
        } else {
            push_level(a, step + 1, vcur, qcur, qpack, qlong, 16 * L.reached > a.n, qnext, out, nf, mf);
        }
        flush_counts(nf, mf, out, pull ? &s_cn : nullptr);
        const int done = step + 1;
        if (!grid_barrier(ctl, bar, bar_target, a.spin_limit, out, s_snap, [advance, pull, done]() {
                if (pull) {
                    s_cprev = s_cin;  // the list just tested (read by a list push)
                    s_cin = s_cn;     // the list just written is the one the next list pull reads
                    s_cn = 0;
                }
                advance(done);
            }))
            return;
        if (tracer) trace_rec(a, tslot, kind == kPush ? 2 : (kind == kBitmapPull ? 3 : 5), step + 1, (long long)s_snap[1]);
        if (kind == kListPull && (s_snap[3] >> 32) != 0 && L.kind != kStop) {
            // the list pull's look-ahead showed la vertices at levels step + 2
            // and step + 3 (la2 of them at step + 3); when they are all that
            // is left of the component (their dist is written), those levels
            // are not run.  They count as pull levels (pull tests decided
            // them), the first in place of the one the rule had chosen.
            const long long la = (long long)(s_snap[3] >> 32);
            if (L.reached + la >= a.reach_target) {
                __syncthreads();  // every thread has read L.kind
                if (threadIdx.x == 0) {
                    const bool la2 = (s_snap[4] >> 32) != 0;
                    L.reached += la;
                    L.edges += (long long)(s_snap[4] & 0xffffffffull);
                    if (L.kind == kPush) --L.pushes;
                    else --L.pulls;
                    L.pulls += la2 ? 2 : 1;
                    L.levels = step + (la2 ? 3 : 2);
                }
                break;
            }
        }
        if (kind == kBitmapPull) {
            vpar ^= 1;
        }
        ++step;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) {
        dawn_sssp_stats s;
        s.levels = L.levels;
        s.push_steps = L.pushes;
        s.pull_steps = L.pulls;
        s.reserved = 0;
        s.reached = L.reached;
        s.edges = L.edges;
        *a.stats = s;
    }
}

}  // namespace

// Largest bitmap the pull levels copy into shared memory (n up to 1,638,400).
constexpr int kSmemBitmapMax = DAWN_SSSP_SMEM_BITMAP_MAX;

// Dynamic shared memory of a launch: the pull levels' bitmap copy (0 when it
// does not fit) or the push levels' row buffers, whichever is larger.
int sssp_dynamic_smem(int bitmap_bytes) { return bitmap_bytes > kPushBufBytes ? bitmap_bytes : kPushBufBytes; }

int sssp_occupancy(dawn_graph* g) {
    int nb = 0;
    DAWN_CUDA_TRY(cudaFuncSetAttribute(sssp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       sssp_dynamic_smem(kSmemBitmapMax)));
    const size_t words4 = (size_t)(g->nwords + 3) / 4 * 4;
    g->sssp_smem_bytes = words4 * 4 <= (size_t)kSmemBitmapMax ? (int)(words4 * 4) : 0;
    DAWN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sssp_kernel, kThreads,
                                                                sssp_dynamic_smem(g->sssp_smem_bytes)));
    if (nb < 1) return fail(DAWN_E_CUDA, "persistent SSSP kernel cannot be resident on an SM");
    g->sssp_blocks_per_sm = nb;
    return DAWN_OK;
}

int sssp_launch(dawn_graph* g, int32_t src, int32_t* dist_dev, const dawn_sssp_opts* opts,
                dawn_sssp_stats* stats_dev, cudaStream_t st) {
    if (src < 0 || src >= g->n) return fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, g->n);
    const int engine = opts ? opts->engine : DAWN_ENGINE_AUTO;
    if (engine < DAWN_ENGINE_AUTO || engine > DAWN_ENGINE_CLUSTER) return fail(DAWN_E_INVALID, "unknown engine %d", engine);
    if (opts && (opts->mode < DAWN_MODE_AUTO || opts->mode > DAWN_MODE_PULL))
        return fail(DAWN_E_INVALID, "unknown mode %d", opts->mode);
    if (engine == DAWN_ENGINE_CLUSTER) return cluster_launch(g, src, dist_dev, opts, stats_dev, st);
    if (engine == DAWN_ENGINE_AUTO && g->m < 8 * (int64_t)g->n && g->cl_size >= 0 &&
        (!opts || (opts->mode != DAWN_MODE_PULL && !opts->trace))) {
        // low-degree graph: many levels with small frontiers, one cluster runs them
        const int rc = cluster_launch(g, src, dist_dev, opts, stats_dev, st);
        if (rc == DAWN_OK || g->cl_size >= 0) return rc;  // else unavailable: the grid below
    }
    SsspArgs a;
    a.row_ptr = g->row_ptr;
    a.col_idx = g->col_idx;
    a.in_ptr = g->in_ptr;
    a.in_idx = g->in_idx;
    a.excl = g->excl;
    a.vis0 = g->vis[0];
    a.vis1 = g->vis[1];
    a.q0 = g->queue[0];
    a.q1 = g->queue[1];
    a.q0off = g->queue_off[0];
    a.q1off = g->queue_off[1];
    a.dist = dist_dev;
    a.ctl = g->ctl;
    a.stats = stats_dev;
    a.m = g->m;
    a.n = g->n;
    a.nwords = g->nwords;
    a.src = src;
    a.srb = g->row_ptr_host[src];
    a.sre = g->row_ptr_host[src + 1];
    a.reach_target = g->csize_host.empty() ? LLONG_MAX : (long long)g->csize_host[src];
    a.mode = opts ? opts->mode : DAWN_MODE_AUTO;
    a.alpha = (opts && opts->alpha > 0) ? opts->alpha : (g->tuning.alpha > 0 ? g->tuning.alpha : 15);
    a.beta = (opts && opts->beta > 0) ? opts->beta : (g->tuning.beta > 0 ? g->tuning.beta : 18);
    a.pull_serial = (opts && opts->pull_serial > 0) ? opts->pull_serial
                                                    : (g->tuning.pull_serial > 0 ? g->tuning.pull_serial : 8);
    a.spin_limit = (opts && opts->spin_limit > 0) ? opts->spin_limit : kDefaultSpin;
    a.trace = opts ? reinterpret_cast<long long*>(opts->trace) : nullptr;
    a.trace_cap = (opts && opts->trace) ? opts->trace_cap : 0;
    if (a.trace && (a.trace_cap < 0 || !is_device_ptr(a.trace)))
        return fail(DAWN_E_INVALID, "trace must be device memory with trace_cap >= 0");
    if (a.mode < DAWN_MODE_AUTO || a.mode > DAWN_MODE_PULL)
        return fail(DAWN_E_INVALID, "unknown mode %d", a.mode);
    int bps = g->sssp_blocks_per_sm;
    if (opts && opts->blocks_per_sm > 0 && opts->blocks_per_sm < bps) bps = opts->blocks_per_sm;
    a.smem_words = g->sssp_smem_bytes / 4;
    a.pull_idx = g->pull_idx;
    a.first2 = g->first2;
    a.cand0 = g->cand[0];
    a.cand1 = g->cand[1];
    a.cand_cap = g->cand_cap;
    a.bar_parity = (int32_t)(g->sssp_launches & 1u);
    dim3 grid(g->sms * bps), block(kThreads);
    void* args[] = {&a};
    DAWN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)sssp_kernel, grid, block, args,
                                              (size_t)sssp_dynamic_smem(g->sssp_smem_bytes), st));
    g->sssp_launches += 1;  // only a launch that was accepted zeroes the other counter
    return DAWN_OK;
}


// ------------------------------------------------- allocation-free variant --
// Scratch of dawn_sssp_noalloc: a file-scope device array, so that callers
// which cannot allocate device memory can still run the level loop.  Every
// GPU that loads this library holds it until the process exits.  Layout
// (256-byte aligned parts): control block | CSR check flags | visited bitmap
// | two frontier queues | their arc-offset arrays.
constexpr int32_t kNoAllocMaxN = 1 << 20;
constexpr int64_t kNoAllocMaxM = 1LL << 25;
constexpr int64_t kNoAllocQueueCap = kNoAllocMaxN + kNoAllocMaxM / kEntryArcs + 64;
constexpr size_t kNoAllocCtlOff = 0;
constexpr size_t kNoAllocBadOff = (sizeof(Ctl) + 255) / 256 * 256;
constexpr size_t kNoAllocVisOff = kNoAllocBadOff + 256;
constexpr size_t kNoAllocQ0Off = kNoAllocVisOff + (size_t)kNoAllocMaxN / 8;
constexpr size_t kNoAllocQ1Off = kNoAllocQ0Off + (size_t)kNoAllocQueueCap * sizeof(int2);
constexpr size_t kNoAllocQ0OffOff = kNoAllocQ1Off + (size_t)kNoAllocQueueCap * sizeof(int2);
constexpr size_t kNoAllocQ1OffOff = kNoAllocQ0OffOff + ((size_t)kNoAllocQueueCap * sizeof(int32_t) + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocQ1OffOff + (size_t)kNoAllocQueueCap * sizeof(int32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// bad[0]: smallest bad row_ptr index; bad[1]: smallest bad col_idx index.
__global__ void noalloc_check_csr_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                         int32_t n, long long m, unsigned long long* bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = t0; i <= n; i += stride) {
        const int v = rp[i];
        bool ok = v >= 0 && v <= m && (i == 0 ? v == 0 : v >= rp[i - 1]);
        if (i == n) ok = ok && v == m;
        if (!ok) atomicMin(&bad[0], (unsigned long long)i);
    }
    for (long long j = t0; j < m; j += stride) {
        const int c = ci[j];
        if (c < 0 || c >= n) atomicMin(&bad[1], (unsigned long long)j);
    }
}

struct NoAllocDevice {
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
    int blocks_per_sm = 0;
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// Once per device, with that device current: the scratch array's device
// address (host code only sees a host-side stand-in for its name) and the
// persistent kernel's occupancy.
int noalloc_setup(NoAllocDevice** out) {
    int dev = 0;
    DAWN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(DAWN_E_INVALID, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.scratch) {
        void* p = nullptr;
        DAWN_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        DAWN_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        DAWN_CUDA_TRY(cudaFuncSetAttribute(sssp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       sssp_dynamic_smem(kSmemBitmapMax)));
        DAWN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.blocks_per_sm, sssp_kernel, kThreads,
                                                                    kPushBufBytes));
        if (d.blocks_per_sm < 1) return fail(DAWN_E_CUDA, "persistent SSSP kernel cannot be resident on an SM");
        d.scratch = static_cast<unsigned char*>(p);
    }
    *out = &d;
    return DAWN_OK;
}

}  // namespace

int sssp_noalloc(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t m, int32_t src,
                 int32_t* dist, cudaStream_t st) {
    if (n < 1 || n > kNoAllocMaxN)
        return fail(DAWN_E_INVALID, "n = %d: dawn_sssp_noalloc handles 1 <= n <= %d", n, kNoAllocMaxN);
    if (m < 0 || m > kNoAllocMaxM)
        return fail(DAWN_E_INVALID, "m = %lld: dawn_sssp_noalloc handles 0 <= m <= %lld", (long long)m,
                    (long long)kNoAllocMaxM);
    if (src < 0 || src >= n) return fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, n);
    if (!is_device_ptr(row_ptr) || (m > 0 && !is_device_ptr(col_idx)) || !is_device_ptr(dist))
        return fail(DAWN_E_INVALID, "row_ptr, col_idx and dist must be device memory");
    NoAllocDevice* d = nullptr;
    int rc = noalloc_setup(&d);
    if (rc != DAWN_OK) return rc;
    Ctl* ctl = reinterpret_cast<Ctl*>(d->scratch + kNoAllocCtlOff);
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(d->scratch + kNoAllocBadOff);

    // the CSR comes straight from the caller: check it before any traversal
    unsigned long long bad_h[2] = {0, 0};
    DAWN_CUDA_TRY(cudaMemsetAsync(bad, 0xff, 2 * sizeof(unsigned long long), st));
    const long long work = (long long)n + 1 > m ? (long long)n + 1 : (long long)m;
    long long nb = (work + 255) / 256;
    if (nb > (long long)d->sms * 8) nb = (long long)d->sms * 8;
    noalloc_check_csr_kernel<<<(int)(nb < 1 ? 1 : nb), 256, 0, st>>>(row_ptr, col_idx, n, (long long)m, bad);
    DAWN_CUDA_TRY(cudaGetLastError());
    DAWN_CUDA_TRY(cudaMemcpyAsync(bad_h, bad, sizeof(bad_h), cudaMemcpyDeviceToHost, st));
    DAWN_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad_h[0] != ~0ULL)
        return fail(DAWN_E_INVALID, "row_ptr[%llu] breaks row_ptr[0] = 0 <= ... <= row_ptr[n] = m", bad_h[0]);
    if (bad_h[1] != ~0ULL) return fail(DAWN_E_INVALID, "col_idx[%llu] is outside [0, n)", bad_h[1]);

    // the array keeps the previous call's contents: the barrier state and the
    // status word must start at zero (the kernel clears its own counters)
    DAWN_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
    SsspArgs a;
    a.row_ptr = row_ptr;
    a.col_idx = col_idx;
    a.in_ptr = nullptr;  // push (SOVM) only: the in-adjacency is never read
    a.in_idx = nullptr;
    a.excl = nullptr;
    a.vis0 = reinterpret_cast<uint32_t*>(d->scratch + kNoAllocVisOff);
    a.vis1 = nullptr;
    a.q0 = reinterpret_cast<int2*>(d->scratch + kNoAllocQ0Off);
    a.q1 = reinterpret_cast<int2*>(d->scratch + kNoAllocQ1Off);
    a.q0off = reinterpret_cast<int32_t*>(d->scratch + kNoAllocQ0OffOff);
    a.q1off = reinterpret_cast<int32_t*>(d->scratch + kNoAllocQ1OffOff);
    a.dist = dist;
    a.ctl = ctl;
    a.stats = nullptr;
    a.trace = nullptr;
    a.trace_cap = 0;
    a.m = m;
    a.n = n;
    a.nwords = (int32_t)(((int64_t)n + 31) / 32);
    a.src = src;
    a.srb = a.sre = -1;  // the caller's CSR: read on the device
    a.reach_target = LLONG_MAX;
    a.mode = DAWN_MODE_PUSH;
    a.bar_parity = 0;  // the whole control block was just zeroed
    a.smem_words = 0;
    a.pull_idx = nullptr;  // push only
    a.first2 = nullptr;
    a.cand0 = nullptr;  // push only: no candidate lists
    a.cand1 = nullptr;
    a.cand_cap = 0;
    a.alpha = 15;
    a.beta = 18;
    a.pull_serial = 8;
    a.spin_limit = kDefaultSpin;
    dim3 grid(d->sms * d->blocks_per_sm), block(kThreads);
    void* args[] = {&a};
    DAWN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)sssp_kernel, grid, block, args, kPushBufBytes, st));
    int status = 0;
    DAWN_CUDA_TRY(cudaMemcpyAsync(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DAWN_CUDA_TRY(cudaStreamSynchronize(st));
    if (status == DEV_TIMEOUT) return fail(DAWN_E_TIMEOUT, "a grid-barrier wait on the device ran out of its spin budget");
    if (status != DEV_OK) return fail(DAWN_E_CUDA, "unknown device status %d", status);
    return DAWN_OK;
}

}  // namespace dawn

extern "C" {

DAWN_API int dawn_sssp_ex(dawn_graph_t g, int32_t src, int32_t* dist, const dawn_sssp_opts* opts,
                          dawn_sssp_stats* stats, void* stream) {
    if (!g) return dawn::fail(DAWN_E_INVALID, "graph is NULL");
    if (!dist) return dawn::fail(DAWN_E_INVALID, "dist is NULL");
    if (src < 0 || src >= g->n) return dawn::fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, g->n);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = dawn::is_device_ptr(dist);
    int32_t* d = dev ? dist : g->dist_tmp;
    int rc = dawn::sssp_launch(g, src, d, opts, g->stats_dev, st);
    if (rc != DAWN_OK) return rc;
    if (!dev) DAWN_CUDA_TRY(cudaMemcpyAsync(dist, d, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost, st));
    if (stats) DAWN_CUDA_TRY(cudaMemcpyAsync(g->stats_host, g->stats_dev, sizeof(dawn_sssp_stats), cudaMemcpyDeviceToHost, st));
    rc = dawn::graph_sync_status(g, st);
    if (rc != DAWN_OK) return rc;
    if (stats) *stats = *g->stats_host;
    return DAWN_OK;
}

DAWN_API int dawn_sssp(dawn_graph_t g, int32_t src, int32_t* dist, void* stream) {
    return dawn_sssp_ex(g, src, dist, nullptr, nullptr, stream);
}

DAWN_API int dawn_sssp_async(dawn_graph_t g, int32_t src, int32_t* dist_dev, const dawn_sssp_opts* opts,
                             dawn_sssp_stats* stats_dev, void* stream) {
    if (!g) return dawn::fail(DAWN_E_INVALID, "graph is NULL");
    if (!dist_dev || !dawn::is_device_ptr(dist_dev)) return dawn::fail(DAWN_E_INVALID, "dist_dev must be device memory");
    if (stats_dev && !dawn::is_device_ptr(stats_dev)) return dawn::fail(DAWN_E_INVALID, "stats_dev must be device memory or NULL");
    if (src < 0 || src >= g->n) return dawn::fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, g->n);
    return dawn::sssp_launch(g, src, dist_dev, opts, stats_dev, (cudaStream_t)stream);
}

DAWN_API int dawn_sssp_noalloc(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t m,
                              int32_t src, int32_t* dist, void* stream) {
    return dawn::sssp_noalloc(row_ptr, col_idx, n, m, src, dist, (cudaStream_t)stream);
}

}  // extern "C"
