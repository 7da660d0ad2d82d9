// Weighted extension: single-source shortest paths over the (min, +)
// semiring.  Sec. 5 names (min, +) operations on weighted graphs as the
// direction in which DAWN is to be extended; the unweighted path's SOVM
// (Alg. 3) carries over with (OR, AND) replaced by (min, +):
//
//   round r: every frontier vertex u (its distance fell in round r - 1)
//            offers d(u) + w(u, v) to each out-neighbour v; v keeps the
//            smaller value (an atomic minimum on 64 bits); the vertices
//            whose distance fell form the frontier of round r + 1.
//
// The loop stops on a round that lowers nothing; with non-negative weights
// at most n - 1 rounds lower something.  A vertex is queued at most once per
// round (a mark bit per round parity).  Rounds run in one persistent
// cooperative kernel separated by a bounded grid barrier, as in sssp.cu.
// The distances a round reads are whatever is in memory when it reads them
// (a value lowered earlier in the same round is offered at once): after
// round k every distance is at most the synchronous iterate d_k, so the
// result is the same fixpoint and the rounds are no more than the
// synchronous ones.
//
// Work per round is split by arcs: the frontier is a queue of records
// {vertex, first arc, arc count} with each record's offset in the round's
// concatenated arc list, and every warp takes an equal range of arcs (a
// 32-ary search finds the record holding its first arc), so a hub row is
// spread over many warps.
//
// Distances are unsigned 64-bit in the kernel with ~0 for "no path", which
// is -1 when read as the int64 the caller sees.
#include <climits>

#include "dawn_internal.cuh"

namespace dawn {
namespace {

constexpr int kWThreads = 512;
constexpr int kWWarps = kWThreads / 32;
constexpr unsigned kWFull = 0xffffffffu;
constexpr unsigned long long kNoPath = ~0ull;

// Counters of one round, on their own 128-byte line.
struct alignas(128) WSlot {
    unsigned long long qpack;    // frontier records (high 32 bits) | their arcs (low 32 bits)
    unsigned long long lowered;  // atomic minimums that lowered a distance
    unsigned long long reached;  // ... of which the first for their vertex (it was unreached)
    unsigned long long pad[13];
};

// Launches alternate between two barrier counters and two sets of three
// round slots (slot r % 3 holds round r's frontier counts); each launch
// zeroes the other parity's for the next one.
struct alignas(128) WCtl {
    BarCounter bar[2];
    WSlot slot[2][3];
};

struct WeightedState {
    int32_t* w = nullptr;               // arc weights, aligned with col_idx
    int2* cw = nullptr;                 // {col_idx, weight} per arc: one 8-byte load per offered arc
    int32_t* qv[2] = {nullptr, nullptr};  // frontier records: vertex
    int2* qe[2] = {nullptr, nullptr};     // {first arc, arc count}
    int32_t* qo[2] = {nullptr, nullptr};  // arc offset within the round
    uint32_t* mark[2] = {nullptr, nullptr};  // queued-this-round bits, by round parity
    WCtl* ctl = nullptr;
    int64_t* dist_tmp = nullptr;        // staging for host outputs
    dawn_wsssp_stats* stats_dev = nullptr;
    int blocks_per_sm = 0;
    unsigned launches = 0;
};

struct WArgs {
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col_idx;
    const int32_t* __restrict__ w;
    const int2* __restrict__ cw;
    unsigned long long* dist;
    int32_t* qv[2];
    int2* qe[2];
    int32_t* qo[2];
    uint32_t* mark[2];
    WCtl* ctl;
    int* status;
    dawn_wsssp_stats* stats;
    long long spin_limit;
    int32_t n, nwords, src, parity;
};

__device__ __forceinline__ unsigned w_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int w_ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long w_ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier (same protocol as the single-source one): release-add on the
// launch's arrival counter, acquire polls up to a running target, bounded by
// spin_limit clock cycles (DEV_TIMEOUT, and every CTA returns).  Thread 0
// copies the three counters of `snap` into s_snap for the CTA.
__device__ bool w_barrier(const WArgs& a, unsigned* count, unsigned& target, const WSlot* snap,
                          unsigned long long* s_snap) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const long long t0 = clock64();
        unsigned polls = 0;
        while ((int)(w_ld_acquire(count) - target) < 0) {
            if (clock64() - t0 > a.spin_limit) {
                atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
            if ((++polls & 15u) == 0 && w_ld_relaxed_s32(a.status) != DEV_OK) { ok = 0; break; }
        }
        if (ok) {
            s_snap[0] = w_ld_relaxed_u64(&snap->qpack);
            s_snap[1] = w_ld_relaxed_u64(&snap->lowered);
            s_snap[2] = w_ld_relaxed_u64(&snap->reached);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int w_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kWFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Sum the per-thread counts over the CTA and add them to the round's slot.
__device__ __forceinline__ void w_flush(long long lowered, long long reached, WSlot* out) {
    __shared__ long long s_a[kWWarps], s_b[kWWarps];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lowered += __shfl_down_sync(kWFull, lowered, o);
        reached += __shfl_down_sync(kWFull, reached, o);
    }
    if (lane == 0) { s_a[wl] = lowered; s_b[wl] = reached; }
    __syncthreads();
    if (wl == 0) {
        long long x = lane < kWWarps ? s_a[lane] : 0, y = lane < kWWarps ? s_b[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(kWFull, x, o);
            y += __shfl_down_sync(kWFull, y, o);
        }
        if (lane == 0) {
            if (x) atomicAdd(&out->lowered, (unsigned long long)x);
            if (y) atomicAdd(&out->reached, (unsigned long long)y);
        }
    }
}

// Windows of 32 arcs a warp takes per group (see relax_round).
constexpr int kWGroup = 4;

// Queue records gathered per warp in shared memory and reserved in the next
// round's queue in batches: one 64-bit atomic on the round's counter per
// batch (>= kWFlush records) rather than one per group of windows, since the
// reservations of every warp meet on that one counter.
constexpr int kWBuf = 192;                     // records a warp's buffer holds
constexpr int kWFlush = kWBuf - 32 * kWGroup;  // flush at this fill: a group adds at most 32 * kWGroup
__shared__ int s_wbuf_v[kWWarps][kWBuf];       // vertex
__shared__ int2 s_wbuf_e[kWWarps][kWBuf];      // {first arc, arc count}

// Append the lanes' queued vertices with a non-empty row to the warp's buffer
// (nbuf records, warp-uniform).  Full warp.
__device__ __forceinline__ void w_buffer_group(unsigned q, const int* v, const int* rb, const int* re, int lane,
                                               int* bv, int2* be, int& nbuf) {
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < kWGroup; ++i) cnt += ((q >> i) & 1u) && re[i] > rb[i];
    const int incl = w_scan(cnt, lane);
    int pos = nbuf + incl - cnt;
#pragma unroll
    for (int i = 0; i < kWGroup; ++i) {
        if (((q >> i) & 1u) && re[i] > rb[i]) {
            bv[pos] = v[i];
            be[pos] = make_int2(rb[i], re[i] - rb[i]);
            ++pos;
        }
    }
    nbuf += __shfl_sync(kWFull, incl, 31);
    __syncwarp();
}

// Reserve the warp's nbuf buffered records in the next round's queue (one
// atomic: records in the high word, arcs in the low word) and copy them
// there with each record's arc offset.  Full warp.
__device__ __forceinline__ void w_flush_buffer(const int* bv, const int2* be, int nbuf, int lane, int32_t* qv,
                                               int2* qe, int32_t* qo, WSlot* out) {
    int arcs = 0;
    for (int i = lane; i < nbuf; i += 32) arcs += be[i].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arcs += __shfl_xor_sync(kWFull, arcs, o);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&out->qpack, ((unsigned long long)nbuf << 32) | (unsigned)arcs);
    base = __shfl_sync(kWFull, base, 0);
    const int slot0 = (int)(base >> 32);
    int carry = (int)(base & 0xffffffffu);
    for (int i0 = 0; i0 < nbuf; i0 += 32) {
        const int i = i0 + lane;
        const int2 e = i < nbuf ? be[i] : make_int2(0, 0);
        const int incl = w_scan(e.y, lane);
        if (i < nbuf) {
            qv[slot0 + i] = bv[i];
            qe[slot0 + i] = e;
            qo[slot0 + i] = carry + incl - e.y;
        }
        carry += __shfl_sync(kWFull, incl, 31);
    }
    __syncwarp();
}

// One (min, +) round over the frontier of round r (qn records, E arcs).  A
// warp walks its arc range in groups of kWGroup windows of 32 consecutive
// arcs; within a group the loads of every step (arcs and weights, the heads'
// distances, the atomic minimums, the marks, the heads' rows) are issued for
// all windows together, so the warp waits for one chain of round trips per
// group, not per window.
__device__ void relax_round(const WArgs& a, int r, int qn, long long E, WSlot* out, long long& lowered,
                            long long& reached) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * kWWarps;
    const long long gw = (long long)blockIdx.x * kWWarps + (threadIdx.x >> 5);
    const int32_t* qv = a.qv[r & 1];
    const int2* qe = a.qe[r & 1];
    const int32_t* qo = a.qo[r & 1];
    uint32_t* mark = a.mark[(r + 1) & 1];
    long long chunk = (E + nw - 1) / nw;
    chunk = (chunk + 31) & ~31LL;
    const long long a0 = gw * chunk;
    if (a0 >= E) return;  // warp-uniform
    const long long a1 = min(E, a0 + chunk);
    // the record holding arc a0: the largest i with qo[i] <= a0 (qo[0] = 0)
    int lo = 0, hi = qn;
    while (hi - lo > 32) {
        const int stp = (hi - lo + 31) >> 5;
        const int p = lo + lane * stp;
        const int v = p < hi ? __ldcg(qo + p) : INT_MAX;
        const unsigned b = __ballot_sync(kWFull, (long long)v <= a0);
        const int k = 31 - __clz(b);
        lo += k * stp;
        hi = min(hi, lo + stp);
    }
    int bstart = lo;
    // the batch: lane k holds record bstart + k and its vertex's distance
    int2 e;
    int off;
    unsigned long long du;
    auto load = [&](int b) {
        const int i = b + lane;
        if (i < qn) {
            e = __ldcg(qe + i);
            off = __ldcg(qo + i);
            du = __ldcg(a.dist + __ldcg(qv + i));
        } else {
            e = make_int2(0, 0);
            off = INT_MAX;
            du = kNoPath;
        }
    };
    load(bstart);
    int32_t* nqv = a.qv[(r + 1) & 1];
    int2* nqe = a.qe[(r + 1) & 1];
    int32_t* nqo = a.qo[(r + 1) & 1];
    int* bv = s_wbuf_v[threadIdx.x >> 5];
    int2* be = s_wbuf_e[threadIdx.x >> 5];
    int nbuf = 0;  // warp-uniform
    // the record holding the last arc of the window before (warp-uniform):
    // its arcs [c_lo, c_hi) of the round's list start at col_idx[c_ost], and
    // its vertex's distance is c_du.  A window inside it (a long row) needs
    // no search.
    int c_lo = 1, c_hi = 0;  // arc offsets within a round stay below 2^31
    int c_ost = 0;
    unsigned long long c_du = 0;
    for (long long gb = a0; gb < a1; gb += 32 * kWGroup) {
        int j[kWGroup];
        unsigned long long odu[kWGroup];
#pragma unroll
        for (int q = 0; q < kWGroup; ++q) {
            const long long wb = gb + 32 * q;
            j[q] = -1;
            odu[q] = 0;
            if (wb >= a1) continue;  // warp-uniform
            const long long last = min(wb + 31, a1 - 1);
            const long long t = wb + lane;
            if (wb >= (long long)c_lo && last < (long long)c_hi) {  // warp-uniform
                odu[q] = c_du;
                if (t < a1) j[q] = c_ost + (int)(t - c_lo);
                continue;
            }
            // keep the batch covering the window [wb, last]: if its last arc
            // lies past the batch's last record, restart the batch at the
            // record holding wb
            const int off31 = __shfl_sync(kWFull, off, 31);
            const int len31 = __shfl_sync(kWFull, e.y, 31);
            if (bstart + 32 < qn && last >= (long long)off31 + len31) {
                int k;
                if (wb >= (long long)off31 + len31) k = 32;
                else k = 31 - __clz(__ballot_sync(kWFull, (long long)off <= wb));
                bstart += k;
                load(bstart);
            }
            int o = 0;
#pragma unroll
            for (int b = 16; b > 0; b >>= 1) {
                const int pv = __shfl_sync(kWFull, off, o + b);
                if ((long long)pv <= t) o += b;
            }
            const int ost = __shfl_sync(kWFull, e.x, o);
            const int ooff = __shfl_sync(kWFull, off, o);
            odu[q] = __shfl_sync(kWFull, du, o);
            if (t < a1) j[q] = ost + (int)(t - ooff);
            // remember the record of the window's last arc
            const int ol = __shfl_sync(kWFull, o, (int)(last - wb));
            c_ost = __shfl_sync(kWFull, e.x, ol);
            c_lo = __shfl_sync(kWFull, off, ol);
            c_hi = c_lo + __shfl_sync(kWFull, e.y, ol);
            c_du = __shfl_sync(kWFull, du, ol);
        }
        int c[kWGroup];
        unsigned long long nd[kWGroup];
#pragma unroll
        for (int q = 0; q < kWGroup; ++q) {
            const int2 t = j[q] >= 0 ? __ldg(a.cw + j[q]) : make_int2(0, 0);
            c[q] = t.x;
            nd[q] = j[q] >= 0 ? odu[q] + (unsigned long long)(unsigned)t.y : kNoPath;
        }
        unsigned long long cur[kWGroup];
#pragma unroll
        for (int q = 0; q < kWGroup; ++q) cur[q] = j[q] >= 0 ? __ldcg(a.dist + c[q]) : 0ull;
        // an offer below the head's current distance: the head's distance
        // falls this round (to this offer or to a smaller one), so the head
        // belongs to the next frontier whatever the atomic minimum returns;
        // the minimum, the mark and the head's row are issued together
        unsigned offer = 0;
#pragma unroll
        for (int q = 0; q < kWGroup; ++q)
            if (j[q] >= 0 && nd[q] < cur[q]) offer |= 1u << q;
        unsigned long long old[kWGroup];
        uint32_t mw[kWGroup];
        int rb[kWGroup], re[kWGroup];
#pragma unroll
        for (int q = 0; q < kWGroup; ++q) {
            old[q] = kNoPath;
            mw[q] = ~0u;
            rb[q] = re[q] = 0;
            if ((offer >> q) & 1u) {
                old[q] = atomicMin(a.dist + c[q], nd[q]);
                mw[q] = atomicOr(mark + (c[q] >> 5), 1u << (c[q] & 31));
                rb[q] = __ldg(a.row_ptr + c[q]);
                re[q] = __ldg(a.row_ptr + c[q] + 1);
            }
        }
        // queued once per round: the offer that set the mark queues the head
        unsigned qd = 0;
#pragma unroll
        for (int q = 0; q < kWGroup; ++q) {
            if (!((offer >> q) & 1u)) continue;
            if (nd[q] < old[q]) {
                lowered += 1;
                reached += old[q] == kNoPath;
            }
            if (!((mw[q] >> (c[q] & 31)) & 1u)) qd |= 1u << q;
        }
        w_buffer_group(qd, c, rb, re, lane, bv, be, nbuf);
        if (nbuf >= kWFlush) {
            w_flush_buffer(bv, be, nbuf, lane, nqv, nqe, nqo, out);
            nbuf = 0;
        }
    }
    if (nbuf > 0) w_flush_buffer(bv, be, nbuf, lane, nqv, nqe, nqo, out);
}

__global__ void __launch_bounds__(kWThreads, 2) wsssp_kernel(WArgs a) {
    __shared__ unsigned long long s_snap[3];
    __shared__ int s_status;
    if (threadIdx.x == 0) s_status = w_ld_relaxed_s32(a.status);
    const long long gtid = (long long)blockIdx.x * kWThreads + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * kWThreads;
    WSlot* slot = a.ctl->slot[a.parity];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x < 3 * (int)(sizeof(WSlot) / 8))
        reinterpret_cast<unsigned long long*>(a.ctl->slot[a.parity ^ 1])[threadIdx.x] = 0;
    unsigned* bar = &a.ctl->bar[a.parity].count;
    unsigned target = 0;

    // init: every distance "no path" but the source's; no marks; frontier = {src}
    for (long long v = gtid; v < a.n; v += gthreads)
        if (v != a.src) a.dist[v] = kNoPath;
    for (long long i = gtid; i < 2LL * a.nwords; i += gthreads) a.mark[i >= a.nwords][i % a.nwords] = 0u;
    if (gtid == 0) {
        a.dist[a.src] = 0;
        const int rb = __ldg(a.row_ptr + a.src), re = __ldg(a.row_ptr + a.src + 1);
        if (re > rb) {
            a.qv[0][0] = a.src;
            a.qe[0][0] = make_int2(rb, re - rb);
            a.qo[0][0] = 0;
            slot[0].qpack = (1ull << 32) | (unsigned)(re - rb);
        }
        slot[0].reached = 1;
    }
    __syncthreads();
    if (s_status != DEV_OK) return;  // an earlier call failed: no barrier (outputs undefined)
    if (!w_barrier(a, bar, target, &slot[0], s_snap)) return;
    if (gtid == 0) a.ctl->bar[a.parity ^ 1].count = 0;  // the next launch's counter

    long long rounds = 0, reached_total = (long long)s_snap[2], lowered_total = 0, relax_total = 0;
    for (int r = 0;; ++r) {
        const unsigned long long qp = s_snap[0];
        const int qn = (int)(qp >> 32);
        const long long E = (long long)(qp & 0xffffffffull);
        if (qn == 0) break;
        if (r >= a.n) {  // cannot happen with non-negative weights
            if (gtid == 0) atomicCAS(a.status, DEV_OK, DEV_TIMEOUT);
            return;
        }
        relax_total += E;
        WSlot* out = &slot[(r + 1) % 3];
        if (blockIdx.x == 0 && threadIdx.x < (int)(sizeof(WSlot) / 8))
            reinterpret_cast<unsigned long long*>(&slot[(r + 2) % 3])[threadIdx.x] = 0;
        // this round's records were marked when they were queued; clear the
        // marks so that round r + 2 finds its mark bits at zero
        for (long long i = gtid; i < qn; i += gthreads) {
            const int v = __ldcg(a.qv[r & 1] + i);
            atomicAnd(a.mark[r & 1] + (v >> 5), ~(1u << (v & 31)));
        }
        long long lowered = 0, reached = 0;
        relax_round(a, r, qn, E, out, lowered, reached);
        w_flush(lowered, reached, out);
        if (!w_barrier(a, bar, target, out, s_snap)) return;
        if (s_snap[1] > 0) ++rounds;
        lowered_total += (long long)s_snap[1];
        reached_total += (long long)s_snap[2];
    }
    if (gtid == 0 && a.stats) {
        dawn_wsssp_stats s;
        s.rounds = (int32_t)rounds;
        s.reserved = 0;
        s.reached = reached_total;
        s.relaxations = relax_total;
        s.improvements = lowered_total;
        *a.stats = s;
    }
}

// First index j with w[j] < 0 (atomicMin over a 64-bit slot preset to ~0).
__global__ void interleave_kernel(const int32_t* __restrict__ ci, const int32_t* __restrict__ w, long long m,
                                  int2* __restrict__ cw) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x)
        cw[j] = make_int2(ci[j], w[j]);
}

__global__ void negative_weight_kernel(const int32_t* __restrict__ w, long long m, unsigned long long* first) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x)
        if (w[j] < 0) atomicMin(first, (unsigned long long)j);
}

WeightedState* state(dawn_graph* g) { return static_cast<WeightedState*>(g->weighted); }

int w_grid(int64_t work, int sms) {
    int64_t b = (work + 255) / 256;
    if (b > (int64_t)sms * 8) b = (int64_t)sms * 8;
    return b < 1 ? 1 : (int)b;
}

int wsssp_launch(dawn_graph* g, int32_t src, int64_t* dist_dev, dawn_wsssp_stats* stats_dev, cudaStream_t st) {
    WeightedState* s = state(g);
    if (!s || !s->w) return fail(DAWN_E_INVALID, "graph has no weights (dawn_graph_set_weights)");
    if (src < 0 || src >= g->n) return fail(DAWN_E_INVALID, "source %d outside [0, %d)", src, g->n);
    if (!dist_dev || !is_device_ptr(dist_dev)) return fail(DAWN_E_INVALID, "dist must be device memory");
    if (stats_dev && !is_device_ptr(stats_dev)) return fail(DAWN_E_INVALID, "stats must be device memory or NULL");
    WArgs a;
    a.row_ptr = g->row_ptr;
    a.col_idx = g->col_idx;
    a.w = s->w;
    a.cw = s->cw;
    a.dist = reinterpret_cast<unsigned long long*>(dist_dev);
    for (int p = 0; p < 2; ++p) {
        a.qv[p] = s->qv[p];
        a.qe[p] = s->qe[p];
        a.qo[p] = s->qo[p];
        a.mark[p] = s->mark[p];
    }
    a.ctl = s->ctl;
    a.status = &g->ctl->status;
    a.stats = stats_dev;
    a.spin_limit = kDefaultSpin;
    a.n = g->n;
    a.nwords = g->nwords;
    a.src = src;
    a.parity = (int32_t)(s->launches & 1u);
    void* args[] = {&a};
    const dim3 grid((unsigned)(g->sms * s->blocks_per_sm)), block(kWThreads);
    DAWN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)wsssp_kernel, grid, block, args, 0, st));
    s->launches += 1;
    return DAWN_OK;
}

}  // namespace

void weighted_release(dawn_graph* g) {
    WeightedState* s = state(g);
    if (!s) return;
    auto f = [](void* p) { if (p) cudaFree(p); };
    f(s->w);
    f(s->cw);
    for (int p = 0; p < 2; ++p) {
        f(s->qv[p]);
        f(s->qe[p]);
        f(s->qo[p]);
        f(s->mark[p]);
    }
    f(s->ctl);
    f(s->dist_tmp);
    f(s->stats_dev);
    delete s;
    g->weighted = nullptr;
}

int weighted_reset(dawn_graph* g, cudaStream_t st) {
    WeightedState* s = state(g);
    if (!s || !s->ctl) return DAWN_OK;
    DAWN_CUDA_TRY(cudaMemsetAsync(s->ctl, 0, sizeof(WCtl), st));
    return DAWN_OK;
}

}  // namespace dawn

extern "C" {

DAWN_API int dawn_graph_set_weights(dawn_graph_t g, const int32_t* weights, void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!weights && g->m > 0) return fail(DAWN_E_INVALID, "weights is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    WeightedState* s = state(g);
    if (!s) {
        s = new WeightedState();
        g->weighted = s;
        const size_t n = (size_t)g->n, words = (size_t)g->nwords;
        const size_t mw = (size_t)(g->m > 0 ? g->m : 1);
        cudaError_t e = cudaMalloc((void**)&s->w, sizeof(int32_t) * mw);
        for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
            e = cudaMalloc((void**)&s->qv[p], sizeof(int32_t) * n);
            if (e == cudaSuccess) e = cudaMalloc((void**)&s->qe[p], sizeof(int2) * n);
            if (e == cudaSuccess) e = cudaMalloc((void**)&s->qo[p], sizeof(int32_t) * n);
            if (e == cudaSuccess) e = cudaMalloc((void**)&s->mark[p], sizeof(uint32_t) * words);
        }
        if (e == cudaSuccess) e = cudaMalloc((void**)&s->ctl, sizeof(WCtl));
        if (e == cudaSuccess) e = cudaMalloc((void**)&s->stats_dev, sizeof(dawn_wsssp_stats));
        if (e == cudaSuccess) e = cudaMemsetAsync(s->ctl, 0, sizeof(WCtl), st);
        if (e == cudaSuccess) {
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wsssp_kernel, kWThreads, 0);
            s->blocks_per_sm = nb;
            if (e == cudaSuccess && nb < 1) {
                weighted_release(g);
                return fail(DAWN_E_CUDA, "weighted kernel cannot be resident on an SM");
            }
        }
        if (e != cudaSuccess) {
            weighted_release(g);
            return cuda_fail(e, "dawn_graph_set_weights (allocation)", __FILE__, __LINE__);
        }
    }
    if (!s->w) {  // an earlier set was rejected
        const cudaError_t ea = cudaMalloc((void**)&s->w, sizeof(int32_t) * (size_t)(g->m > 0 ? g->m : 1));
        if (ea != cudaSuccess) return cuda_fail(ea, "dawn_graph_set_weights (allocation)", __FILE__, __LINE__);
    }
    if (g->m == 0) return DAWN_OK;
    unsigned long long* first = nullptr;
    unsigned long long first_h = ~0ull;
    cudaError_t e = cudaMemcpyAsync(s->w, weights, sizeof(int32_t) * (size_t)g->m, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&first, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(first, 0xff, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        negative_weight_kernel<<<w_grid(g->m, g->sms), 256, 0, st>>>(s->w, (long long)g->m, first);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&first_h, first, sizeof(first_h), cudaMemcpyDeviceToHost, st);
    if (first) cudaFreeAsync(first, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "dawn_graph_set_weights", __FILE__, __LINE__);
    if (first_h != ~0ull) {
        cudaFree(s->w);  // no weights until a valid set arrives
        s->w = nullptr;
        return fail(DAWN_E_INVALID, "weights[%llu] is negative", first_h);
    }
    if (!s->cw) DAWN_CUDA_TRY(cudaMalloc((void**)&s->cw, sizeof(int2) * (size_t)g->m));
    interleave_kernel<<<w_grid(g->m, g->sms), 256, 0, st>>>(g->col_idx, s->w, (long long)g->m, s->cw);
    DAWN_CUDA_TRY(cudaGetLastError());
    return DAWN_OK;
}

DAWN_API int dawn_wsssp_async(dawn_graph_t g, int32_t src, int64_t* dist_dev, dawn_wsssp_stats* stats_dev,
                              void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    return wsssp_launch(g, src, dist_dev, stats_dev, (cudaStream_t)stream);
}

DAWN_API int dawn_wsssp(dawn_graph_t g, int32_t src, int64_t* dist, dawn_wsssp_stats* stats, void* stream) {
    using namespace dawn;
    if (!g) return fail(DAWN_E_INVALID, "graph is NULL");
    if (!dist) return fail(DAWN_E_INVALID, "dist is NULL");
    WeightedState* s = state(g);
    if (!s || !s->w) return fail(DAWN_E_INVALID, "graph has no weights (dawn_graph_set_weights)");
    cudaStream_t st = (cudaStream_t)stream;
    const bool ddev = is_device_ptr(dist);
    if (!ddev && !s->dist_tmp)
        DAWN_CUDA_TRY(cudaMalloc((void**)&s->dist_tmp, sizeof(int64_t) * (size_t)g->n));
    int64_t* d = ddev ? dist : s->dist_tmp;
    const bool sdev = stats && is_device_ptr(stats);
    int rc = wsssp_launch(g, src, d, stats ? (sdev ? stats : s->stats_dev) : nullptr, st);
    if (rc != DAWN_OK) return rc;
    if (!ddev)
        DAWN_CUDA_TRY(cudaMemcpyAsync(dist, d, sizeof(int64_t) * (size_t)g->n, cudaMemcpyDeviceToHost, st));
    if (stats && !sdev)
        DAWN_CUDA_TRY(cudaMemcpyAsync(stats, s->stats_dev, sizeof(dawn_wsssp_stats), cudaMemcpyDeviceToHost, st));
    return graph_sync_status(g, st);
}

}  // extern "C"
