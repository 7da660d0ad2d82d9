// Single-source level loop on one thread-block cluster (the SOVM push of
// Alg. 3 / Eq. 5-7), for graphs with small frontiers and many levels
// (high-diameter, low-degree graphs), where the grid-wide version spends most
// of a level in the grid barrier and in round trips to L2.
//
// The cluster's CTAs (16, or 8) share the visited bitmap through distributed
// shared memory: CTA r holds words [r*S, (r+1)*S).  A level expands the
// frontier: every out-arc (u, x) of a frontier vertex claims x with an atomic
// OR on the owner CTA's word (a shared-memory atomic when the claiming CTA
// owns x, which on a lattice of contiguous rows is nearly always; a test and
// then a distributed-shared-memory atomic otherwise); the claim that sets the
// bit writes dist[x] = level and appends x to its owner's next frontier list
// (shared memory, spilling to a global list when full), so each CTA expands
// the vertices of its own slice.  Levels are separated by the hardware cluster
// barrier.  A vertex is claimed once, at the first level an arc reaches it,
// which is its distance (Thm 1).
//
// Many sources (dawn_sssp_many): a grid of several clusters, each taking the
// next source from a device counter and running its level loop alone (its
// own overflow lists), so independent searches fill the SMs one cluster
// cannot; no cluster ever waits for another (Sec. 3.3: APSP as one SSSP per
// source).
#include <algorithm>
#include <cooperative_groups.h>

#include "dawn_internal.cuh"

namespace cg = cooperative_groups;

namespace dawn {
namespace {

constexpr int kClThreads = 1024;
constexpr int kClWarpRow = 32;  // longer rows are expanded by the whole warp

struct ClArgs {
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col_idx;
    int32_t* dist;         // many sources: row i of source srcs[i] at dist + i * dist_stride
    int32_t* ovf;          // per cluster: 3 overflow lists of n entries (frontier of level L: list L % 3)
    unsigned* ovf_n;       // per cluster: their counts (4 per cluster)
    const int32_t* srcs;   // device, many sources (null: the single source src)
    unsigned* next;        // many sources: the next index into srcs to take (zero at launch)
    long long dist_stride;
    int32_t k;
    const int* status;     // sticky status of the graph's control block
    dawn_sssp_stats* stats;
    int32_t n;
    int32_t nwords;
    int32_t src;
    int32_t S;             // bitmap words held by each CTA
    int32_t qcap;          // entries of each shared-memory frontier list
};

struct ClShared {
    int qn[2];             // entries appended to this CTA's list at levels of each parity (own + spill)
    int claims[2];         // vertices this CTA claimed at levels of each parity
    int cnt[2][16];        // every CTA's claims of the level, posted by the CTAs themselves
    int quit;
    int task;              // many sources: the index of the source the cluster runs now
    long long edges[kClThreads / 32];
};

// Append x to the frontier list of CTA `owner` (this CTA or a remote one):
// its shared list while it has room, else the level's global overflow list.
__device__ __forceinline__ void cl_append(cg::cluster_group& cluster, unsigned owner, unsigned rank, int x,
                                          int* s_next, int* s_qn, int32_t* ovf_next, unsigned* ovf_next_n, int qcap) {
    int* qn = owner == rank ? s_qn : cluster.map_shared_rank(s_qn, owner);
    const int slot = atomicAdd(qn, 1);
    if (slot < qcap) {
        int* list = owner == rank ? s_next : cluster.map_shared_rank(s_next, owner);
        list[slot] = x;
    } else {
        ovf_next[atomicAdd(ovf_next_n, 1u)] = x;
    }
}

__global__ void __launch_bounds__(kClThreads, 1) cluster_sssp_kernel(ClArgs a) {
    extern __shared__ __align__(16) uint32_t cl_dyn[];
    __shared__ ClShared sh;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const unsigned C = cluster.num_blocks();
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int S = a.S;
    uint32_t* s_bm = cl_dyn;                                   // S words
    int* s_list[2] = {reinterpret_cast<int*>(cl_dyn + S), reinterpret_cast<int*>(cl_dyn + S) + a.qcap};
    // this cluster's overflow lists and counts
    const unsigned cid = blockIdx.x / C;
    int32_t* const ovf = a.ovf + (long long)cid * 3 * a.n;
    unsigned* const ovf_n = a.ovf_n + 4 * cid;

  for (;;) {  // one source per pass: the single source, or the next of srcs
    int32_t src = a.src;
    int32_t* dist = a.dist;
    dawn_sssp_stats* stats = a.stats;
    // CTA 0 of the cluster takes the next source and reads the sticky status
    // (an earlier failure on this graph leaves every later call idle), and
    // posts both into every CTA of the cluster, so all decide alike
    if (rank == 0 && threadIdx.x == 0) {
        const int t = a.srcs ? (int)atomicAdd(a.next, 1u) : 0;
        const int q = *(volatile const int*)a.status != DEV_OK;
        for (unsigned r = 0; r < C; ++r) {
            *cluster.map_shared_rank(&sh.task, r) = t;
            *cluster.map_shared_rank(&sh.quit, r) = q;
        }
    }
    cluster.sync();
    if (sh.quit) return;
    if (a.srcs) {
        const int t = sh.task;
        if (t >= a.k) break;
        src = __ldg(a.srcs + t);
        dist = a.dist + (long long)t * a.dist_stride;
        stats = a.stats ? a.stats + t : nullptr;
    }

    // ---- init: bitmap slice 0, distances -1 (each CTA its share), source
    for (int i = threadIdx.x; i < S; i += kClThreads) s_bm[i] = 0u;
    const long long chunk = ((long long)a.n + C - 1) / C;
    const long long lo = (long long)rank * chunk, hi = min((long long)a.n, lo + chunk);
    for (long long v = lo + threadIdx.x; v < hi; v += kClThreads) dist[v] = -1;
    if (threadIdx.x == 0) {
        sh.qn[0] = sh.qn[1] = 0;
        sh.claims[0] = sh.claims[1] = 0;
        if (rank == 0) ovf_n[0] = ovf_n[1] = ovf_n[2] = 0u;
    }
    __syncthreads();
    const int sw = src >> 5;
    const unsigned sowner = (unsigned)(sw / S);
    if (threadIdx.x == 0 && rank == sowner) {
        s_bm[sw - (int)sowner * S] = 1u << (src & 31);
        s_list[0][0] = src;
        sh.qn[0] = 1;
    }
    if (threadIdx.x == 0 && src >= lo && src < hi) dist[src] = 0;
    long long edges = 0;
    long long reached = 1;
    int levels = 0;
    cluster.sync();

    for (int level = 1;; ++level) {
        const int pc = (level - 1) & 1, pn = level & 1;
        // this CTA's frontier: the vertices of its slice found at the last level
        const int qn_all = sh.qn[pc];
        const int own = min(qn_all, a.qcap);
        // plus its share of the frontier that spilled to the overflow list
        const int32_t* ovf_cur = ovf + (long long)((level - 1) % 3) * a.n;
        const unsigned on = __ldcg(ovf_n + (level - 1) % 3);
        const long long olo = (long long)on * rank / C, ohi = (long long)on * (rank + 1) / C;
        int32_t* ovf_next = ovf + (long long)(level % 3) * a.n;
        unsigned* ovf_next_n = ovf_n + level % 3;
        const int items = own + (int)(ohi - olo);
        __syncthreads();  // every thread has read this list's count
        if (threadIdx.x == 0) {
            sh.qn[pc] = 0;      // appended to again at the next level, after the barrier
            sh.claims[pc] = 0;
            if (rank == 0) ovf_n[(level + 1) % 3] = 0u;  // used from the next level on
        }
        int my_claims = 0;
        // one frontier vertex per thread and round; the loop bound is the same for the whole warp
        for (int base = threadIdx.x & ~31; base < items; base += kClThreads) {
            const int i = base + lane;
            const bool has = i < items;
            int u = 0, rb = 0, re = 0;
            if (has) {
                u = i < own ? s_list[pc][i] : __ldcg(ovf_cur + olo + (i - own));
                rb = __ldg(a.row_ptr + u);
                re = __ldg(a.row_ptr + u + 1);
                edges += re - rb;
            }
            const bool wide = re - rb > kClWarpRow;
            const int deg = (has && !wide) ? re - rb : 0;
            const int dmax = (int)__reduce_max_sync(kFull, (unsigned)deg);
            // short rows: the thread's own arcs, four at a time, the warp in step
            for (int d0 = 0; d0 < dmax; d0 += 4) {
                int x[4];
                bool won[4];
                unsigned owner[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = d0 + q < deg ? __ldg(a.col_idx + rb + d0 + q) : -1;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    won[q] = false;
                    owner[q] = 0u;
                    if (x[q] < 0) continue;
                    const int w = x[q] >> 5;
                    owner[q] = (unsigned)(w / S);
                    const uint32_t bit = 1u << (x[q] & 31);
                    if (owner[q] == rank) {
                        won[q] = (atomicOr(s_bm + (w - (int)rank * S), bit) & bit) == 0u;
                    } else {
                        uint32_t* word = cluster.map_shared_rank(s_bm, owner[q]) + (w - (int)owner[q] * S);
                        won[q] = (*(volatile uint32_t*)word & bit) == 0u && (atomicOr(word, bit) & bit) == 0u;
                    }
                }
                // local appends of all four arcs: one shared reservation per warp
                unsigned lb[4];
                int ltot = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (won[q]) dist[x[q]] = level;
                    my_claims += won[q];
                    lb[q] = __ballot_sync(kFull, won[q] && owner[q] == rank);
                    ltot += __popc(lb[q]);
                }
                if (ltot) {
                    int slot0 = 0;
                    if (lane == 0) slot0 = atomicAdd(&sh.qn[pn], ltot);
                    slot0 = __shfl_sync(kFull, slot0, 0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if ((lb[q] >> lane) & 1u) {
                            const int slot = slot0 + __popc(lb[q] & ((1u << lane) - 1u));
                            if (slot < a.qcap) s_list[pn][slot] = x[q];
                            else ovf_next[atomicAdd(ovf_next_n, 1u)] = x[q];
                        }
                        slot0 += __popc(lb[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (won[q] && owner[q] != rank)
                        cl_append(cluster, owner[q], rank, x[q], s_list[pn], &sh.qn[pn], ovf_next, ovf_next_n, a.qcap);
            }
            unsigned wl = __ballot_sync(kFull, has && wide);
            while (wl) {  // long rows: the whole warp, one arc per thread
                const int sl = __ffs(wl) - 1;
                wl &= wl - 1;
                const int jb = __shfl_sync(kFull, rb, sl);
                const int je = __shfl_sync(kFull, re, sl);
                for (int j = jb + lane; j < je; j += 32) {
                    const int x = __ldg(a.col_idx + j);
                    const int w = x >> 5;
                    const unsigned ow = (unsigned)(w / S);
                    const uint32_t bit = 1u << (x & 31);
                    uint32_t* word = (ow == rank ? s_bm : cluster.map_shared_rank(s_bm, ow)) + (w - (int)ow * S);
                    if ((atomicOr(word, bit) & bit) == 0u) {
                        dist[x] = level;
                        ++my_claims;
                        cl_append(cluster, ow, rank, x, s_list[pn], &sh.qn[pn], ovf_next, ovf_next_n, a.qcap);
                    }
                }
            }
        }
        // this CTA's claims, posted into every CTA's shared memory before the barrier
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) my_claims += __shfl_xor_sync(kFull, my_claims, o);
        if (lane == 0 && my_claims) atomicAdd(&sh.claims[pn], my_claims);
        __syncthreads();
        if (threadIdx.x < C) *cluster.map_shared_rank(&sh.cnt[pn][rank], threadIdx.x) = sh.claims[pn];
        cluster.sync();
        int total = 0;
        for (unsigned r = 0; r < C; ++r) total += sh.cnt[pn][r];
        if (total == 0) break;
        reached += total;
        levels = level;
        if (level > a.n) {  // a level that claims a vertex claims a new one: cannot happen
            if (rank == 0 && threadIdx.x == 0) atomicCAS(const_cast<int*>(a.status), DEV_OK, DEV_TIMEOUT);
            break;
        }
    }
    // ---- statistics: E_r summed over the cluster
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) edges += __shfl_xor_sync(kFull, edges, o);
    if (lane == 0) sh.edges[threadIdx.x >> 5] = edges;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long e = 0;
        for (int w = 0; w < kClThreads / 32; ++w) e += sh.edges[w];
        sh.edges[0] = e;
    }
    cluster.sync();  // every CTA's total is in place
    if (rank == 0 && threadIdx.x == 0 && stats) {
        long long e = 0;
        for (unsigned r = 0; r < C; ++r) e += *cluster.map_shared_rank(&sh.edges[0], r);
        dawn_sssp_stats s;
        s.levels = levels;
        s.push_steps = levels + 1;
        s.pull_steps = 0;
        s.reserved = 0;
        s.reached = reached;
        s.edges = e;
        *stats = s;
    }
    cluster.sync();  // no CTA leaves (or starts over) while its shared memory may still be read
    if (!a.srcs) break;
  }
}

}  // namespace

namespace {

// Set up once per graph: the largest cluster (16 CTAs, else 8) whose CTAs can
// hold the bitmap slice and two frontier lists and that the device can place,
// and how many such clusters fit on the device at once.  DAWN_E_INVALID when
// none can.
int cluster_setup(dawn_graph* g) {
    if (g->cl_size != 0) return g->cl_size > 0 ? DAWN_OK : fail(DAWN_E_INVALID, "the cluster engine is not available for this graph");
    g->cl_size = -1;
    int dev_smem = 0;
    DAWN_CUDA_TRY(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
    DAWN_CUDA_TRY(cudaFuncSetAttribute(cluster_sssp_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    // the dynamic shared memory limit belongs to the kernel, not to the graph:
    // raise it once to all the kernel can take, so that graphs set up later
    // never lower it under an earlier graph's launches
    cudaFuncAttributes fa;
    DAWN_CUDA_TRY(cudaFuncGetAttributes(&fa, cluster_sssp_kernel));
    const int dyn_max = dev_smem - (int)fa.sharedSizeBytes;
    DAWN_CUDA_TRY(cudaFuncSetAttribute(cluster_sssp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
    for (int C : {16, 8}) {
        const long long S = ((long long)g->nwords + C - 1) / C;
        const long long room = (long long)dev_smem - (long long)sizeof(ClShared) - 1024 - S * 4;
        const long long qcap = std::min<long long>(8192, room / 8);
        if (qcap < 1024) continue;
        const int smem = (int)(S * 4 + qcap * 8);
        if (smem > dyn_max) continue;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, cluster_sssp_kernel, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters < 1) continue;
        g->cl_size = C;
        g->cl_smem = smem;
        g->cl_qcap = (int)qcap;
        g->cl_active = nclusters;
        return DAWN_OK;
    }
    return fail(DAWN_E_INVALID, "the cluster engine is not available for this graph");
}

// Overflow lists and counts for `clusters` clusters running at once (3n
// entries and 4 counts each), plus the counter of a many-source launch after
// the last cluster's counts.
int cluster_buffers(dawn_graph* g, int clusters) {
    if (g->cl_bufs >= clusters) return DAWN_OK;
    cudaFree(g->cl_ovf);
    cudaFree(g->cl_ovf_n);
    g->cl_ovf = nullptr;
    g->cl_ovf_n = nullptr;
    g->cl_bufs = 0;
    cudaError_t e = cudaMalloc((void**)&g->cl_ovf, sizeof(int32_t) * 3 * (size_t)std::max(g->n, 1) * (size_t)clusters);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->cl_ovf_n, sizeof(unsigned) * (4 * (size_t)clusters + 4));
    if (e != cudaSuccess) {
        cudaFree(g->cl_ovf);
        g->cl_ovf = nullptr;
        return cuda_fail(e, "cluster engine buffers", __FILE__, __LINE__);
    }
    g->cl_bufs = clusters;
    return DAWN_OK;
}

int cluster_run(dawn_graph* g, ClArgs& a, int clusters, cudaStream_t st) {
    a.row_ptr = g->row_ptr;
    a.col_idx = g->col_idx;
    a.ovf = g->cl_ovf;
    a.ovf_n = g->cl_ovf_n;
    a.status = &g->ctl->status;
    a.n = g->n;
    a.nwords = g->nwords;
    a.S = (g->nwords + g->cl_size - 1) / g->cl_size;
    a.qcap = g->cl_qcap;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g->cl_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(g->cl_size * clusters);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = g->cl_smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DAWN_CUDA_TRY(cudaLaunchKernelEx(&cfg, cluster_sssp_kernel, a));
    return DAWN_OK;
}

}  // namespace

int cluster_launch(dawn_graph* g, int32_t src, int32_t* dist_dev, const dawn_sssp_opts* opts,
                   dawn_sssp_stats* stats_dev, cudaStream_t st) {
    if (opts && (opts->mode == DAWN_MODE_PULL || opts->trace))
        return fail(DAWN_E_INVALID, "the cluster engine runs SOVM push only, without a trace");
    int rc = cluster_setup(g);
    if (rc == DAWN_OK) rc = cluster_buffers(g, 1);
    if (rc != DAWN_OK) return rc;
    ClArgs a = {};
    a.dist = dist_dev;
    a.stats = stats_dev;
    a.src = src;
    a.srcs = nullptr;
    a.next = nullptr;
    a.k = 1;
    a.dist_stride = 0;
    return cluster_run(g, a, 1, st);
}

int cluster_launch_many(dawn_graph* g, const int32_t* srcs_dev, int32_t k, int32_t* dist_dev, long long stride,
                        const dawn_sssp_opts* opts, dawn_sssp_stats* stats_dev, cudaStream_t st) {
    if (opts && (opts->mode == DAWN_MODE_PULL || opts->trace))
        return fail(DAWN_E_INVALID, "the cluster engine runs SOVM push only, without a trace");
    int rc = cluster_setup(g);
    if (rc != DAWN_OK) return rc;
    const int clusters = std::max(1, std::min<int>(k, g->cl_active));
    rc = cluster_buffers(g, clusters);
    if (rc != DAWN_OK) return rc;
    ClArgs a = {};
    a.dist = dist_dev;
    a.stats = stats_dev;
    a.src = 0;
    a.srcs = srcs_dev;
    a.next = g->cl_ovf_n + 4 * (size_t)g->cl_bufs;
    a.k = k;
    a.dist_stride = stride;
    DAWN_CUDA_TRY(cudaMemsetAsync(a.next, 0, sizeof(unsigned), st));
    return cluster_run(g, a, clusters, st);
}

}  // namespace dawn
