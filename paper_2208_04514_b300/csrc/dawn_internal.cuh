// Internal declarations of the DAWN CUDA library (sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "dawn.h"

namespace dawn {

// ------------------------------------------------------------------ errors --
// Thread-local message behind dawn_last_error(); every failing call sets it.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define DAWN_CUDA_TRY(call)                                                      \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return ::dawn::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

// True when p is device (or managed) memory of the current device.
bool is_device_ptr(const void* p);

// ---------------------------------------------------------- device status --
// Sticky device-side status word values (0 = fine).
enum DeviceStatus : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,   // a bounded grid-barrier wait expired
    DEV_OVERFLOW = 2,  // an int16 distance would exceed 32767
    DEV_PLANES = 3,    // the sliced batched kernel needs more level planes than it was given
};

// A push level whose queue holds a row longer than this splits its work by
// arcs (a search over the record offsets), not by record index.
constexpr int kEntryArcs = 256;

// One counter slot per level, padded to its own 128-byte line.  Levels use
// slots (step % 3): written during step s, read after the barrier that ends
// step s, reset during step s + 1 (see the level loop in sssp.cu).  Launches
// alternate between two sets of three slots (the barrier counter's parity);
// each launch zeroes the other set for the next one, so a launch finds its
// own slots zero on entry.
struct alignas(128) CtrSlot {
    unsigned long long qpack;  // queue size: entries (high 32 bits) | arcs (low 32 bits)
    unsigned long long nf;     // vertices first reached at this level
    unsigned long long mf;     // sum of their out-degrees
    unsigned long long nc;     // pull levels: vertices still unreached (candidate lists), low 32 bits;
                               // list pulls: vertices their look-ahead showed at the next level, high 32 bits
    unsigned long long lr;     // nonzero when a queued row has more than kEntryArcs arcs; list pulls
                               // (which queue nothing): the out-degree sum of the look-ahead's vertices
                               // (low 32 bits) and how many of them it placed two levels ahead (high 32)
    unsigned long long pad[11];
};

// Arrival counter of the grid barrier, on its own 128-byte line.
struct alignas(128) BarCounter {
    unsigned int count;
    unsigned int pad[31];
};

struct alignas(128) Ctl {
    // Launches alternate between the two counters: a launch counts its
    // barrier arrivals on bar[parity] from zero and zeroes bar[parity ^ 1]
    // for the next launch, so no host-side reset sits between launches.
    BarCounter bar[2];
    int status;                // sticky DeviceStatus
    int pad2[31];
    CtrSlot ctr[2][3];         // [launch parity][step % 3]
};

// Default barrier spin budget in SM clock cycles (~2 s at 2 GHz).
constexpr long long kDefaultSpin = 4000000000LL;

}  // namespace dawn

// ------------------------------------------------------------- the graph --
struct dawn_graph {
    int device = 0;
    int sms = 0;
    int32_t n = 0;
    int64_t m = 0;
    uint32_t flags = 0;
    int32_t nwords = 0;               // ceil(n / 32), bitmap words
    int32_t* row_ptr = nullptr;       // CSR, device
    std::vector<int32_t> row_ptr_host;  // copy of row_ptr: the source row bounds travel as launch arguments
    std::vector<int32_t> csize_host;    // symmetric graphs: size of each vertex's connected component
    int32_t* col_idx = nullptr;
    int32_t* in_ptr = nullptr;        // CSC (== CSR when symmetric), device
    int32_t* in_idx = nullptr;
    uint32_t* excl = nullptr;         // bit v set: v has no in-arc (or v >= n)
    int32_t in_sorted = 0;            // 1: every in-adjacency row is in ascending order
    int32_t* pull_idx = nullptr;      // in-adjacency rows ordered by out-degree, largest first (pull levels)
    int2* first2 = nullptr;           // the first two entries of each pull_idx row (-1 where the row is shorter)
    // single-source work buffers
    uint32_t* vis[2] = {nullptr, nullptr};
    int2* queue[2] = {nullptr, nullptr};        // frontier entries {first arc, arc count}
    int32_t* queue_off[2] = {nullptr, nullptr}; // each entry's arc offset within its level
    int64_t queue_cap = 0;
    int32_t* dist_tmp = nullptr;      // result staging for host outputs
    int32_t* cand[2] = {nullptr, nullptr};  // per-CTA lists of unreached pull candidates
    // cluster engine (set up on first use): CTAs per cluster (0 = not yet, -1 = unavailable),
    // dynamic shared memory per CTA, frontier entries per CTA list, overflow lists + counters
    int cl_size = 0;
    int cl_smem = 0;
    int cl_qcap = 0;
    int cl_active = 0;                // clusters of that size the device holds at once
    int cl_bufs = 0;                  // clusters the overflow buffers below serve
    int32_t* cl_ovf = nullptr;        // per cluster: 3 lists of n entries
    unsigned* cl_ovf_n = nullptr;     // per cluster: their 3 counts (4 slots); then a many-source counter
    void* many_graph = nullptr;       // dawn_sssp_many: last captured CUDA graph of launches (many.cu)
    int64_t cand_cap = 0;             // entries per list
    dawn::Ctl* ctl = nullptr;         // device control block
    dawn_sssp_stats* stats_dev = nullptr;
    dawn_sssp_stats* stats_host = nullptr;  // pinned
    int* status_host = nullptr;              // pinned
    int sssp_blocks_per_sm = 0;       // occupancy of the persistent kernel
    int sssp_smem_bytes = 0;          // dynamic shared memory: the pull levels' bitmap copy
    unsigned sssp_launches = 0;       // picks the barrier counter of the next launch
    dawn_tuning tuning = {0, 0, 0, 0, 0.0, 0.0};  // 0 fields: built-in defaults
    // multi-source work buffers (allocated on first use)
    uint64_t* ms_vis[2] = {nullptr, nullptr};
    uint64_t* ms_acc = nullptr;       // per-vertex OR accumulators of dense batched levels
    int ms_words_cap = 0;             // W capacity of ms_vis (n + 1 rows of 4 words; row n stays zero)
    void* ms_plan = nullptr;          // sliced batched kernel: in-arc rows cut into warp tasks (msbfs.cu)
    uint64_t* ms_nb = nullptr;        // its per-level new bits: ms_nb_levels x (n + 1) x 4 words
    int ms_nb_levels = 0;
    uint64_t* ms_planes = nullptr;    // and bit-sliced levels past those: ms_planes_cap x (n + 1) x 4 words
    int ms_planes_cap = 0;
    int ms_sliced_off = 0;            // 1: a run needed more levels than the sliced kernel holds; use the per-level kernel
    int ms_vis_dirty = 0;             // 1: ms_vis holds words a run left behind (the sliced kernel wants zeros)
    int ms_sliced_w = 0;              // lane words of the last sliced run (its level arrays are laid out by it)
    int ms_harm_deep = 0;             // 1: a harmonic-centrality pass outran the sliced kernel's level arrays
    void* ms_scratch = nullptr;       // per-pass distance block when the caller passes none
    size_t ms_scratch_bytes = 0;
    int32_t* ms_counts = nullptr;     // per-lane per-level new-vertex counts
    size_t ms_counts_cap = 0;
    int ms_blocks_per_sm = 0;
    unsigned ms_launches = 0;         // picks the barrier counter of the next batched launch
    void* weighted = nullptr;         // weights and work buffers of the (min, +) path (weighted.cu)
    int32_t* tree_flag = nullptr;     // tree.cu: 1 when the last tree pass pushes level 2 (set on the device)
};

namespace dawn {
// sssp.cu
int sssp_launch(dawn_graph* g, int32_t src, int32_t* dist_dev, const dawn_sssp_opts* opts,
                dawn_sssp_stats* stats_dev, cudaStream_t stream);
int sssp_occupancy(dawn_graph* g);
// graph.cu
int graph_sync_status(dawn_graph* g, cudaStream_t stream);
// many.cu: release the captured graph of dawn_sssp_many
void many_release(dawn_graph* g);
// msbfs.cu: release the sliced batched kernel's plan and planes
void ms_release(dawn_graph* g);
// weighted.cu: release the weighted path's buffers; zero its control block
// after a failed launch (graph_sync_status)
void weighted_release(dawn_graph* g);
int weighted_reset(dawn_graph* g, cudaStream_t st);
// cluster.cu: one source on a single thread-block cluster; DAWN_E_INVALID when unavailable
int cluster_launch(dawn_graph* g, int32_t src, int32_t* dist_dev, const dawn_sssp_opts* opts,
                   dawn_sssp_stats* stats_dev, cudaStream_t st);
// cluster.cu: k sources (device array) on as many clusters as the device holds
// at once, each taking the next source; row i at dist_dev + i * stride
int cluster_launch_many(dawn_graph* g, const int32_t* srcs_dev, int32_t k, int32_t* dist_dev, long long stride,
                        const dawn_sssp_opts* opts, dawn_sssp_stats* stats_dev, cudaStream_t st);
}  // namespace dawn
