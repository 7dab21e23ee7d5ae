// gz_internal.h - data structures shared by the host planner and the CUDA kernels
// of libgz. Not part of the public C ABI (include/gz.h is).
#pragma once
#include <stdint.h>
#include <atomic>
#include <utility>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/gz.h"

#define GZ_MAXOPS 40
#define GZ_MAXBUF 24
#define GZ_MAXRIGHT 7

// One set operation of the compiled nested loops. It runs right after e_level is
// bound. out = left[<b] filtered by each right list N(e_pos)[<b] (present for an
// intersection, absent for a difference), b = e_bound_pos or +inf (Sec. 6: the
// restriction's vertex id bounds the scan).
struct GzOp {
    int8_t level;      // t: executed once e_t is fixed
    int8_t dst;        // scratch buffer written, or -1: count only (last loop)
    int8_t left_buf;   // scratch buffer of the left operand, or -1: a view of N(e_left_pos)
    int8_t left_pos;   // list owner when left_buf == -1
    int8_t left_dag;   // left view lies inside the owner's out-list (bound <= owner)
    int8_t left_iter;  // left[<b] is exactly the first i_t entries of level t's candidates
    int8_t nright;
    int8_t bound_pos;  // -1 = unbounded
    int8_t right_pos[GZ_MAXRIGHT];
    int8_t right_sub[GZ_MAXRIGHT];  // 0 = intersect, 1 = subtract
    int8_t right_dag[GZ_MAXRIGHT];  // 1 = bounded part lies in the out-list; 2 = whole out-list
    uint8_t excl_mask;              // count ops: positions whose vertex is not counted
};

// Device-side program: the schedule compiled into per-loop operation lists.
struct GzProg {
    int32_t k;
    int32_t nops;
    int32_t nbuf;
    int32_t unit_dag;                 // level-1 candidates are out-lists (bp[1] == 0)
    int32_t flat;                     // last loop flattened: 1 fixed left operand, 2 left = N(e_{k-2}), 0 no
    GzOp ops[GZ_MAXOPS];
    int8_t level_begin[GZ_MAX_K];     // ops[level_begin[t] .. level_end[t]) run at loop t
    int8_t level_end[GZ_MAX_K];
    // candidates of loop d (2 <= d <= k-2); loop 1 candidates come from the work unit
    int8_t cand_buf[GZ_MAX_K];        // buffer, or -1: view of N(e_cand_pos)[<e_cand_bound]
    int8_t cand_pos[GZ_MAX_K];
    int8_t cand_bound[GZ_MAX_K];
    int8_t cand_dag[GZ_MAX_K];
    uint8_t cand_excl[GZ_MAX_K];      // positions whose vertex is skipped
    int8_t buf_dag[GZ_MAXBUF];        // 1: contents bounded by the max out-degree
};

// Host-side plan (opaque gz_plan).
struct gz_plan {
    uint64_t hash;                     // of (k, adj, order): identifies the program for caches
    int k;
    uint8_t adj[GZ_MAX_K * GZ_MAX_K];  // pattern, labels
    int32_t order[GZ_MAX_K];           // schedule (labels)
    int32_t bp[GZ_MAX_K];              // bound parent per schedule position, -1 none
    uint64_t aut_size;
    double est_cost;
    GzProg prog;
};

// CSR view on the device.
struct GzCsr {
    const int64_t* rp;   // [n+1]
    const int32_t* col;  // [nnz]
};

// Device graph (opaque gz_graph).
struct GzView {
    // one id space: the original ids, or the degree-reindexed ones
    int64_t* rp = nullptr;       // full CSR
    int32_t* col = nullptr;
    int64_t* dag_rp = nullptr;   // out-lists: N(v) intersect [0, v)
    int32_t* dag_col = nullptr;
    int32_t* dag_src = nullptr;  // source vertex of each out-list entry
    int32_t* src = nullptr;      // source vertex of each full-CSR entry (built on demand)
    int64_t dag_nnz = 0;
    int64_t dag_cap = 0;         // entries dag_col / dag_src can hold (kept across rebuilds)
    int64_t max_out = 0;
    bool owned_csr = true;
    bool has_dag = false;
    // roots whose out-list is long enough that the clique kernels split them
    // over several CTAs: (root, out-degree) pairs, gathered once per DAG build
    std::vector<std::pair<int32_t, int32_t>> heavy;
    bool heavy_built = false;
    // bitset rows of those roots (out-degree <= kCliqueMaxOut), built once and
    // kept for every later clique count of this view: heavy_off[i] is the word
    // offset of heavy[i]'s rows in heavy_rows (UINT32_MAX: none)
    uint32_t* heavy_rows = nullptr;
    uint64_t heavy_rows_cap = 0;  // words heavy_rows can hold (kept across rebuilds)
    std::vector<uint32_t> heavy_off;
    bool heavy_rows_built = false;  // the build has run for this out-list view
    bool heavy_rows_ok = false;     // ... and left rows in heavy_rows
    // the cached roots as clique-kernel slots (root, 1 << 16, row offset,
    // out-degree), heaviest first: host copy and device copy (kept across rebuilds)
    std::vector<int4> slot_host;
    int4* slot_dev = nullptr;
    int64_t slot_cap = 0;
};

struct gz_graph {
    uint64_t id = 0;       // unique in the process (never reused), for caches
    int64_t n = 0, nnz = 0, max_deg = 0;
    int device = 0;
    GzView orig;
    GzView ori;            // oriented view (after gz_orient)
    int32_t* new_id = nullptr;  // old -> new id
    bool oriented = false;
};

namespace gz {

// NVTX range around one library call (shows up in Nsight timelines; a no-op
// without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GZ_CAT2(a, b) a##b
#define GZ_CAT(a, b) GZ_CAT2(a, b)
#define GZ_RANGE(name) ::gz::NvtxRange GZ_CAT(gz_range_, __LINE__)(name)

// Kernels this library has launched in this process (for launch accounting).
extern std::atomic<unsigned long long> g_launches;
#define GZ_COUNT_LAUNCH() (::gz::g_launches.fetch_add(1, std::memory_order_relaxed))

// Memory allocation calls (device, stream-ordered and pinned host) this library
// has made in this process. Every allocation of the library goes through these
// wrappers, so a caller can check that a path allocated nothing.
extern std::atomic<unsigned long long> g_allocs;
template <typename T>
inline cudaError_t gz_malloc(T** p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
template <typename T>
inline cudaError_t gz_malloc_async(T** p, size_t bytes, cudaStream_t s) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
}
template <typename T>
inline cudaError_t gz_malloc_host(T** p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}

// Raises a kernel's dynamic shared-memory limit on the current device, once per
// device (the attribute is per device; devices past 64 set it on every call).
// `done` is the kernel's own bitmask of devices already set.
template <typename K>
inline cudaError_t smem_attr_once(K* kernel, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

void set_error(const char* fmt, ...);
gz_status cuda_fail(cudaError_t e, const char* what);

// graph side (gz_graph.cu)
gz_status build_dag(gz_graph* g, GzView* v, cudaStream_t s);
gz_status build_src(gz_graph* g, GzView* v, cudaStream_t s);
gz_status orient(gz_graph* g, cudaStream_t s);

// counting side (gz_count.cu)
struct Query {
    const GzProg* prog;   // host pointer to the program
    const gz_graph* g;
    const GzView* view;
    int64_t unit_lo, unit_hi;  // work units (edges of the unit CSR) in this launch
    const gz_plan* plan = nullptr;
    int64_t root_lo = 0, root_hi = -1;  // the roots those units belong to (hi < 0: n)
    int64_t min_root_out = 0;  // > 0: only roots with at least this out-degree
    int out_slot = -1;         // count slot in the launch's count array (-1: its index)
    int64_t split_min = 0;     // split thresholds of this query (0: the launch's)
    int64_t split_chunk = 0;
};
struct LaunchCfg {
    int block_warps = 8;     // warps per CTA
    int chunk = 4;           // work units per queue pop
    int blocks = 0;          // 0 = auto (resident CTAs on every SM)
    int64_t split_min = 0;     // loop-2 candidates from which a unit goes to the split pass (0 = auto_split)
    int64_t split_chunk = 0;   // loop-2 candidates per split-pass work item (0 = auto_split)
    double grid_frac = 1.0;    // < 1: grids take this share of the resident CTAs only
};
uint64_t scratch_words_per_warp(const GzProg& p, const gz_graph& g, const GzView& v);
// Device bytes count_launch needs beside the scratch (descriptors, counters,
// deferred records).
uint64_t launch_meta_bytes(const Query* qs, int nq);
gz_status count_launch(const Query* qs, int nq, const LaunchCfg& cfg, cudaStream_t s,
                       unsigned long long* d_counts, void* scratch, uint64_t scratch_bytes,
                       int* d_status, void* meta, uint64_t meta_bytes);
int resident_warps(const LaunchCfg& cfg);
// Split thresholds of a query with this program and number of work units when
// neither the caller nor the autotuner set them (see gz_count.cu).
void auto_split(const GzProg& p, int64_t units, int warps, int64_t* split_min, int64_t* split_chunk);

// Bytes of counters (queue, count, status) at the start of a count region.
constexpr uint64_t kRegionHeader = 256;
// Bytes of a single-query region before its scratch (counters, and with split
// the deferred records of the second pass).
uint64_t one_meta_bytes(const Query& Q, bool split);
gz_status count_one_in_region(const Query& Q, const LaunchCfg& cfg, cudaStream_t s, void* region,
                              uint64_t scratch_bytes, bool split, uint64_t* out_count,
                              unsigned long long* pinned = nullptr);

// merged programs (gz_plan.cpp builds them, gz_count.cu runs them): several
// plans that share a unit space compiled into one mining program (Sec. 3: one
// program for several patterns). The loop-1 set operations that write buffers
// are deduplicated across the plans into `shared` (buffers [0, shared.nbuf));
// each plan's program keeps its other operations, with its own buffers
// numbered after the shared ones. One warp per unit binds (e0, e1), runs the
// shared operations once, then each plan's remaining loops.
struct GzMerged {
    int unit_dag = 0;
    GzProg shared;                      // level-1 buffer-writing operations only
    std::vector<GzProg> progs;          // per plan, rewritten
    std::vector<const gz_plan*> plans;
    std::vector<int> plan_index;        // each plan's index in the caller's list (count slot)
};
// Groups the plans idx[0..n) by unit space and merges each group (a group is
// split where the merged program would outgrow the kernel's limits).
gz_status merge_plans(const gz_plan* const* plans, const int* idx, int n, std::vector<GzMerged>& out);
// Scratch words per warp and device bytes beside the scratch of one merged launch.
uint64_t merged_scratch_words(const GzMerged& m, const gz_graph& g, const GzView& v);
uint64_t merged_meta_bytes(const GzMerged& m, int64_t units);
// One merged launch (plus its split pass) over all units of view v: plan i of
// the group adds its count to d_counts[m.plan_index[i]]. scratch must hold
// resident_warps(cfg) * merged_scratch_words words; meta merged_meta_bytes.
gz_status count_merged(const GzMerged& m, const gz_graph* g, const GzView* v, const LaunchCfg& cfg,
                       cudaStream_t s, unsigned long long* d_counts, int* d_status, void* scratch,
                       uint64_t scratch_bytes, void* meta, uint64_t meta_bytes);

// clique side (gz_clique.cu): oriented k-cliques as bitsets over the root's out-list
constexpr int kCliqueMaxOut = 1024;   // largest out-list whose rows fit in shared memory
constexpr int kCliqueWork = 3;        // zeroed work counters a clique query needs
constexpr int kCliqueLongOut = 8192;  // largest out-list of the clique kernels (rows in global)
bool clique_eligible(const GzProg& p, const gz_plan& plan, const GzView& v);
// Enqueues nq queries on stream s: oriented cliques on the bitset kernels (their
// roots with out-lists longer than kCliqueLongOut on the general kernel), the rest
// in one persistent general launch. Query i adds its count to d_counts[i];
// d_work holds kCliqueWork zeroed counters per query; scratch as for count_launch; meta
// holds mixed_meta_bytes(qs, nq) bytes for the general launch. With overlap, a
// mix of queries forks onto a per-device stream pool and joins s again (the
// server passes false: its slots already overlap on their own streams).
gz_status launch_mixed(const Query* qs, int nq, const LaunchCfg& cfg, cudaStream_t s,
                       unsigned long long* d_counts, int* d_status, unsigned long long* d_work,
                       void* scratch, uint64_t scratch_bytes, void* meta, uint64_t meta_bytes,
                       bool overlap);
// Scratch and metadata bytes launch_mixed needs for these queries.
uint64_t mixed_scratch_bytes(const Query* qs, int nq, const LaunchCfg& cfg);
uint64_t mixed_meta_bytes(const Query* qs, int nq);
gz_status clique_prepare(const GzView& v, int64_t n, cudaStream_t s);
gz_status clique_launch(int k, const GzView& v, int64_t n, int64_t lo, int64_t hi, double frac, cudaStream_t s,
                        unsigned long long* d_count, unsigned long long* d_work);
// Fused K4 + K5 clique pass (both counts from one walk over the pairs), for
// views whose longest out-list fits the shared-memory row kernels.
bool clique45_fusable(const GzView& v);
gz_status clique_launch45(const GzView& v, int64_t n, int64_t lo, int64_t hi, double frac, cudaStream_t s,
                          unsigned long long* d_count5, unsigned long long* d_count4, unsigned long long* d_work);

}  // namespace gz
