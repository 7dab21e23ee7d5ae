// gz_api.cpp - the C ABI of libgz (declared in include/gz.h): argument checks,
// ownership, device memory, launch configuration and the autotuner cache.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "gz_internal.h"

namespace gz {

namespace {
thread_local char g_err[512] = "";
}

std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_allocs{0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

gz_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? GZ_ENOMEM : GZ_ECUDA;
}

gz_status max_degree(const int64_t* rp, int64_t n, int64_t* out, cudaStream_t s);
gz_status validate_csr(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz,
                       bool symmetric, cudaStream_t s);
gz_status make_plan(int k, const uint8_t* adj, const int32_t* forced_order, gz_plan** out);
gz_status list_schedules(int k, const uint8_t* adj, int32_t* orders, int cap, int* count);

// ------------------------------------------------------------ scratch arena

// One growable device scratch region for the synchronous counting calls.
struct Arena {
    std::mutex mu;
    void* ptr = nullptr;
    uint64_t bytes = 0;
    int device = -1;
    unsigned long long* pinned = nullptr;  // 16 bytes of page-locked memory for count read-backs
};
Arena& arena() {
    static Arena a;
    return a;
}

gz_status arena_reserve(Arena& a, uint64_t bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (a.ptr && a.bytes >= bytes && a.device == dev) return GZ_OK;
    if (a.ptr) {
        cudaDeviceSynchronize();
        cudaFree(a.ptr);
        a.ptr = nullptr;
        a.bytes = 0;
    }
    uint64_t want = bytes < (64ull << 20) ? (64ull << 20) : bytes;
    cudaError_t e = gz_malloc(&a.ptr, want);
    if (e != cudaSuccess) {
        a.ptr = nullptr;
        return cuda_fail(e, "scratch cudaMalloc");
    }
    a.bytes = want;
    a.device = dev;
    return GZ_OK;
}

// ------------------------------------------------------------ autotune cache

// Tuned launch shape and split thresholds per (program, graph, view). Keys use
// the plan's program hash and the graph's process-unique id, so a plan or graph
// freed and another allocated at the same address never inherits an entry.
struct TuneKey {
    uint64_t plan;
    uint64_t graph;
    int ori;
    bool operator<(const TuneKey& o) const {
        return std::tie(plan, graph, ori) < std::tie(o.plan, o.graph, o.ori);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, LaunchCfg>& tune_cache() {
    static std::map<TuneKey, LaunchCfg> m;
    return m;
}
std::atomic<uint64_t> g_graph_ids{1};

bool tuned_cfg(const gz_plan* p, const gz_graph* g, int ori, LaunchCfg* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = tune_cache().find(TuneKey{p->hash, g->id, ori ? 1 : 0});
    if (it == tune_cache().end()) return false;
    *out = it->second;
    return true;
}

void forget_graph(const gz_graph* g) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto& m = tune_cache();
    for (auto it = m.begin(); it != m.end();) it = it->first.graph == g->id ? m.erase(it) : std::next(it);
}

// ------------------------------------------------------------ device setup

// Once per device: the stream-ordered pool the library allocates its per-call
// buffers from keeps freed memory for reuse instead of returning it at every
// synchronisation (the default), so a count's allocations cost no new mappings.
// This sets an attribute of this process's memory pool only.
void device_setup() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

// ------------------------------------------------------------ query preparation

// Picks the view, builds the out-list / unit arrays it needs, and turns a root
// range into a unit (edge) range.
gz_status prepare_query(const gz_plan* p, const gz_graph* gc, int use_orientation, int64_t root_lo,
                        int64_t root_hi, cudaStream_t s, Query& q) {
    device_setup();
    gz_graph* g = const_cast<gz_graph*>(gc);
    if (use_orientation && !g->oriented) {
        set_error("count: use_orientation = 1 needs gz_orient first");
        return GZ_EINVAL;
    }
    GzView* v = use_orientation ? &g->ori : &g->orig;
    gz_status st = build_dag(g, v, s);
    if (st != GZ_OK) return st;
    if (!p->prog.unit_dag) {
        st = build_src(g, v, s);
        if (st != GZ_OK) return st;
    }
    q.prog = &p->prog;
    q.plan = p;
    q.g = g;
    q.view = v;
    if (root_lo < 0) root_lo = 0;
    if (root_hi < 0 || root_hi > g->n) root_hi = g->n;
    q.root_lo = root_lo;
    q.root_hi = root_hi;
    if (root_lo >= root_hi) {
        q.unit_lo = q.unit_hi = 0;
        return GZ_OK;
    }
    const int64_t* urp = p->prog.unit_dag ? v->dag_rp : v->rp;
    if (root_lo == 0 && root_hi == g->n) {
        q.unit_lo = 0;
        q.unit_hi = p->prog.unit_dag ? v->dag_nnz : g->nnz;
        return GZ_OK;
    }
    int64_t ends[2];
    cudaError_t e = cudaMemcpyAsync(&ends[0], urp + root_lo, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], urp + root_hi, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "count: unit range");
    q.unit_lo = ends[0];
    q.unit_hi = ends[1];
    return GZ_OK;
}

// Like prepare_query for the full root range, but never builds anything: the
// views the plan needs must already exist (gz_orient, or one gz_count).
gz_status prepare_check(const gz_plan* p, const gz_graph* g, int use_orientation, Query& q) {
    if (use_orientation && !g->oriented) {
        set_error("count: use_orientation = 1 needs gz_orient first");
        return GZ_EINVAL;
    }
    const GzView* v = use_orientation ? &g->ori : &g->orig;
    if (!v->has_dag || (!p->prog.unit_dag && !v->src)) {
        set_error("count: the graph's views for this plan are not built yet; run gz_orient or one "
                  "gz_count with this plan first");
        return GZ_EINVAL;
    }
    q.prog = &p->prog;
    q.g = g;
    q.view = v;
    q.unit_lo = 0;
    q.unit_hi = p->prog.unit_dag ? v->dag_nnz : g->nnz;
    return GZ_OK;
}

LaunchCfg default_cfg() {
    LaunchCfg c;
    c.block_warps = 8;
    c.chunk = 4;
    return c;
}

// Splits queries into those of the general kernel (with out_slot = their index;
// cliques with out-lists past kCliqueLongOut keep their long roots there) and
// the indices of those the clique kernels take.
void split_kinds(const Query* qs, int nq, std::vector<Query>& gen, std::vector<int>* cliq) {
    for (int i = 0; i < nq; ++i) {
        Query q = qs[i];
        q.out_slot = i;
        if (q.unit_hi <= q.unit_lo) continue;
        if (q.plan && clique_eligible(*q.prog, *q.plan, *q.view)) {
            if (cliq) cliq->push_back(i);
            if (q.view->max_out <= kCliqueLongOut) continue;
            q.min_root_out = kCliqueLongOut + 1;  // roots the bitset kernels leave out
        }
        gen.push_back(q);
    }
}

uint64_t mixed_scratch_bytes(const Query* qs, int nq, const LaunchCfg& cfg) {
    std::vector<Query> gen;
    split_kinds(qs, nq, gen, nullptr);
    uint64_t words = 0;
    for (const Query& q : gen) words = std::max(words, scratch_words_per_warp(*q.prog, *q.g, *q.view));
    return (uint64_t)resident_warps(cfg) * words * sizeof(int32_t);
}

uint64_t mixed_meta_bytes(const Query* qs, int nq) {
    std::vector<Query> gen;
    split_kinds(qs, nq, gen, nullptr);
    return launch_meta_bytes(gen.data(), (int)gen.size());
}

// A small pool of streams per device on which one batch's queries overlap.
constexpr int kPool = 4;
gz_status stream_pool(cudaStream_t** out) {
    static std::mutex mu;
    static std::map<int, std::vector<cudaStream_t>> pools;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto& p = pools[dev];
    if (p.empty()) {
        p.resize(kPool);
        for (auto& st : p) {
            cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                p.clear();
                return cuda_fail(e, "stream pool");
            }
        }
    }
    *out = p.data();
    return GZ_OK;
}

gz_status launch_mixed(const Query* qs, int nq, const LaunchCfg& cfg, cudaStream_t s,
                       unsigned long long* d_counts, int* d_status, unsigned long long* d_work,
                       void* scratch, uint64_t scratch_bytes, void* meta, uint64_t meta_bytes,
                       bool overlap) {
    std::vector<Query> gen;
    std::vector<int> cliq;
    split_kinds(qs, nq, gen, &cliq);
    for (int i : cliq) {
        gz_status st = clique_prepare(*qs[i].view, qs[i].g->n, s);
        if (st != GZ_OK) return st;
    }
    // one query (or one kind) runs on s; a mix of several forks onto the pool so
    // the general kernel and the clique launches overlap on the device
    const int kinds = (int)cliq.size() + (gen.empty() ? 0 : 1);
    cudaStream_t* pool = nullptr;
    if (overlap && kinds > 1 && stream_pool(&pool) != GZ_OK) pool = nullptr;
    std::vector<cudaEvent_t> evs;
    auto fork = [&](int j) -> cudaStream_t {
        if (!pool) return s;
        cudaStream_t t = pool[j % kPool];
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return s;
        cudaEventRecord(ev, s);
        cudaStreamWaitEvent(t, ev, 0);
        evs.push_back(ev);
        return t;
    };
    std::vector<cudaStream_t> used;
    gz_status st = GZ_OK;
    if (!gen.empty()) {
        cudaStream_t t = fork(0);
        used.push_back(t);
        st = count_launch(gen.data(), (int)gen.size(), cfg, t, d_counts, scratch, scratch_bytes, d_status,
                          meta, meta_bytes);
    }
    for (size_t c = 0; c < cliq.size() && st == GZ_OK; ++c) {
        const Query& q = qs[cliq[c]];
        const int64_t lo = q.root_lo < 0 ? 0 : q.root_lo;
        const int64_t hi = (q.root_hi < 0 || q.root_hi > q.g->n) ? q.g->n : q.root_hi;
        cudaStream_t t = fork((int)c + 1);
        used.push_back(t);
        st = clique_launch(q.plan->k, *q.view, q.g->n, lo, hi, cfg.grid_frac, t, d_counts + cliq[c],
                           d_work + kCliqueWork * cliq[c]);
    }
    // join: s waits for every stream used
    for (cudaStream_t t : used) {
        if (t == s) continue;
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, t);
            cudaStreamWaitEvent(s, ev, 0);
            evs.push_back(ev);
        }
    }
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    return st;
}

// Runs nq queries and copies their counts to the host. All device state comes
// from the library's scratch arena (grown when needed, then reused): a single
// general-kernel query runs through count_one_in_region (descriptor as a kernel
// parameter: one memset, the launches, one 16-byte read-back); anything else
// through launch_mixed with the counts, descriptors and scratch in the arena.
gz_status run_queries(const Query* qs, int nq, const LaunchCfg& cfg, cudaStream_t s,
                      uint64_t* out_counts) {
    Arena& a = arena();
    std::lock_guard<std::mutex> lk(a.mu);
    if (nq == 1 && !(qs[0].plan && clique_eligible(*qs[0].prog, *qs[0].plan, *qs[0].view))) {
        const Query& q = qs[0];
        const uint64_t meta = one_meta_bytes(q, true);
        const uint64_t scr = (uint64_t)resident_warps(cfg) * scratch_words_per_warp(*q.prog, *q.g, *q.view) * 4;
        gz_status st = arena_reserve(a, meta + scr);
        if (st != GZ_OK) return st;
        if (!a.pinned && gz_malloc_host(&a.pinned, 2 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            a.pinned = nullptr;  // fall back to a pageable read-back
        }
        return count_one_in_region(q, cfg, s, a.ptr, a.bytes - meta, true, out_counts, a.pinned);
    }
    // arena: counts [nq], status, clique work counters [kCliqueWork nq] | launch metadata | scratch
    const size_t hwords = (size_t)nq + 1 + kCliqueWork * (size_t)nq;
    const uint64_t head = ((sizeof(unsigned long long) * hwords) + 255) & ~255ull;
    const uint64_t meta = (mixed_meta_bytes(qs, nq) + 255) & ~255ull;
    const uint64_t need = head + meta + mixed_scratch_bytes(qs, nq, cfg);
    gz_status st = arena_reserve(a, need);
    if (st != GZ_OK) return st;
    unsigned long long* d = reinterpret_cast<unsigned long long*>(a.ptr);
    char* mp = reinterpret_cast<char*>(a.ptr) + head;
    int* d_status = reinterpret_cast<int*>(d + nq);
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * hwords, s);
    if (e != cudaSuccess) return cuda_fail(e, "memset counts");
    st = launch_mixed(qs, nq, cfg, s, d, d_status, d + nq + 1, mp + meta, a.bytes - head - meta, mp, meta, true);
    std::vector<unsigned long long> h(nq + 1);
    if (st == GZ_OK) {
        e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * (nq + 1), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "count");
    } else {
        cudaStreamSynchronize(s);  // launches already queued must finish before the arena is reused
    }
    if (st != GZ_OK) return st;
    if (*reinterpret_cast<int*>(&h[nq]) != 0) {
        set_error("count: a scratch buffer overflowed (planner capacity bug)");
        return GZ_EOVERFLOW;
    }
    for (int i = 0; i < nq; ++i) out_counts[i] = h[i];
    return GZ_OK;
}

bool check_graph(const gz_graph* g, const char* who) {
    if (!g) {
        set_error("%s: graph is NULL", who);
        return false;
    }
    return true;
}

}  // namespace gz

using namespace gz;

extern "C" {

const char* gz_last_error(void) { return gz::g_err; }
const char* gz_version(void) { return "gz-gb300 0.1 (sm_103a)"; }

uint64_t gz_kernel_launches(void) { return g_launches.load(); }

uint64_t gz_allocations(void) { return g_allocs.load(); }

gz_status gz_load_csr(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t nnz,
                      int device_ptrs, uint32_t flags, void* stream, gz_graph** out) {
    GZ_RANGE("gz_load_csr");
    device_setup();
    if (!out) { set_error("gz_load_csr: out is NULL"); return GZ_EINVAL; }
    *out = nullptr;
    if (n < 0 || nnz < 0 || !row_ptr || (nnz > 0 && !col_idx)) {
        set_error("gz_load_csr: bad sizes or NULL arrays (n = %lld, nnz = %lld)", (long long)n, (long long)nnz);
        return GZ_EINVAL;
    }
    if (n > (int64_t)INT32_MAX - 1 || nnz > ((int64_t)1 << 40)) {
        set_error("gz_load_csr: graph too large for int32 ids");
        return GZ_EOVERFLOW;
    }
    cudaStream_t s = (cudaStream_t)stream;
    gz_graph* g = new (std::nothrow) gz_graph;
    if (!g) { set_error("gz_load_csr: out of host memory"); return GZ_ENOMEM; }
    g->n = n;
    g->nnz = nnz;
    g->id = g_graph_ids.fetch_add(1);
    cudaGetDevice(&g->device);
    cudaError_t e = cudaSuccess;
    if (device_ptrs) {
        g->orig.rp = const_cast<int64_t*>(row_ptr);
        g->orig.col = const_cast<int32_t*>(col_idx);
        g->orig.owned_csr = false;
    } else {
        e = gz_malloc(&g->orig.rp, sizeof(int64_t) * (n + 1));
        if (e == cudaSuccess) e = gz_malloc(&g->orig.col, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        if (e == cudaSuccess) e = cudaMemcpyAsync(g->orig.rp, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && nnz > 0)
            e = cudaMemcpyAsync(g->orig.col, col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            gz_status st = cuda_fail(e, "gz_load_csr: copy");
            gz_graph_destroy(g);
            return st;
        }
    }
    gz_status st = GZ_OK;
    if (flags & (GZ_VALIDATE | GZ_VALIDATE_SYMMETRIC))
        st = validate_csr(g->orig.rp, g->orig.col, n, nnz, (flags & GZ_VALIDATE_SYMMETRIC) != 0, s);
    if (st == GZ_OK) st = max_degree(g->orig.rp, n, &g->max_deg, s);
    if (st != GZ_OK) {
        gz_graph_destroy(g);
        return st;
    }
    *out = g;
    return GZ_OK;
}

gz_status gz_orient(gz_graph* g, void* stream) {
    GZ_RANGE("gz_orient");
    if (!check_graph(g, "gz_orient")) return GZ_EINVAL;
    return gz::orient(g, (cudaStream_t)stream);
}

gz_status gz_graph_info(const gz_graph* g, gz_graph_stats* out) {
    if (!check_graph(g, "gz_graph_info") || !out) return GZ_EINVAL;
    gz_graph* gg = const_cast<gz_graph*>(g);
    gz_status st = build_dag(gg, &gg->orig, 0);
    if (st != GZ_OK) return st;
    cudaStreamSynchronize(0);
    memset(out, 0, sizeof(*out));
    out->n = g->n;
    out->nnz = g->nnz;
    out->max_degree = g->max_deg;
    out->max_out_degree_original = g->orig.max_out;
    out->max_out_degree_oriented = g->oriented ? g->ori.max_out : 0;
    out->oriented = g->oriented ? 1 : 0;
    int64_t b = 0;
    auto view_bytes = [&](const GzView& v, bool csr) {
        int64_t x = 0;
        if (csr && v.rp) x += 8 * (g->n + 1) + 4 * g->nnz;
        if (v.dag_rp) x += 8 * (g->n + 1);
        x += 8 * v.dag_cap;  // dag_col + dag_src
        if (v.src) x += 4 * g->nnz;
        x += 4 * (int64_t)v.heavy_rows_cap;  // cached clique rows
        return x;
    };
    b += view_bytes(g->orig, g->orig.owned_csr);
    b += view_bytes(g->ori, true);
    if (g->new_id) b += 4 * g->n;
    out->device_bytes = b;
    return GZ_OK;
}

gz_status gz_graph_export(const gz_graph* g, int oriented, int64_t* row_ptr, int32_t* col,
                          int32_t* new_id, void* stream) {
    if (!check_graph(g, "gz_graph_export") || !row_ptr || (g->nnz > 0 && !col)) return GZ_EINVAL;
    if (oriented && !g->oriented) {
        set_error("gz_graph_export: graph not oriented");
        return GZ_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const GzView& v = oriented ? g->ori : g->orig;
    cudaError_t e = cudaMemcpyAsync(row_ptr, v.rp, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && g->nnz > 0)
        e = cudaMemcpyAsync(col, v.col, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && oriented && new_id && g->n > 0)
        e = cudaMemcpyAsync(new_id, g->new_id, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "gz_graph_export");
    return GZ_OK;
}

void gz_graph_destroy(gz_graph* g) {
    if (!g) return;
    forget_graph(g);
    auto free_view = [](GzView& v, bool csr) {
        if (csr) { cudaFree(v.rp); cudaFree(v.col); }
        cudaFree(v.dag_rp); cudaFree(v.dag_col); cudaFree(v.dag_src); cudaFree(v.src);
        cudaFree(v.heavy_rows); cudaFree(v.slot_dev);
    };
    cudaDeviceSynchronize();
    free_view(g->orig, g->orig.owned_csr);
    free_view(g->ori, true);
    cudaFree(g->new_id);
    delete g;
}

gz_status gz_pattern_named(const char* name, int* k, uint8_t* adj) {
    if (!name || !k || !adj) { set_error("gz_pattern_named: NULL argument"); return GZ_EINVAL; }
    struct E { int a, b; };
    std::vector<E> edges;
    int kk = 0;
    auto clique = [&](int n) { kk = n; for (int i = 0; i < n; ++i) for (int j = i + 1; j < n; ++j) edges.push_back({i, j}); };
    auto chordal = [&](int n) { clique(n); edges.erase(std::remove_if(edges.begin(), edges.end(), [&](E e) { return e.a == n - 2 && e.b == n - 1; }), edges.end()); };
    auto cyc = [&](int n) { kk = n; for (int i = 0; i < n; ++i) edges.push_back({i, (i + 1) % n}); };
    std::string s(name);
    if (s == "edge") { kk = 2; edges = {{0, 1}}; }
    else if (s == "wedge") { kk = 3; edges = {{0, 1}, {0, 2}}; }
    else if (s == "triangle" || s == "k3") clique(3);
    else if (s == "path4") { kk = 4; edges = {{0, 1}, {1, 2}, {2, 3}}; }
    else if (s == "star3") { kk = 4; edges = {{0, 1}, {0, 2}, {0, 3}}; }
    else if (s == "c4" || s == "rectangle") cyc(4);
    else if (s == "paw" || s == "tailed_triangle") { kk = 4; edges = {{0, 1}, {1, 2}, {0, 2}, {2, 3}}; }
    else if (s == "diamond" || s == "chordal4") chordal(4);
    else if (s == "k4") clique(4);
    else if (s == "c5" || s == "pentagon") cyc(5);
    else if (s == "house") { cyc(4); edges.push_back({0, 4}); edges.push_back({1, 4}); kk = 5; }
    else if (s == "hourglass") { kk = 5; edges = {{0, 1}, {0, 2}, {1, 2}, {0, 3}, {0, 4}, {3, 4}}; }
    else if (s == "chordal5") chordal(5);
    else if (s == "k5") clique(5);
    else if (s == "k6") clique(6);
    else if (s == "chordal6") chordal(6);
    else if (s == "k7") clique(7);
    else if (s == "chordal7") chordal(7);
    else {
        set_error("gz_pattern_named: unknown pattern '%s'", name);
        return GZ_EINVAL;
    }
    *k = kk;
    memset(adj, 0, (size_t)kk * kk);
    for (const E& e : edges) adj[e.a * kk + e.b] = adj[e.b * kk + e.a] = 1;
    return GZ_OK;
}

gz_status gz_plan_create(int k, const uint8_t* adj, uint32_t flags, gz_plan** out) {
    GZ_RANGE("gz_plan_create");
    (void)flags;
    return make_plan(k, adj, nullptr, out);
}

gz_status gz_plan_create_with_order(int k, const uint8_t* adj, const int32_t* order, gz_plan** out) {
    if (!order) { set_error("gz_plan_create_with_order: order is NULL"); return GZ_EINVAL; }
    return make_plan(k, adj, order, out);
}

gz_status gz_plan_info(const gz_plan* p, int* k, int32_t* order, int32_t* bound_parent,
                       uint64_t* aut_size, double* est_cost) {
    if (!p) { set_error("gz_plan_info: plan is NULL"); return GZ_EINVAL; }
    if (k) *k = p->k;
    if (order) memcpy(order, p->order, sizeof(int32_t) * p->k);
    if (bound_parent) memcpy(bound_parent, p->bp, sizeof(int32_t) * p->k);
    if (aut_size) *aut_size = p->aut_size;
    if (est_cost) *est_cost = p->est_cost;
    return GZ_OK;
}

gz_status gz_schedule_times(int k, const uint8_t* adj, const gz_graph* g, int use_orientation,
                            const int64_t* sample_lo, const int64_t* sample_hi, int nsample,
                            void* stream, double cutoff, int32_t* orders, double* est_cost,
                            double* ms, int cap, int* count) {
    GZ_RANGE("gz_schedule_times");
    if (!count || !check_graph(g, "gz_schedule_times") || nsample < 1 || !sample_lo || !sample_hi) {
        set_error("gz_schedule_times: bad arguments");
        return GZ_EINVAL;
    }
    int ns = 0;
    gz_status st = list_schedules(k, adj, nullptr, 0, &ns);
    if (st != GZ_OK) return st;
    *count = ns;
    if (cap < ns || !orders || !est_cost || !ms) {
        if (orders || est_cost || ms) {
            set_error("gz_schedule_times: orders, est_cost and ms need room for %d schedules (cap %d)", ns, cap);
            return GZ_EINVAL;
        }
        return GZ_OK;
    }
    list_schedules(k, adj, orders, ns, &ns);
    // sum over the sample ranges of one synchronous count each; stops early once
    // the total passes limit (then returns a total above limit)
    auto time_plan = [&](const gz_plan* p, double limit, double* out_ms) -> gz_status {
        double total = 0.0;
        for (int i = 0; i < nsample; ++i) {
            gz_count_opts o{};
            o.use_orientation = use_orientation;
            o.root_lo = sample_lo[i];
            o.root_hi = sample_hi[i];
            uint64_t c = 0;
            const auto t0 = std::chrono::steady_clock::now();
            gz_status r = gz_count_ex(p, g, &o, stream, &c);
            if (r != GZ_OK) return r;
            total += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (total > limit) break;
        }
        *out_ms = total;
        return GZ_OK;
    };
    double best = 1e300;
    for (int i = 0; i < ns && st == GZ_OK; ++i) {
        gz_plan* p = nullptr;
        st = make_plan(k, adj, orders + (size_t)i * k, &p);
        if (st != GZ_OK) break;
        est_cost[i] = p->est_cost;
        double t = 0.0;
        if (i == 0) st = time_plan(p, 1e300, &t);  // warm-up: views, scratch, caches
        const double limit = cutoff > 0.0 && best < 1e300 ? cutoff * best : 1e300;
        if (st == GZ_OK) st = time_plan(p, limit, &t);
        gz_plan_destroy(p);
        if (st != GZ_OK) break;
        ms[i] = t > limit ? -1.0 : t;
        if (t <= limit && t < best) best = t;
    }
    return st;
}

gz_status gz_plan_create_measured(int k, const uint8_t* adj, const gz_graph* g,
                                  int use_orientation, const int64_t* sample_lo,
                                  const int64_t* sample_hi, int nsample, void* stream,
                                  gz_plan** out, double* best_ms, double* model_ms) {
    GZ_RANGE("gz_plan_create_measured");
    if (!out) {
        set_error("gz_plan_create_measured: out is NULL");
        return GZ_EINVAL;
    }
    *out = nullptr;
    int ns = 0;
    gz_status st = gz_schedule_times(k, adj, g, use_orientation, sample_lo, sample_hi, nsample,
                                     stream, 0.0, nullptr, nullptr, nullptr, 0, &ns);
    if (st != GZ_OK) return st;
    std::vector<int32_t> orders((size_t)ns * k);
    std::vector<double> cost(ns), ms(ns);
    st = gz_schedule_times(k, adj, g, use_orientation, sample_lo, sample_hi, nsample, stream, 4.0,
                           orders.data(), cost.data(), ms.data(), ns, &ns);
    if (st != GZ_OK) return st;
    gz_plan* model = nullptr;
    st = make_plan(k, adj, nullptr, &model);
    if (st != GZ_OK) return st;
    int besti = -1, modeli = -1;
    for (int i = 0; i < ns; ++i) {
        if (memcmp(orders.data() + (size_t)i * k, model->order, sizeof(int32_t) * k) == 0) modeli = i;
        if (ms[i] >= 0.0 && (besti < 0 || ms[i] < ms[besti])) besti = i;
    }
    gz_plan_destroy(model);
    st = make_plan(k, adj, orders.data() + (size_t)besti * k, out);
    if (st != GZ_OK) return st;
    if (best_ms) *best_ms = ms[besti];
    if (model_ms) *model_ms = modeli >= 0 ? ms[modeli] : -1.0;
    return GZ_OK;
}

gz_status gz_plan_schedules(int k, const uint8_t* adj, int32_t* orders, int cap, int* count) {
    return list_schedules(k, adj, orders, cap, count);
}

gz_status gz_plan_describe(const gz_plan* p, char* buf, int cap) {
    if (!p || !buf || cap <= 0) { set_error("gz_plan_describe: bad arguments"); return GZ_EINVAL; }
    const GzProg& g = p->prog;
    std::string s = "unit dag=" + std::to_string(g.unit_dag) + " flat=" + std::to_string(g.flat) + "\n";
    for (int i = 0; i < g.nops; ++i) {
        const GzOp& o = g.ops[i];
        char line[256];
        snprintf(line, sizeof(line),
                 "op level=%d dst=%d left_buf=%d left_pos=%d left_dag=%d left_iter=%d bound=%d excl=%d rights=",
                 o.level, o.dst, o.left_buf, o.left_pos, o.left_dag, o.left_iter, o.bound_pos, o.excl_mask);
        s += line;
        for (int r = 0; r < o.nright; ++r) {
            snprintf(line, sizeof(line), "%s%d:%d:%d", r ? "," : "", o.right_pos[r], o.right_sub[r], o.right_dag[r]);
            s += line;
        }
        s += "\n";
    }
    for (int d = 2; d <= g.k - 2; ++d) {
        char line[160];
        snprintf(line, sizeof(line), "cand d=%d buf=%d pos=%d bound=%d dag=%d excl=%d\n", d, g.cand_buf[d],
                 g.cand_pos[d], g.cand_bound[d], g.cand_dag[d], g.cand_excl[d]);
        s += line;
    }
    for (int b = 0; b < g.nbuf; ++b) s += "buf " + std::to_string(b) + " dag=" + std::to_string(g.buf_dag[b]) + "\n";
    snprintf(buf, (size_t)cap, "%s", s.c_str());
    return GZ_OK;
}

void gz_plan_destroy(gz_plan* p) {
    delete p;  // tuned entries are keyed by the program, which other plans may share
}

gz_status gz_count_ex(const gz_plan* p, const gz_graph* g, const gz_count_opts* opts, void* stream,
                      uint64_t* out_count) {
    GZ_RANGE("gz_count");
    if (!p || !check_graph(g, "gz_count") || !out_count) {
        if (!p) set_error("gz_count: plan is NULL");
        if (!out_count) set_error("gz_count: out_count is NULL");
        return GZ_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    gz_count_opts o{};
    o.root_hi = -1;
    if (opts) o = *opts;
    Query q{};
    gz_status st = prepare_query(p, g, o.use_orientation, o.root_lo, o.root_hi, s, q);
    if (st != GZ_OK) return st;
    LaunchCfg cfg = default_cfg();
    tuned_cfg(p, g, o.use_orientation, &cfg);
    if (o.block_warps > 0) cfg.block_warps = std::min(8, o.block_warps);
    if (o.chunk > 0) cfg.chunk = o.chunk;
    if (o.split_min > 0) cfg.split_min = o.split_min;
    if (o.split_chunk > 0) cfg.split_chunk = o.split_chunk;
    *out_count = 0;
    if (q.unit_hi <= q.unit_lo) return GZ_OK;
    return run_queries(&q, 1, cfg, s, out_count);
}

gz_status gz_count(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream,
                   uint64_t* out_count) {
    gz_count_opts o{};
    o.use_orientation = use_orientation;
    o.root_hi = -1;
    return gz_count_ex(p, g, &o, stream, out_count);
}

gz_status gz_prepare(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream) {
    GZ_RANGE("gz_prepare");
    if (!p || !check_graph(g, "gz_prepare")) {
        if (!p) set_error("gz_prepare: plan is NULL");
        return GZ_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Query q{};
    gz_status st = prepare_query(p, g, use_orientation, 0, -1, s, q);
    if (st != GZ_OK) return st;
    if (clique_eligible(*q.prog, *p, *q.view) && q.view->max_out <= kCliqueLongOut)
        st = clique_prepare(*q.view, g->n, s);
    if (st != GZ_OK) return st;
    const cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? GZ_OK : cuda_fail(e, "gz_prepare");
}

gz_status gz_scratch_bytes(const gz_plan* p, const gz_graph* g, int use_orientation, uint64_t* bytes) {
    if (!p || !check_graph(g, "gz_scratch_bytes") || !bytes) return GZ_EINVAL;
    if (use_orientation && !g->oriented) { set_error("gz_scratch_bytes: graph not oriented"); return GZ_EINVAL; }
    gz_graph* gg = const_cast<gz_graph*>(g);
    GzView* v = use_orientation ? &gg->ori : &gg->orig;
    gz_status st = build_dag(gg, v, 0);
    if (st != GZ_OK) return st;
    *bytes = (uint64_t)resident_warps(default_cfg()) * scratch_words_per_warp(p->prog, *g, *v) * 4;
    return GZ_OK;
}

static gz_status count_batch(const char* who, const gz_plan* const* plans, const gz_graph* const* graphs,
                             const int* use_orientation, const int64_t* root_lo, const int64_t* root_hi,
                             int nq, void* stream, uint64_t* out_counts) {
    if (nq < 0 || (nq > 0 && (!plans || !graphs || !out_counts))) {
        set_error("%s: bad arguments", who);
        return GZ_EINVAL;
    }
    if (nq == 0) return GZ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Query> qs(nq);
    for (int i = 0; i < nq; ++i) {
        if (!plans[i] || !graphs[i]) { set_error("%s: NULL plan or graph at %d", who, i); return GZ_EINVAL; }
        gz_status st = prepare_query(plans[i], graphs[i], use_orientation ? use_orientation[i] : 0,
                                     root_lo ? root_lo[i] : 0, root_hi ? root_hi[i] : -1, s, qs[i]);
        if (st != GZ_OK) return st;
    }
    // heaviest queries first (largest unit count x depth), so their tails start early
    std::vector<int> idx(nq);
    for (int i = 0; i < nq; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        double wa = (double)(qs[a].unit_hi - qs[a].unit_lo) * qs[a].prog->k;
        double wb = (double)(qs[b].unit_hi - qs[b].unit_lo) * qs[b].prog->k;
        return wa > wb;
    });
    std::vector<Query> sorted(nq);
    for (int i = 0; i < nq; ++i) sorted[i] = qs[idx[i]];
    // tuned queries keep their own split thresholds; the launch takes the warps
    // per CTA and units per pop tuned for the heaviest tuned query
    LaunchCfg cfg = default_cfg();
    bool shape = false;
    for (int i = 0; i < nq; ++i) {
        LaunchCfg t;
        const int j = idx[i];
        if (!tuned_cfg(plans[j], graphs[j], use_orientation ? use_orientation[j] : 0, &t)) continue;
        sorted[i].split_min = t.split_min;
        sorted[i].split_chunk = t.split_chunk;
        if (!shape) {
            cfg.block_warps = t.block_warps;
            cfg.chunk = t.chunk;
            shape = true;
        }
    }
    std::vector<uint64_t> res(nq, 0);
    gz_status st = run_queries(sorted.data(), nq, cfg, s, res.data());
    if (st != GZ_OK) return st;
    for (int i = 0; i < nq; ++i) out_counts[idx[i]] = res[i];
    return GZ_OK;
}

gz_status gz_count_batch(const gz_plan* const* plans, const gz_graph* const* graphs,
                         const int* use_orientation, int nq, void* stream, uint64_t* out_counts) {
    GZ_RANGE("gz_count_batch");
    return count_batch("gz_count_batch", plans, graphs, use_orientation, nullptr, nullptr, nq, stream,
                       out_counts);
}

gz_status gz_count_batch_ranges(const gz_plan* const* plans, const gz_graph* const* graphs,
                                const int* use_orientation, const int64_t* root_lo,
                                const int64_t* root_hi, int nq, void* stream, uint64_t* out_counts) {
    GZ_RANGE("gz_count_batch_ranges");
    if (nq > 0 && (!root_lo || !root_hi)) {
        set_error("gz_count_batch_ranges: NULL root range arrays");
        return GZ_EINVAL;
    }
    return count_batch("gz_count_batch_ranges", plans, graphs, use_orientation, root_lo, root_hi, nq, stream,
                       out_counts);
}

gz_status gz_count_merged(const gz_plan* const* plans, int np, const gz_graph* g, int use_orientation,
                          void* stream, uint64_t* out_counts) {
    GZ_RANGE("gz_count_merged");
    if (np < 0 || (np > 0 && (!plans || !out_counts)) || !check_graph(g, "gz_count_merged")) {
        set_error("gz_count_merged: bad arguments");
        return GZ_EINVAL;
    }
    if (np == 0) return GZ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Query> qs(np);
    for (int i = 0; i < np; ++i) {
        if (!plans[i]) { set_error("gz_count_merged: NULL plan at %d", i); return GZ_EINVAL; }
        gz_status st = prepare_query(plans[i], g, use_orientation, 0, -1, s, qs[i]);
        if (st != GZ_OK) return st;
    }
    // oriented cliques keep the bitset kernels; the other plans form merged programs
    std::vector<int> gen_idx, cliq_idx;
    std::vector<Query> cliq;
    for (int i = 0; i < np; ++i) {
        if (qs[i].unit_hi <= qs[i].unit_lo) continue;
        if (clique_eligible(*qs[i].prog, *qs[i].plan, *qs[i].view) && qs[i].view->max_out <= kCliqueLongOut) {
            cliq.push_back(qs[i]);
            cliq_idx.push_back(i);
        } else {
            gen_idx.push_back(i);
        }
    }
    // oriented K4 and K5 on one view: one fused clique pass (the K4 loops are a
    // prefix of the K5 loops, so the K5 walk forms every K4 candidate set),
    // placed after the other clique queries
    bool fuse45 = false;
    {
        int f4 = -1, f5 = -1;
        for (size_t c = 0; c < cliq.size(); ++c) {
            if (cliq[c].plan->k == 4 && f4 < 0) f4 = (int)c;
            if (cliq[c].plan->k == 5 && f5 < 0) f5 = (int)c;
        }
        if (f4 >= 0 && f5 >= 0 && cliq[f4].view == cliq[f5].view && clique45_fusable(*cliq[f5].view)) {
            std::vector<Query> q2;
            std::vector<int> i2;
            for (size_t c = 0; c < cliq.size(); ++c)
                if ((int)c != f4 && (int)c != f5) {
                    q2.push_back(cliq[c]);
                    i2.push_back(cliq_idx[c]);
                }
            q2.push_back(cliq[f4]);
            i2.push_back(cliq_idx[f4]);
            q2.push_back(cliq[f5]);
            i2.push_back(cliq_idx[f5]);
            cliq.swap(q2);
            cliq_idx.swap(i2);
            fuse45 = true;
        }
    }
    std::vector<GzMerged> groups;
    gz_status st = merge_plans(plans, gen_idx.data(), (int)gen_idx.size(), groups);
    if (st != GZ_OK) return st;
    const GzView* v = use_orientation ? &g->ori : &g->orig;
    const LaunchCfg cfg = default_cfg();
    uint64_t gwords = 0, gmeta = 0;
    for (const GzMerged& m : groups) {
        gwords = std::max(gwords, merged_scratch_words(m, *g, *v));
        gmeta = std::max(gmeta, merged_meta_bytes(m, m.unit_dag ? v->dag_nnz : g->nnz));
    }
    auto a256 = [](uint64_t x) { return (x + 255) & ~255ull; };
    // arena: counts [np], status, clique counts [nc], clique work [kCliqueWork nc] |
    // merged metadata | merged scratch | clique metadata | clique scratch
    const size_t nc = cliq.size();
    const size_t hwords = (size_t)np + 1 + nc + kCliqueWork * nc;
    const uint64_t head = a256(sizeof(unsigned long long) * hwords);
    const uint64_t gscr = a256((uint64_t)resident_warps(cfg) * gwords * sizeof(int32_t));
    const uint64_t cmeta = a256(mixed_meta_bytes(cliq.data(), (int)nc));
    const uint64_t cscr = a256(mixed_scratch_bytes(cliq.data(), (int)nc, cfg));
    Arena& a = arena();
    std::lock_guard<std::mutex> lk(a.mu);
    st = arena_reserve(a, head + a256(gmeta) + gscr + cmeta + cscr);
    if (st != GZ_OK) return st;
    char* base = reinterpret_cast<char*>(a.ptr);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(base);
    int* d_status = reinterpret_cast<int*>(d + np);
    char* gm = base + head;
    char* gs = gm + a256(gmeta);
    char* cm = gs + gscr;
    char* cs = cm + cmeta;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long) * hwords, s);
    if (e != cudaSuccess) return cuda_fail(e, "gz_count_merged: memset");
    // the merged programs on a pool stream, the cliques forked from s beside them
    cudaStream_t* pool = nullptr;
    cudaStream_t t = s;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (!groups.empty() && nc > 0 && stream_pool(&pool) == GZ_OK &&
        cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming) == cudaSuccess) {
        t = pool[kPool - 1];
        cudaEventRecord(ev0, s);
        cudaStreamWaitEvent(t, ev0, 0);
    }
    for (const GzMerged& m : groups) {
        if (st != GZ_OK) break;
        st = count_merged(m, g, v, cfg, t, d, d_status, gs, gscr, gm, gmeta);
    }
    const size_t nc_mixed = fuse45 ? nc - 2 : nc;
    if (st == GZ_OK && nc_mixed > 0)  // clique counts land in their own slots, moved to their plans' below
        st = launch_mixed(cliq.data(), (int)nc_mixed, cfg, s, d + np + 1, d_status, d + np + 1 + nc, cs, cscr, cm,
                          cmeta, true);
    if (st == GZ_OK && fuse45) {  // K4 in slot nc - 2, K5 in slot nc - 1
        const Query& q5 = cliq[nc - 1];
        st = clique_launch45(*q5.view, g->n, 0, g->n, cfg.grid_frac, s, d + np + 1 + (nc - 1),
                             d + np + 1 + (nc - 2), d + np + 1 + nc + kCliqueWork * (nc - 1));
    }
    if (ev1) {
        cudaEventRecord(ev1, t);
        cudaStreamWaitEvent(s, ev1, 0);
    }
    std::vector<unsigned long long> h(hwords);
    if (st == GZ_OK) {
        e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * hwords, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "gz_count_merged");
    } else {
        cudaStreamSynchronize(s);
        if (t != s) cudaStreamSynchronize(t);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (st != GZ_OK) return st;
    if (*reinterpret_cast<int*>(&h[np]) != 0) {
        set_error("gz_count_merged: a scratch buffer overflowed (planner capacity bug)");
        return GZ_EOVERFLOW;
    }
    for (int i = 0; i < np; ++i) out_counts[i] = h[i];
    for (size_t c = 0; c < nc; ++c) out_counts[cliq_idx[c]] = h[np + 1 + c];
    return GZ_OK;
}

gz_status gz_autotune(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream,
                      int* block_warps, int* chunk, int64_t* split_min, int64_t* split_chunk) {
    GZ_RANGE("gz_autotune");
    if (!p || !check_graph(g, "gz_autotune")) return GZ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Query q{};
    gz_status st = prepare_query(p, g, use_orientation, 0, -1, s, q);
    if (st != GZ_OK) return st;
    // device time of one count with cfg (CUDA events on the stream), the median
    // of reps runs after one untimed run
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune: event");
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(cudaGetLastError(), "autotune: event");
    }
    auto timed = [&](const LaunchCfg& c, double* ms) -> gz_status {
        uint64_t cnt = 0;
        gz_status r = run_queries(&q, 1, c, s, &cnt);
        std::vector<double> t;
        for (int rep = 0; rep < 3 && r == GZ_OK; ++rep) {
            cudaEventRecord(ev[0], s);
            r = run_queries(&q, 1, c, s, &cnt);
            cudaEventRecord(ev[1], s);
            cudaEventSynchronize(ev[1]);
            float x = 0.f;
            cudaEventElapsedTime(&x, ev[0], ev[1]);
            t.push_back(x);
        }
        if (r != GZ_OK) return r;
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return GZ_OK;
    };
    // coordinate descent from the defaults: units per queue pop, warps per
    // CTA, then the split pass's thresholds (plans with k >= 4 only)
    LaunchCfg best = default_cfg();
    auto_split(*q.prog, q.unit_hi - q.unit_lo, resident_warps(best), &best.split_min, &best.split_chunk);
    double best_ms = 0.0;
    // oriented cliques run on the clique kernels, which take none of these settings
    const bool clique = clique_eligible(*q.prog, *p, *q.view) && q.view->max_out <= kCliqueLongOut;
    if (q.unit_hi > q.unit_lo && !clique) {
        st = timed(best, &best_ms);
        auto try_values = [&](auto set, std::initializer_list<int64_t> values) {
            for (int64_t v : values) {
                if (st != GZ_OK) return;
                LaunchCfg c = best;
                set(c, v);
                double ms = 0.0;
                st = timed(c, &ms);
                if (st == GZ_OK && ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
        };
        try_values([](LaunchCfg& c, int64_t v) { c.chunk = (int)v; }, {1, 2, 8, 16});
        try_values([](LaunchCfg& c, int64_t v) { c.block_warps = (int)v; }, {4});
        if (p->k >= 4) {
            try_values([](LaunchCfg& c, int64_t v) { c.split_min = v; }, {4, 16, 128, 512, 4096});
            try_values([](LaunchCfg& c, int64_t v) { c.split_chunk = v; }, {1, 8, 64, 256});
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != GZ_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache()[TuneKey{p->hash, g->id, use_orientation ? 1 : 0}] = best;
    }
    if (block_warps) *block_warps = best.block_warps;
    if (chunk) *chunk = best.chunk;
    if (split_min) *split_min = best.split_min;
    if (split_chunk) *split_chunk = best.split_chunk;
    return GZ_OK;
}

}  // extern "C"
