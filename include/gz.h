/*
 * gz.h - C ABI of libgz: exact vertex-induced pattern counting on one GB300
 * (sm_103a), after GraphZero (Mawhirter et al., "GraphZero: Breaking Symmetry
 * for Efficient Graph Mining", arXiv 1911.12877).
 *
 * Pipeline (Sec. 3): a pattern is planned on the host (schedule explorer,
 * Algorithm 4; restrictions, Algorithm 1 reduced by Theorem 2; performance
 * model, Sec. 5.4), the graph is optionally reindexed by decreasing degree on
 * the GPU (orientation, Sec. 6), and the compiled nested loops run on the GPU
 * with bounded set intersections and differences over sorted int32 neighbor
 * lists, ending in one exact uint64 count.
 *
 * Conventions for every entry point:
 *  - Every call returns a gz_status: GZ_OK (0) or a negative code. No call
 *    aborts and no C++ exception crosses the ABI. gz_last_error() returns a
 *    thread-local message for the last failing call of the calling thread.
 *  - "stream" is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    return host results synchronise that stream before returning.
 *  - Graphs: CSR with row_ptr int64[n+1] (row_ptr[0] = 0, row_ptr[n] = nnz,
 *    non-decreasing) and col_idx int32[nnz]; each list strictly increasing
 *    (sorted, no duplicates), no self-loops, symmetric (undirected graph).
 *  - Patterns: k x k uint8 adjacency (row-major, symmetric, zero diagonal,
 *    connected), 2 <= k <= GZ_MAX_K. Matching is vertex-induced (Sec. 2.1:
 *    pattern edges are intersections, absent edges are differences).
 *  - Objects are owned by the library and freed with their *_destroy call.
 *  - Counts are exact uint64; overflow beyond 2^64 - 1 is not detected.
 */
#ifndef GZ_H
#define GZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gz_status;
#define GZ_OK 0
#define GZ_EINVAL (-1)       /* bad argument, malformed CSR or pattern */
#define GZ_ENOMEM (-2)       /* device or host allocation failed */
#define GZ_ECUDA (-3)        /* a CUDA runtime call failed */
#define GZ_ETIMEOUT (-4)     /* a bounded wait ran out */
#define GZ_EUNSUPPORTED (-5) /* e.g. no sm_100-family device */
#define GZ_EOVERFLOW (-6)    /* a size does not fit the library's limits */
#define GZ_EBUSY (-7)        /* resource in use (server full) */

#define GZ_MAX_K 8

typedef struct gz_graph gz_graph;   /* device CSR (+ oriented view), opaque */
typedef struct gz_plan gz_plan;     /* compiled schedule, opaque */
typedef struct gz_server gz_server; /* continuous-batching request loop, opaque */

/* ------------------------------------------------------------------ graphs */

#define GZ_VALIDATE 1u           /* check sortedness, range, self-loops on the GPU */
#define GZ_VALIDATE_SYMMETRIC 2u /* also check u in N(v) <=> v in N(u) */

/*
 * Loads an undirected graph stored as sorted neighbor lists (Sec. 6: lists are
 * sorted integer arrays scanned linearly).
 *  row_ptr, col_idx: the CSR (layout above). device_ptrs = 0: host arrays,
 *    copied to the device (the library owns the copy); device_ptrs = 1: device
 *    arrays borrowed by the graph, which must outlive it and stay unchanged.
 *  n >= 0 vertices, nnz >= 0 entries (2 x edges). flags: GZ_VALIDATE bits.
 *  *out receives the graph. Errors: GZ_EINVAL (bad sizes or a CSR that fails
 *  validation), GZ_ENOMEM, GZ_ECUDA. On error *out is NULL.
 */
gz_status gz_load_csr(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t nnz,
                      int device_ptrs, uint32_t flags, void* stream, gz_graph** out);

/*
 * Orientation (Sec. 6): reindexes vertices so a higher degree gets a smaller id
 * (ties broken by the original id, ascending), relabels and re-sorts every
 * list, and builds the out-list view N'(v) intersect [0, v) as a compact DAG
 * CSR. The original view is kept; counts may use either (use_orientation).
 * Idempotent. Calling it again rewrites the oriented view in place (its device
 * buffers are reused), so it first waits for all device work of the process.
 * Errors: GZ_EINVAL (NULL graph), GZ_ENOMEM, GZ_ECUDA.
 */
gz_status gz_orient(gz_graph* g, void* stream);

typedef struct {
    int64_t n, nnz;
    int64_t max_degree;
    int64_t max_out_degree_original; /* max |N(v) intersect [0, v)|, original ids */
    int64_t max_out_degree_oriented; /* same after reindexing; 0 if not oriented */
    int32_t oriented;
    int64_t device_bytes;            /* device memory held by the graph */
} gz_graph_stats;

gz_status gz_graph_info(const gz_graph* g, gz_graph_stats* out);

/*
 * Copies a view back to host memory: row_ptr int64[n+1], col int32[nnz] of the
 * original (oriented = 0) or reindexed (oriented = 1) graph, and new_id
 * int32[n] (old id -> new id; may be NULL; only for oriented = 1).
 * Errors: GZ_EINVAL (not oriented when oriented = 1), GZ_ECUDA.
 */
gz_status gz_graph_export(const gz_graph* g, int oriented, int64_t* row_ptr, int32_t* col,
                          int32_t* new_id, void* stream);

void gz_graph_destroy(gz_graph* g);

/* ---------------------------------------------------------------- patterns */

/*
 * Adjacency of a named pattern: edge, wedge, triangle, path4, star3, c4, paw
 * (tailed triangle, Sec. 5.1), diamond, k4, c5, house, hourglass, chordal5
 * (K5 minus an edge, "chordal cycle", Sec. 1), k5, k6, chordal6, k7, chordal7.
 * adj must hold GZ_MAX_K * GZ_MAX_K bytes; the first k*k are written.
 * Errors: GZ_EINVAL (unknown name).
 */
gz_status gz_pattern_named(const char* name, int* k, uint8_t* adj);

/* ------------------------------------------------------------------- plans */

#define GZ_PLAN_DEFAULT 0u

/*
 * Plans a pattern: Aut(P) by trying all k! permutations (Sec. 4.2); the
 * distinct schedules by Algorithm 4 (Sec. 5.3); for each, the restrictions of
 * Algorithm 1 reduced to one bound per loop by Theorem 2 and the cost of the
 * Sec. 5.4 performance model; the cheapest schedule (first on ties) is
 * compiled into the nested-loop program the kernels run.
 * Errors: GZ_EINVAL (k out of range, not symmetric, self-loop, disconnected).
 */
gz_status gz_plan_create(int k, const uint8_t* adj, uint32_t flags, gz_plan** out);

/* Same, with the schedule fixed to `order` (labels; must be valid, Sec. 2.1). */
gz_status gz_plan_create_with_order(int k, const uint8_t* adj, const int32_t* order,
                                    gz_plan** out);

/*
 * Plan summary: k; order[k] = schedule (labels); bound_parent[k] = for each
 * schedule position i, the position z whose vertex bounds it from above
 * (id(e_i) < id(e_z), Theorems 1 and 2) or -1; aut_size = |Aut(P)|; est_cost =
 * the performance model's value. Any output pointer may be NULL.
 */
gz_status gz_plan_info(const gz_plan* p, int* k, int32_t* order, int32_t* bound_parent,
                       uint64_t* aut_size, double* est_cost);

/*
 * Algorithm 4: writes up to cap distinct schedules (k labels each) in
 * generation order to orders and their number to *count.
 */
gz_status gz_plan_schedules(int k, const uint8_t* adj, int32_t* orders, int cap, int* count);

/*
 * Measured schedule times, the measured side of the Sec. 5.4 performance model
 * (whose estimates against measured times are Fig. 11): for every distinct
 * schedule of the pattern (Algorithm 4, generation order, k labels each into
 * orders) writes the model's estimated cost (est_cost, as gz_plan_info) and the
 * host wall time in ms of counting the roots of the nsample ranges
 * [sample_lo[i], sample_hi[i]) with it (ms; one synchronous gz_count_ex per
 * range, summed). The first schedule is run once untimed first, to build the
 * views and scratch. With cutoff > 0 a schedule is dropped (ms = -1) once its
 * total passes cutoff x the best complete total so far; cutoff <= 0 times every
 * schedule in full. The root of a schedule is its first pattern vertex, so a
 * range holds a different share of the total work under each schedule:
 * [0, n) compares whole counts; otherwise use ranges spread over the id range.
 * With orders, est_cost and ms all NULL only *count is written. Errors:
 * GZ_EINVAL (bad pattern, graph or ranges; cap below the count), and those of
 * gz_count_ex.
 */
gz_status gz_schedule_times(int k, const uint8_t* adj, const gz_graph* g, int use_orientation,
                            const int64_t* sample_lo, const int64_t* sample_hi, int nsample,
                            void* stream, double cutoff, int32_t* orders, double* est_cost,
                            double* ms, int cap, int* count);

/*
 * Measured schedule selection: plans the schedule with the smallest time in
 * gz_schedule_times (cutoff 4; first on ties) instead of the one the Sec. 5.4
 * model ranks first on a uniform random graph (n = 1000, degree 5). The count
 * does not depend on the schedule, only the time does. *best_ms (optional)
 * receives the chosen schedule's time on the samples, *model_ms (optional)
 * that of the schedule gz_plan_create picks, or -1 if that one was dropped at
 * 4x the best. Errors: as gz_schedule_times.
 */
gz_status gz_plan_create_measured(int k, const uint8_t* adj, const gz_graph* g,
                                  int use_orientation, const int64_t* sample_lo,
                                  const int64_t* sample_hi, int nsample, void* stream,
                                  gz_plan** out, double* best_ms, double* model_ms);

/*
 * Text listing of the compiled nested-loop program (one line per item, NUL
 * terminated, truncated to cap bytes): "unit dag=D flat=F" (F: how the last loop is
 * flattened across the candidates of loop k-2; 0 = not), then per loop t its set
 * operations "op level=t dst=B left_buf=B left_pos=P left_dag=D left_iter=I
 * bound=P excl=M rights=pos:sub:dag,..." and per loop d >= 2 its candidates
 * "cand d=.. buf=.. pos=.. bound=.. dag=.. excl=..", and "buf b dag=D" per
 * scratch buffer. For inspection and tests; the kernels read the binary form.
 */
gz_status gz_plan_describe(const gz_plan* p, char* buf, int cap);

void gz_plan_destroy(gz_plan* p);

/* ---------------------------------------------------------------- counting */

/*
 * Counts the instances of the plan's pattern in the graph (Sec. 4: each
 * instance is found exactly once under the restrictions, Theorem 1), on the
 * original ids (use_orientation = 0) or the reindexed graph (1; requires
 * gz_orient first). The graph stays on the device; *out_count (host) receives
 * the exact count. Scratch is allocated by the library and reused.
 *
 * Oriented k-cliques (4 <= k <= 8) run on the bitset clique kernels: the rows of
 * roots with 33 to 1024 out-neighbours are built once per out-list view and
 * kept on the device until the view is rebuilt (gz_orient) or the graph is
 * destroyed; roots with more than 8192 out-neighbours go to the general kernel
 * in the same call. Every other plan runs on the general kernel, whose first
 * pass hands edges with many loop-2 candidates to a second, split pass.
 * Errors: GZ_EINVAL, GZ_ENOMEM, GZ_ECUDA.
 */
gz_status gz_count(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream,
                   uint64_t* out_count);

typedef struct {
    int use_orientation;
    int64_t root_lo, root_hi; /* only roots (first scheduled vertex) in [lo, hi); hi < 0 = n */
    int block_warps;          /* warps per CTA, 0 = default */
    int chunk;                /* work units per queue pop, 0 = default or autotuned */
    int64_t split_min;        /* loop-2 candidates from which a unit goes to the split pass, 0 = autotuned or automatic */
    int64_t split_chunk;      /* loop-2 candidates per split-pass work item, 0 = autotuned or automatic */
} gz_count_opts;

/*
 * gz_count with options. Roots are vertex ids in the view being counted
 * (reindexed ids when use_orientation = 1). The sum over a partition of the
 * root range equals the full count. Split thresholds left at 0 (and not set by
 * gz_autotune) are chosen per query: a query with fewer than 64 work units per
 * resident warp defers units from 4 loop-2 candidates on in one-candidate work
 * items when each candidate carries degree-sized work (a flattened subtraction
 * loop, or k >= 5), else from 64 candidates in items of 64; wider queries defer
 * from 512 candidates in items of 256. Errors as gz_count.
 */
gz_status gz_count_ex(const gz_plan* p, const gz_graph* g, const gz_count_opts* opts,
                      void* stream, uint64_t* out_count);

/* Size of the static scratch array that gz_count_noalloc works in (32 MiB). */
#define GZ_NOALLOC_SCRATCH_BYTES (32ull << 20)

/*
 * gz_count for callers that cannot allocate device memory when they count. The
 * paper has no counterpart. Typical callers: real-time or latency-bound loops
 * whose rules forbid allocator calls once they have started (an allocation can
 * block on the driver or fail under memory pressure at a bad moment), and host
 * applications whose own memory manager reserves the whole device up front, so
 * that a cudaMalloc by a library inside them fails or fragments their pool.
 *
 * Counts the plan's pattern over the whole graph (use_orientation as in
 * gz_count) with the general enumeration kernel and writes the exact count to
 * *out_count (host). It calls no cudaMalloc, cudaFree or other allocating
 * routine (gz_allocations() does not change): its counters and set-operation
 * scratch live in a static device array of 256 + GZ_NOALLOC_SCRATCH_BYTES bytes
 * that every GPU using the library holds until the process exits. A plan whose
 * per-warp scratch exceeds GZ_NOALLOC_SCRATCH_BYTES gets GZ_EOVERFLOW with a
 * message naming both sizes; smaller ones run on as many warps as the array
 * holds. The graph's views must already exist: call gz_orient
 * (use_orientation = 1) or one gz_count with this plan first, else GZ_EINVAL.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for later
 * calls. After cudaDeviceReset on a device that address is stale, so do not
 * call this entry point on that device again in the same process. Every call
 * shares the array and clears its counters itself; calls whose kernels overlap
 * on the GPU (other streams, other host threads) race on it, so the caller
 * must serialise them. Synchronous on `stream`: the count is read back into
 * host memory before the call returns.
 */
gz_status gz_count_noalloc(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream,
                           uint64_t* out_count);

/*
 * Builds, on `stream`, the device state that counts of this plan on this graph
 * view read and the library caches (no paper counterpart): the out-list view
 * and source arrays the plan's loops use and, for oriented k-cliques, the
 * bitset rows of the roots with 33 to 1024 out-neighbours. A later count then
 * does only the counting. The state lasts until gz_orient rebuilds the view or
 * the graph is destroyed; counting without this call builds it on first use.
 * Synchronous on `stream`. Errors: GZ_EINVAL, GZ_ENOMEM, GZ_ECUDA.
 */
gz_status gz_prepare(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream);

/*
 * Device scratch gz_count needs for this plan and graph (bytes), so callers can
 * budget memory before admitting a query.
 */
gz_status gz_scratch_bytes(const gz_plan* p, const gz_graph* g, int use_orientation,
                           uint64_t* bytes);

/*
 * Batched counting: nq independent (plan, graph, use_orientation[i]) queries in
 * one call (no paper counterpart; the merged multi-pattern program of Sec. 3 is
 * the closest). The non-clique queries share one persistent launch over a device
 * work queue, each with the split thresholds gz_autotune chose for it (else the
 * automatic choice described at gz_count_opts, from the query's own width) and
 * the launch shape tuned for the heaviest tuned query; clique queries take
 * the clique kernels; both kinds overlap on a small per-device stream pool and
 * join `stream` before the call returns.
 * out_counts[nq] (host) receives each query's exact count, identical to gz_count
 * of that query. Errors: GZ_EINVAL, GZ_ENOMEM, GZ_ECUDA.
 */
gz_status gz_count_batch(const gz_plan* const* plans, const gz_graph* const* graphs,
                         const int* use_orientation, int nq, void* stream,
                         uint64_t* out_counts);

/*
 * gz_count_batch over root ranges: query i counts only the instances whose root
 * (first scheduled vertex) lies in [root_lo[i], root_hi[i]), as gz_count_ex
 * does (root_lo < 0 is 0; root_hi < 0 or > n is n; an empty range counts 0).
 * The ranges of one (plan, graph) partition its count, so disjoint ranges of a
 * heavy query spread over one launch. root_lo and root_hi are host arrays of nq
 * entries. Errors: as gz_count_batch; GZ_EINVAL for NULL range arrays.
 */
gz_status gz_count_batch_ranges(const gz_plan* const* plans, const gz_graph* const* graphs,
                                const int* use_orientation, const int64_t* root_lo,
                                const int64_t* root_hi, int nq, void* stream,
                                uint64_t* out_counts);

/*
 * Autotuner (no paper counterpart): times candidate launch settings of the
 * general kernel for this (plan, graph, view) with CUDA events on `stream`
 * (median of 3 runs each) and keeps the fastest; later gz_count and
 * gz_count_batch calls on the same program, graph and view use it. The search
 * is one pass of coordinate descent from the defaults over the units per queue
 * pop (1..16), the warps per CTA (4 or 8) and, for k >= 4, the split pass's
 * thresholds: the loop-2 candidate count from which a work unit is deferred to
 * the split pass (4..4096) and the candidates per split work item (1..256),
 * starting from the automatic choice described at gz_count_opts.
 * The choices are written to the non-NULL outputs. The count never depends on
 * them. Entries are keyed by the plan's program and a process-unique graph id,
 * and a graph's entries are dropped when it is destroyed.
 * Errors: as gz_count.
 */
gz_status gz_autotune(const gz_plan* p, const gz_graph* g, int use_orientation, void* stream,
                      int* block_warps, int* chunk, int64_t* split_min, int64_t* split_chunk);

/*
 * Merged multi-pattern counting (Sec. 3: with several patterns GraphZero merges
 * their schedules into one mining program; Sec. 7.2 counts motifs that way):
 * the exact count of each of the np plans' patterns in one graph, written to
 * out_counts[np] (host). The plans whose loop-1 candidates come from the same
 * lists (out-lists or whole lists) form one merged program: their loop-1 set
 * operations that build candidate sets are deduplicated, and one kernel walks
 * the edges (e0, e1) once, computing those shared sets once per edge and then
 * running each plan's remaining loops against them; a plan's edges with many
 * loop-2 candidates go to a split pass as in gz_count. Oriented k-cliques
 * (use_orientation = 1) run on the bitset clique kernels beside it; a K4 and a
 * K5 plan together, on a view whose out-lists hold at most 1024 vertices, take
 * one fused clique pass (the K4 loops are a prefix of the K5 loops: each pair's
 * K4 count is the size of the candidate set the K5 walk forms). The counts
 * equal gz_count's. Errors: GZ_EINVAL, GZ_ENOMEM, GZ_ECUDA.
 */
gz_status gz_count_merged(const gz_plan* const* plans, int np, const gz_graph* g, int use_orientation,
                          void* stream, uint64_t* out_counts);

/* ------------------------------------------------------------------ motifs */

#define GZ_MOTIF_MAX_K 7

/*
 * Motif patterns (the workload of the paper's Table 2, Sec. 7.1-7.2): every
 * connected graph on k vertices (2 <= k <= GZ_MOTIF_MAX_K) up to isomorphism,
 * ordered by edge count and then by canonical code; 1, 2, 6, 21, 112 and 853
 * patterns for k = 2..7 (Sec. 7.2 quotes 2 on 3 vertices and 21 on 5; Sec. 1,
 * 112 of size 6 and 853 of size 7). Writes up to cap
 * patterns as k*k uint8 adjacencies (row-major, consecutive) to adjs (may be
 * NULL) and the number of patterns to *count. Errors: GZ_EINVAL (k out of range).
 */
gz_status gz_motif_patterns(int k, uint8_t* adjs, int cap, int* count);

/*
 * Motif counting: the exact vertex-induced count of every pattern of
 * gz_motif_patterns(k), in that order, each planned like gz_plan_create and all
 * counted in one merged program (gz_count_merged). counts must hold the number of patterns
 * (*count receives it; with counts NULL only *count is written).
 * Errors: GZ_EINVAL (k out of range, cap too small), GZ_ENOMEM, GZ_ECUDA.
 */
gz_status gz_count_motifs(const gz_graph* g, int k, int use_orientation, void* stream,
                          uint64_t* counts, int cap, int* count);

/* --------------------------------------------------------------- serving */

typedef struct {
    int max_inflight_launches; /* concurrent launches (streams), >= 1 */
    int max_batch;             /* fast queries per launch */
    uint64_t scratch_budget;   /* device bytes for in-flight scratch, 0 = 4 GiB */
    double heavy_ms;           /* slow-request threshold (ms), 0 = 20, < 0 = none */
    double slow_share;         /* share of the device a slow request's grids take, 0 = 0.75 */
} gz_server_opts;

/*
 * Continuous-batching request loop over device-resident graphs. The loop keeps
 * a moving average of each (plan, graph)'s service time when it runs alone.
 * Fast requests (at most heavy_ms) are admitted as launch slots and scratch
 * memory free up, batched with whatever else is waiting, and run on separate
 * streams so their work overlaps. A slow request (above heavy_ms, or not yet
 * measured) runs alone in its launch, one at a time. When fast requests are
 * waiting or running and no other slow request waits, its grids take
 * slow_share of the resident CTAs: its kernels are persistent, so the rest of
 * the device stays free for the fast batches while it runs; otherwise it takes
 * the whole device.
 */
gz_status gz_server_create(const gz_server_opts* opts, gz_server** out);

/* Submits one query; *ticket identifies it. Errors: GZ_EINVAL, GZ_EBUSY. */
gz_status gz_server_submit(gz_server* s, const gz_plan* p, const gz_graph* g,
                           int use_orientation, int64_t* ticket);

/*
 * Waits up to timeout_ms (< 0: forever) for ticket; on completion writes the
 * count and the latency from submission to completion in nanoseconds.
 * Errors: GZ_ETIMEOUT (not done yet), GZ_EINVAL (unknown ticket).
 */
gz_status gz_server_wait(gz_server* s, int64_t ticket, int64_t timeout_ms, uint64_t* count,
                         int64_t* latency_ns);

/*
 * Replays a request trace in real time: request i (plan_idx[i] into plans,
 * graph_idx[i] into graphs) is submitted at arrival_ns[i] after the call
 * starts. Fills counts[i] and latency_ns[i] (arrival to completion).
 * fifo = 1 runs the plain baseline instead: one whole-graph query per launch, in
 * arrival order, one at a time. stats_out (optional, 4 values): achieved requests/s,
 * max queue depth, launches, wall seconds.
 */
gz_status gz_server_replay(gz_server* s, const gz_plan* const* plans,
                           const gz_graph* const* graphs, const int* use_orientation,
                           int64_t nreq, const int64_t* arrival_ns, const int32_t* plan_idx,
                           const int32_t* graph_idx, int fifo, uint64_t* counts,
                           int64_t* latency_ns, double* stats_out);

void gz_server_destroy(gz_server* s);

/* ------------------------------------------------------------------ misc */

const char* gz_last_error(void);

/* Library version string. */
const char* gz_version(void);

/* Number of CUDA kernels libgz has launched in this process (all streams). */
uint64_t gz_kernel_launches(void);

/*
 * Number of memory allocation calls (cudaMalloc, cudaMallocAsync,
 * cudaMallocHost) libgz has made in this process. Lets a caller check that a
 * path allocated nothing, e.g. around gz_count_noalloc.
 */
uint64_t gz_allocations(void);

#ifdef __cplusplus
}
#endif

#endif /* GZ_H */
