// gz_count.cu - the enumeration kernels: the compiled nested loops of GraphZero
// (Sec. 4) run by one warp per work unit, with bounded set operations on sorted
// int32 neighbor lists (Sec. 6) and an exact uint64 reduction.
//
// Execution model
//  - A work unit is one edge (e0, e1) of the level-1 candidate lists: an
//    out-list entry (e1 < e0) when loop 1 is bounded by loop 0, else a full
//    adjacency entry. Units are popped from a device counter in chunks by a
//    persistent grid (resident CTAs on every SM), which splits skewed roots at
//    edge granularity.
//  - A warp binds e0, e1, runs loop 1's operations, then walks loops 2..k-2 as
//    an explicit DFS. Each set operation streams its left list 32 elements at a
//    time (coalesced), probes every right list by binary search, and either
//    compacts the survivors into the warp's scratch buffer (ballot + popc) or,
//    on the last loop, only counts them. The last loop is flattened across the
//    candidates of the loop before it (fixed operands hashed in shared memory
//    or in warp scratch; subtraction-only shapes counted by inclusion-exclusion).
//  - Edges with many loop-2 candidates are deferred by the first pass and run
//    in chunks of candidates by a second pass (k_enumerate_split).
//  - Counts are per-lane uint64, reduced by warp shuffles and added to the
//    query's slot with one atomic per warp per query. Integer adds are exact and
//    order-independent, so the result is bit-exact whatever the schedule.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "gz_internal.h"

namespace gz {

namespace {

constexpr unsigned kFull = 0xffffffffu;
// Shared memory per warp stays small (6.6 KB): the rest of the SM's unified
// L1/shared storage caches the neighbour lists the binary searches walk.
constexpr int kStageWords = 512;   // per-warp shared staging of a fixed operand (int32)
constexpr int kHashLog2 = 10;
constexpr int kHashSlots = 1 << kHashLog2;  // per-warp open-addressing hash set of that operand
// per warp: staged operand, lane offsets, lengths, list pointers, hash set
constexpr int kWarpSmemWords = kStageWords + 64 + 64 + kHashSlots;

// Per-query descriptor in device memory.
struct KQ {
    GzProg prog;
    const int64_t* rp;
    const int32_t* col;
    const int64_t* drp;
    const int32_t* dcol;
    const int32_t* usrc;   // unit CSR: source of each unit edge
    const int32_t* ucol;   // unit CSR: target of each unit edge
    const int64_t* urp;    // unit CSR rows (position of e1 within e0's list)
    int64_t unit_lo;       // first unit (edge index) of this query
    int64_t unit_begin;    // offset of this query in the launch's unit space
    int64_t unit_count;
    int64_t min_root_out;  // > 0: units whose root has a shorter out-list are skipped
    int32_t out_slot;      // count slot of this query
    int64_t buf_off[GZ_MAXBUF];
    int64_t buf_cap[GZ_MAXBUF];
    int64_t hash_off;      // per-warp hash table for a fixed operand too long for shared memory
    int32_t hash_log2;     // its slot count is 1 << hash_log2 (0: none)
    int64_t split_min;     // loop-2 candidates from which a unit goes to the split pass
    int64_t split_chunk;   // loop-2 candidates per split-pass work item
    int32_t merge_pos;     // merged launches: this plan's position in its group
    uint64_t shared_mask;  // merged launches: the shared loop-1 operations this plan reads
};

constexpr int kGlobalHashLog2 = 17;  // largest per-warp hash table in scratch (slots)

// Per-warp scratch layout of a query: one buffer per compiled set operation
// (max out-degree or max degree ids) and, when the last loop is flattened with
// a fixed left operand that can outgrow the shared-memory hash set, a hash
// table of up to 2^kGlobalHashLog2 slots. Returns the words per warp.
uint64_t scratch_layout(const GzProg& p, const gz_graph& g, const GzView& v, KQ* k) {
    uint64_t off = 0, capmax = 0;
    for (int b = 0; b < p.nbuf; ++b) {
        const uint64_t cap = (uint64_t)(p.buf_dag[b] ? v.max_out : g.max_deg);
        if (k) {
            k->buf_off[b] = (int64_t)off;
            k->buf_cap[b] = (int64_t)cap;
        }
        off += (cap + 31) & ~31ull;
    }
    capmax = (uint64_t)g.max_deg;
    int lg = 0;
    if (p.flat == 1 && capmax > (uint64_t)kStageWords) {
        while ((1ull << lg) < 2 * capmax && lg < kGlobalHashLog2) ++lg;
    }
    if (k) {
        k->hash_off = (int64_t)off;
        k->hash_log2 = lg;
    }
    if (lg) off += 1ull << lg;
    return off;
}

// Splitting of heavy units. A unit whose loop-2 candidate list holds at least
// its query's split_min vertices is not run by the warp that popped it: the
// first pass records it (launch-space unit index, candidate count and the
// query's split_chunk), a one-CTA scan turns the records into chunks of
// split_chunk candidates, and a second pass hands the chunks to warps, each
// recomputing loop 1 and walking its chunk of loop 2. A hub edge then spreads
// over many warps instead of holding one. Both thresholds are per query (the
// autotuner picks them).
struct Deferred {
    int64_t unit;   // launch-space unit index
    int64_t n2;     // loop-2 candidates
    int64_t chunk;  // candidates per split-pass work item
    int64_t plan;   // merged launches: the plan's position in its group
};

struct DeferCtl {
    Deferred* list;              // NULL: no deferral
    unsigned long long* count;   // records written (may exceed cap)
    int64_t cap;
};

// Number of elements of sorted L[0, n) that are < beta (warp-cooperative
// 32-ary search; every lane returns the same value).
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t* __restrict__ L, int64_t n,
                                                    int32_t beta, int lane) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 32) {
        int64_t step = (hi - lo + 31) >> 5;
        int64_t p = lo + (int64_t)lane * step;
        bool less = p < hi && __ldg(L + p) < beta;
        int c = __popc(__ballot_sync(kFull, less));
        if (c == 0) return lo;
        int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
        int64_t nhi = lo + (int64_t)c * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    int64_t p = lo + lane;
    bool less = p < hi && __ldg(L + p) < beta;
    return lo + __popc(__ballot_sync(kFull, less));
}

// Same, for scratch buffers written earlier by this warp (no read-only path).
__device__ __forceinline__ int64_t warp_lower_bound_rw(const int32_t* L, int64_t n, int32_t beta,
                                                       int lane) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 32) {
        int64_t step = (hi - lo + 31) >> 5;
        int64_t p = lo + (int64_t)lane * step;
        bool less = p < hi && L[p] < beta;
        int c = __popc(__ballot_sync(kFull, less));
        if (c == 0) return lo;
        int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
        int64_t nhi = lo + (int64_t)c * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    int64_t p = lo + lane;
    bool less = p < hi && L[p] < beta;
    return lo + __popc(__ballot_sync(kFull, less));
}

// Is x in sorted R[0, n)? (per-lane binary search)
__device__ __forceinline__ bool contains(const int32_t* __restrict__ R, int n, int32_t x) {
    int lo = 0, len = n;
    while (len > 0) {
        int half = len >> 1;
        int32_t v = __ldg(R + lo + half);
        if (v < x) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo < n && __ldg(R + lo) == x;
}

struct ListRef {
    const int32_t* p;
    int64_t n;
};

// N(v), or its out-list part when dag != 0.
__device__ __forceinline__ ListRef adj_list(const KQ& q, int32_t v, int dag) {
    ListRef r;
    if (dag) {
        int64_t b = q.drp[v];
        r.p = q.dcol + b;
        r.n = q.drp[v + 1] - b;
    } else {
        int64_t b = q.rp[v];
        r.p = q.col + b;
        r.n = q.rp[v + 1] - b;
    }
    return r;
}

struct WarpState {
    int32_t emb[GZ_MAX_K];     // bound vertices e_0..e_{k-1}
    int64_t itp[GZ_MAX_K];     // index of e_t within loop t's candidate list
    int64_t blen[GZ_MAXBUF];   // current length of each scratch buffer
};

// Executes one compiled set operation (see GzOp).
__device__ void exec_op(const KQ& q, const GzOp& op, WarpState& ws, int32_t* scratch, int lane,
                        unsigned long long& acc, int* status) {
    const bool bounded = op.bound_pos >= 0;
    const int32_t beta = bounded ? ws.emb[op.bound_pos] : INT_MAX;
    const int32_t* L;
    int64_t nL;
    if (op.left_buf >= 0) {
        L = scratch + q.buf_off[op.left_buf];
        nL = ws.blen[op.left_buf];
        if (op.left_iter) nL = ws.itp[op.level];
        else if (bounded) nL = warp_lower_bound_rw(L, nL, beta, lane);
    } else {
        ListRef r = adj_list(q, ws.emb[op.left_pos], op.left_dag);
        L = r.p;
        nL = r.n;
        if (op.left_iter) nL = ws.itp[op.level];
        else if (bounded && op.left_dag != 2) nL = warp_lower_bound(L, nL, beta, lane);
    }
    ListRef R[GZ_MAXRIGHT];
    const int nr = op.nright;
    for (int r = 0; r < nr; ++r) R[r] = adj_list(q, ws.emb[op.right_pos[r]], op.right_dag[r]);

    const bool count_only = op.dst < 0;
    int32_t* out = count_only ? nullptr : scratch + q.buf_off[op.dst];
    const int64_t cap = count_only ? 0 : q.buf_cap[op.dst];
    int64_t w = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t base = 0; base < nL; base += 32) {
        int64_t idx = base + lane;
        bool keep = idx < nL;
        int32_t x = keep ? L[idx] : 0;
        for (int r = 0; r < nr && keep; ++r) {
            bool f = contains(R[r].p, (int)R[r].n, x);
            keep = f != (op.right_sub[r] != 0);
        }
        if (count_only) {
            if (keep && op.excl_mask) {
                for (int j = 0; j < GZ_MAX_K; ++j)
                    if ((op.excl_mask >> j & 1) && ws.emb[j] == x) keep = false;
            }
            acc += keep ? 1ull : 0ull;
        } else {
            unsigned m = __ballot_sync(kFull, keep);
            int64_t pos = w + __popc(m & lt_mask);
            if (keep) {
                if (pos < cap) out[pos] = x;
                else atomicExch(status, 1);
            }
            w += __popc(m);
        }
    }
    if (!count_only) {
        ws.blen[op.dst] = w < cap ? w : cap;
        __syncwarp();
    }
}

__device__ __forceinline__ void run_level(const KQ& q, int t, WarpState& ws, int32_t* scratch,
                                          int lane, unsigned long long& acc, int* status) {
    const GzProg& P = q.prog;
    for (int i = P.level_begin[t]; i < P.level_end[t]; ++i) exec_op(q, P.ops[i], ws, scratch, lane, acc, status);
}

// Candidate list of loop d (2 <= d <= k-2) once e_{d-1} is bound.
__device__ __forceinline__ ListRef cand_list(const KQ& q, int d, const WarpState& ws,
                                             int32_t* scratch, int lane) {
    const GzProg& P = q.prog;
    ListRef r;
    if (P.cand_buf[d] >= 0) {
        r.p = scratch + q.buf_off[P.cand_buf[d]];
        r.n = ws.blen[P.cand_buf[d]];
    } else {
        r = adj_list(q, ws.emb[P.cand_pos[d]], P.cand_dag[d]);
        if (P.cand_bound[d] >= 0 && P.cand_dag[d] != 2)
            r.n = warp_lower_bound(r.p, r.n, ws.emb[P.cand_bound[d]], lane);
    }
    return r;
}

// Per-lane lower bound in a sorted list: number of elements < beta.
__device__ __forceinline__ int64_t lane_lower_bound(const int32_t* p, int64_t n, int32_t beta) {
    int64_t lo = 0, len = n;
    while (len > 0) {
        int64_t half = len >> 1;
        if (p[lo + half] < beta) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo;
}

// Membership in a sorted array (shared or global memory).
__device__ __forceinline__ bool in_sorted(const int32_t* A, int64_t n, int32_t x) {
    int64_t lo = 0, len = n;
    while (len > 0) {
        int64_t half = len >> 1;
        if (A[lo + half] < x) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo < n && A[lo] == x;
}

__device__ __forceinline__ bool excluded(uint8_t mask, const WarpState& ws, int32_t x) {
    bool ex = false;
    if (mask)
        for (int j = 0; j < GZ_MAX_K; ++j)
            if ((mask >> j & 1) && ws.emb[j] == x) ex = true;
    return ex;
}

// Open-addressing hash set of distinct non-negative ids in shared memory
// (kHashSlots slots, -1 = empty, linear probing). At most kStageWords keys, so
// the load factor stays <= 1/2 and every probe ends at an empty slot.
__device__ __forceinline__ uint32_t hash_slot(int32_t x) {
    return ((uint32_t)x * 0x9E3779B1u) >> (32 - kHashLog2);
}

__device__ __forceinline__ void hash_build(int32_t* H, const int32_t* F, int64_t nF, int lane) {
    for (int i = lane; i < kHashSlots; i += 32) H[i] = -1;
    __syncwarp();
    for (int64_t i = lane; i < nF; i += 32) {
        const int32_t x = F[i];
        uint32_t s = hash_slot(x);
        while (atomicCAS(&H[s], -1, x) != -1) s = (s + 1) & (kHashSlots - 1);
    }
    __syncwarp();
}

// The same open-addressing scheme in the warp's global scratch, 2^lg slots
// (at least twice the keys), for fixed operands longer than kStageWords.
__device__ __forceinline__ void ghash_build(int32_t* H, int lg, const int32_t* F, int64_t nF, int lane) {
    const uint32_t mask = (1u << lg) - 1u;
    for (int64_t i = lane; i <= (int64_t)mask; i += 32) H[i] = -1;
    __syncwarp();
    for (int64_t i = lane; i < nF; i += 32) {
        const int32_t x = F[i];
        uint32_t s = ((uint32_t)x * 0x9E3779B1u) >> (32 - lg);
        while (atomicCAS(&H[s], -1, x) != -1) s = (s + 1) & mask;
    }
    __syncwarp();
}

__device__ __forceinline__ bool ghash_has(const int32_t* H, int lg, int32_t x) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = ((uint32_t)x * 0x9E3779B1u) >> (32 - lg);
    for (;;) {
        const int32_t v = H[s];
        if (v == x) return true;
        if (v < 0) return false;
        s = (s + 1) & mask;
    }
}

__device__ __forceinline__ bool hash_has(const int32_t* H, int32_t x) {
    uint32_t s = hash_slot(x);
    for (;;) {
        const int32_t v = H[s];
        if (v == x) return true;
        if (v < 0) return false;
        s = (s + 1) & (kHashSlots - 1);
    }
}

// The last loop, flattened over every candidate c of loop k-2. The one count
// operation of loop k-2 reads N(c) and otherwise only sets fixed for this call:
//  shape 1: |F[<b_c] op N(c)[<b_c]| with F fixed (the left operand);
//  shape 2: |N(c)[<b_c] filtered by fixed right lists|.
// For each group of 32 candidates and each candidate, the shorter side is
// streamed: (A) N(c)[<b_c], probing F (staged in shared memory when it fits) or
// the fixed right lists; (B) F[<b_c], binary-searching N(c)[<b_c]. Both passes
// are flattened, so lanes stream the concatenated lists of many candidates and
// no lane idles on a short list.
__device__ void last_level_flat(const KQ& q, const GzOp& op, WarpState& ws, ListRef S, int64_t ioff,
                                int32_t* scratch, int32_t* sm, int lane, unsigned long long& acc) {
    const GzProg& P = q.prog;
    const int t = P.k - 2;
    const uint8_t cex = P.cand_excl[t];
    const bool shape2 = P.flat == 2;
    int32_t* offs = sm + kStageWords;
    int32_t* lens = sm + kStageWords + 32;
    const int32_t** rptr = reinterpret_cast<const int32_t**>(sm + kStageWords + 64);
    const int32_t* F = nullptr;
    int64_t nF = 0;
    int32_t* H = sm + kStageWords + 128;
    bool hashed = false;
    int32_t* GH = nullptr;  // global hash table (F too long for H), else NULL
    int glg = 0;
    const bool sub = !shape2 && op.right_sub[0] != 0;
    const bool bounded = op.bound_pos >= 0;
    if (!shape2) {
        if (op.left_buf >= 0) {
            F = scratch + q.buf_off[op.left_buf];
            nF = ws.blen[op.left_buf];
        } else {
            ListRef r = adj_list(q, ws.emb[op.left_pos], op.left_dag);
            F = r.p;
            nF = r.n;
        }
        if (bounded && op.bound_pos != t) nF = warp_lower_bound_rw(F, nF, ws.emb[op.bound_pos], lane);
        if (nF <= kStageWords) {
            for (int64_t i = lane; i < nF; i += 32) sm[i] = F[i];
            __syncwarp();
            F = sm;
            // probes of F are then O(1) hash lookups instead of binary searches
            if (S.n >= 2 && nF >= 16) {
                hash_build(H, F, nF, lane);
                hashed = true;
            }
        } else if (q.hash_log2 && S.n >= 16 && S.n * 64 >= nF && (2 * nF) <= (1ll << q.hash_log2)) {
            // too long for shared memory: a hash table in the warp's scratch,
            // sized to the next power of two >= 2 nF, when enough candidates
            // probe it to pay for filling it
            int lg = 1;
            while ((1ll << lg) < 2 * nF) ++lg;
            GH = scratch + q.hash_off;
            glg = lg;
            ghash_build(GH, lg, F, nF, lane);
            hashed = true;
        }
    }
    const int sdag = shape2 ? op.left_dag : op.right_dag[0];
    // e_t is the candidate c itself and is not stored in ws.emb on this path. A
    // streamed or matched x lies in N(c), so x != c; only the subtraction's
    // exclusion count below has to consider c.
    const uint8_t xm = op.excl_mask & (uint8_t)~(1u << t);
    const bool excl_self = (op.excl_mask >> t) & 1;
    // Shape 2 whose right lists are all subtracted (at most two) under a bound
    // that does not move with c: |L - R0 - R1| with L = N(c)[<b] is counted as
    // |L| - |L & R0| - |L & R1| + |L & R0 & R1| (a set identity), each
    // intersection streaming its shortest list and probing the others, instead
    // of streaming L and probing both. A hub candidate then costs about the
    // length of the fixed lists, not its own degree.
    bool ie = shape2 && op.nright >= 1 && op.nright <= 2 && (!bounded || op.bound_pos != t);
    for (int r = 0; r < op.nright && ie; ++r) ie = op.right_sub[r] != 0;
    ListRef rl[2] = {{nullptr, 0}, {nullptr, 0}};
    if (ie) {
        const int32_t bfix = bounded ? ws.emb[op.bound_pos] : INT_MAX;
        for (int r = 0; r < op.nright; ++r) {
            rl[r] = adj_list(q, ws.emb[op.right_pos[r]], op.right_dag[r]);
            if (bounded && op.right_dag[r] != 2) rl[r].n = warp_lower_bound(rl[r].p, rl[r].n, bfix, lane);
        }
    }
    const int32_t** spt = reinterpret_cast<const int32_t**>(sm);  // shape 2 leaves F's staging free
    int32_t* pmask = sm + 64;
    for (int64_t base = 0; base < S.n; base += 32) {
        const int64_t idx = base + lane;
        bool valid = idx < S.n;
        const int32_t c = valid ? S.p[idx] : 0;
        if (valid && excluded(cex, ws, c)) valid = false;
        const int32_t* R = nullptr;
        int64_t m = 0, Lc = 0;
        int32_t beta = INT_MAX;
        if (valid) {
            ListRef r = adj_list(q, c, sdag);
            R = r.p;
            m = r.n;
            if (bounded) beta = op.bound_pos == t ? c : ws.emb[op.bound_pos];
            if (bounded && sdag != 2) m = lane_lower_bound(R, m, beta);
            if (!shape2) {
                if (bounded && op.bound_pos == t) Lc = op.left_iter ? idx + ioff : lane_lower_bound(F, nF, c);
                else Lc = nF;
                if (Lc == 0) valid = false;  // empty left part: contributes nothing
            }
        }
        if (ie) {
            if (valid) {
                acc += (unsigned long long)m;
                for (int j = 0; j < GZ_MAX_K; ++j)  // excluded vertices the identity would count
                    if (xm >> j & 1) {
                        const int32_t e = ws.emb[j];
                        if (e < beta && in_sorted(R, m, e)) {
                            bool keep = true;
                            for (int r = 0; r < op.nright; ++r) keep = keep && !in_sorted(rl[r].p, rl[r].n, e);
                            if (keep) acc -= 1ull;
                        }
                    }
            }
            const int nterms = op.nright == 2 ? 3 : 1;
            for (int term = 0; term < nterms; ++term) {
                const unsigned set = term == 0 ? 1u : (term == 1 ? 2u : 3u);  // which R_r
                const bool plus = term == 2;
                // stream the shortest of L and the set's lists; probe the others
                // (mask bit 0: L = N(c)[<b], bits 1-2: R0, R1)
                const int32_t* sp = R;
                int64_t sl = m;
                unsigned pm = set << 1;
                for (int r = 0; r < 2; ++r)
                    if ((set >> r & 1) && rl[r].n < sl) {
                        sp = rl[r].p;
                        sl = rl[r].n;
                        pm = (set << 1 | 1u) & ~(2u << r);
                    }
                if (!valid) sl = 0;
                if (!__any_sync(kFull, sl > 0)) continue;
                int64_t incl = sl;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int64_t v = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += v;
                }
                const int64_t total = __shfl_sync(kFull, incl, 31);
                __syncwarp();
                offs[lane] = (int32_t)incl;
                lens[lane] = (int32_t)m;
                rptr[lane] = R;
                spt[lane] = sp;
                pmask[lane] = (int32_t)pm;
                __syncwarp();
                int lo = 0;
                for (int64_t f = lane; f < total; f += 32) {
                    while (offs[lo] <= f) ++lo;
                    const int64_t i = f - (lo ? offs[lo - 1] : 0);
                    const int32_t x = __ldg(spt[lo] + i);
                    const unsigned msk = (unsigned)pmask[lo];
                    bool found = true;
                    if (msk & 1u) found = contains(rptr[lo], lens[lo], x);
                    if (found && (msk & 2u)) found = in_sorted(rl[0].p, rl[0].n, x);
                    if (found && (msk & 4u)) found = in_sorted(rl[1].p, rl[1].n, x);
                    if (found) acc += plus ? 1ull : ~0ull;
                }
                __syncwarp();
            }
            continue;
        }
        if (valid && sub) {
            acc += (unsigned long long)Lc;  // |F part|; matches are subtracted below
            for (int j = 0; j < GZ_MAX_K; ++j)
                if ((xm >> j & 1) || (j == t && excl_self)) {
                    const int32_t e = j == t ? c : ws.emb[j];
                    if (e < beta && in_sorted(F, Lc, e) && !in_sorted(R, m, e)) acc -= 1ull;
                }
        }
        // A streams N(c) and probes F (a hash lookup when F is hashed); B streams
        // F and binary-searches N(c) in global memory, several dependent loads
        // per element, so A is taken up to 8x (shared-memory hash) or 2x (hash
        // in global scratch) the length of B
        const bool dirA = valid && (shape2 || m <= (!hashed ? Lc : (GH ? 2 * Lc : 8 * Lc)));
        const bool dirB = valid && !dirA;
        for (int pass = 0; pass < 2; ++pass) {
            const bool mine = pass == 0 ? dirA : dirB;
            if (!__any_sync(kFull, mine)) continue;
            const int64_t len = mine ? (pass == 0 ? m : Lc) : 0;
            int64_t incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            const int64_t total = __shfl_sync(kFull, incl, 31);
            __syncwarp();
            offs[lane] = (int32_t)incl;
            lens[lane] = (int32_t)m;
            rptr[lane] = R;
            __syncwarp();
            int lo = 0;  // first lane whose inclusive offset exceeds f (monotone in f)
            for (int64_t f = lane; f < total; f += 32) {
                while (offs[lo] <= f) ++lo;
                const int64_t i = f - (lo ? offs[lo - 1] : 0);
                bool found;
                int32_t x;
                if (pass == 0) {
                    x = __ldg(rptr[lo] + i);
                    if (shape2) {
                        bool keep = true;
                        for (int r = 0; r < op.nright && keep; ++r) {
                            ListRef rl = adj_list(q, ws.emb[op.right_pos[r]], op.right_dag[r]);
                            keep = in_sorted(rl.p, rl.n, x) != (op.right_sub[r] != 0);
                        }
                        if (keep && !excluded(xm, ws, x)) acc += 1ull;
                        continue;
                    }
                    found = !hashed ? in_sorted(F, nF, x) : (GH ? ghash_has(GH, glg, x) : hash_has(H, x));
                } else {
                    x = F[i];
                    found = contains(rptr[lo], lens[lo], x);
                }
                if (!sub) acc += (found && !excluded(xm, ws, x)) ? 1ull : 0ull;
                else acc -= found ? 1ull : 0ull;
            }
            __syncwarp();
        }
    }
    __syncwarp();
}

// Runs one unit (e0, e1), loop 2 restricted to candidates [lo2, hi2) (hi2 < 0:
// all). With df.list set, a unit with at least q.split_min loop-2 candidates is
// recorded for the split pass instead (u = its launch-space index).
__device__ void process_unit(const KQ& q, int64_t unit, WarpState& ws, int32_t* scratch,
                             int32_t* sm, int lane, unsigned long long& acc, int* status,
                             int64_t lo2 = 0, int64_t hi2 = -1, const DeferCtl* df = nullptr,
                             int64_t u = 0) {
    const GzProg& P = q.prog;
    const int k = P.k;
    const int32_t e0 = q.usrc[unit];
    if (q.min_root_out > 0 && q.drp[e0 + 1] - q.drp[e0] < q.min_root_out) return;
    const int32_t e1 = q.ucol[unit];
    ws.emb[0] = e0;
    ws.emb[1] = e1;
    ws.itp[1] = unit - q.urp[e0];
    if (k == 2) {
        if (lane == 0) acc += 1;
        return;
    }
    run_level(q, 1, ws, scratch, lane, acc, status);
    if (k == 3) return;
    const ListRef c2 = cand_list(q, 2, ws, scratch, lane);
    if (df && df->list && c2.n >= q.split_min) {
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(df->count, 1ull);
        slot = __shfl_sync(kFull, slot, 0);
        if ((int64_t)slot < df->cap) {
            if (lane == 0) df->list[slot] = Deferred{u, c2.n, q.split_chunk, q.merge_pos};
            __syncwarp();
            return;
        }
    }
    if (hi2 < 0 || hi2 > c2.n) hi2 = c2.n;
    if (lo2 >= hi2) return;
    const bool flat = P.flat != 0;
    if (k == 4 && flat) {
        ListRef S{c2.p + lo2, hi2 - lo2};
        last_level_flat(q, P.ops[P.level_begin[2]], ws, S, lo2, scratch, sm, lane, acc);
        return;
    }
    // explicit DFS over loops 2..k-2 (2..k-3 when the last loop is flattened)
    const int dmax = flat ? k - 3 : k - 2;
    const int32_t* cp[GZ_MAX_K];
    int64_t cn[GZ_MAX_K], it[GZ_MAX_K];
    int d = 2;
    cp[2] = c2.p; cn[2] = hi2; it[2] = lo2;
    while (d >= 2) {
        if (it[d] >= cn[d]) { --d; continue; }
        const int64_t pos = it[d]++;
        const int32_t c = cp[d][pos];
        bool skip = false;
        const uint8_t ex = P.cand_excl[d];
        if (ex)
            for (int j = 0; j < d; ++j)
                if ((ex >> j & 1) && ws.emb[j] == c) skip = true;
        if (skip) continue;
        ws.emb[d] = c;
        ws.itp[d] = pos;
        run_level(q, d, ws, scratch, lane, acc, status);
        if (d < dmax) {
            ++d;
            ListRef r = cand_list(q, d, ws, scratch, lane);
            cp[d] = r.p; cn[d] = r.n; it[d] = 0;
        } else if (flat) {
            last_level_flat(q, P.ops[P.level_begin[k - 2]], ws, cand_list(q, k - 2, ws, scratch, lane), 0,
                            scratch, sm, lane, acc);
        }
    }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Persistent enumeration kernel over a batch of queries (nq >= 1).
__global__ void __launch_bounds__(256, 3) k_enumerate(const KQ* __restrict__ qs, int nq,
                                                   int64_t total_units, int chunk,
                                                   unsigned long long* __restrict__ work,
                                                   unsigned long long* __restrict__ counts,
                                                   int* __restrict__ status,
                                                   int32_t* __restrict__ scratch,
                                                   int64_t words_per_warp, DeferCtl df) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t* my = scratch + gwarp * words_per_warp;
    int32_t* sm = smem + (threadIdx.x >> 5) * kWarpSmemWords;
    WarpState ws;
    unsigned long long acc = 0;
    int cur = -1;
    for (;;) {
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(work, (unsigned long long)chunk);
        start = __shfl_sync(kFull, start, 0);
        if ((int64_t)start >= total_units) break;
        int64_t end = (int64_t)start + chunk;
        if (end > total_units) end = total_units;
        for (int64_t u = (int64_t)start; u < end; ++u) {
            if (cur < 0 || u < qs[cur].unit_begin || u >= qs[cur].unit_begin + qs[cur].unit_count) {
                if (cur >= 0) {
                    unsigned long long s = warp_sum(acc);
                    if (lane == 0 && s) atomicAdd(&counts[qs[cur].out_slot], s);
                    acc = 0;
                }
                int lo = 0, hi = nq - 1;  // last query with unit_begin <= u
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (qs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
                }
                cur = lo;
            }
            const KQ& q = qs[cur];
            process_unit(q, q.unit_lo + (u - q.unit_begin), ws, my, sm, lane, acc, status, 0, -1, &df, u);
        }
    }
    if (cur >= 0) {
        unsigned long long s = warp_sum(acc);
        if (lane == 0 && s) atomicAdd(&counts[qs[cur].out_slot], s);
    }
}

// prefix[i] = chunks of the deferred records before record i (exclusive), for
// the min(count, cap) records of the first pass; prefix[n] = all chunks. One CTA.
__global__ void __launch_bounds__(1024) k_split_scan(const Deferred* __restrict__ dl,
                                                     const unsigned long long* __restrict__ dcount,
                                                     int64_t cap, int64_t* __restrict__ prefix) {
    __shared__ int64_t part[1024];
    const int64_t n = (int64_t)*dcount < cap ? (int64_t)*dcount : cap;
    const int64_t per = (n + 1023) / 1024;
    const int64_t b = threadIdx.x * per, e = b + per < n ? b + per : n;
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += (dl[i].n2 + dl[i].chunk - 1) / dl[i].chunk;
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int64_t x = part[i];
            part[i] = run;
            run += x;
        }
        prefix[n] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        prefix[i] = run;
        run += (dl[i].n2 + dl[i].chunk - 1) / dl[i].chunk;
    }
}

// Second pass: chunk t of the deferred units, one per warp pop.
__global__ void __launch_bounds__(256, 3) k_enumerate_split(const KQ* __restrict__ qs, int nq,
                                                         const Deferred* __restrict__ dl,
                                                         const unsigned long long* __restrict__ dcount,
                                                         int64_t cap,
                                                         const int64_t* __restrict__ prefix,
                                                         unsigned long long* __restrict__ work,
                                                         unsigned long long* __restrict__ counts,
                                                         int* __restrict__ status,
                                                         int32_t* __restrict__ scratch,
                                                         int64_t words_per_warp) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t* my = scratch + gwarp * words_per_warp;
    int32_t* sm = smem + (threadIdx.x >> 5) * kWarpSmemWords;
    const int64_t n = (int64_t)*dcount < cap ? (int64_t)*dcount : cap;
    const int64_t total = prefix[n];
    WarpState ws;
    unsigned long long acc = 0;
    int cur = -1;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(work, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= total) break;
        int64_t lo = 0, hi = n - 1;  // last record with prefix <= t
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= (int64_t)t) lo = mid; else hi = mid - 1;
        }
        const Deferred rec = dl[lo];
        const int64_t c0 = ((int64_t)t - prefix[lo]) * rec.chunk;
        const int64_t u = rec.unit;
        if (cur < 0 || u < qs[cur].unit_begin || u >= qs[cur].unit_begin + qs[cur].unit_count) {
            if (cur >= 0) {
                unsigned long long s = warp_sum(acc);
                if (lane == 0 && s) atomicAdd(&counts[qs[cur].out_slot], s);
                acc = 0;
            }
            int a = 0, b = nq - 1;
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (qs[mid].unit_begin <= u) a = mid; else b = mid - 1;
            }
            cur = a;
        }
        const KQ& q = qs[cur];
        process_unit(q, q.unit_lo + (u - q.unit_begin), ws, my, sm, lane, acc, status, c0,
                     c0 + rec.chunk);
    }
    if (cur >= 0) {
        unsigned long long s = warp_sum(acc);
        if (lane == 0 && s) atomicAdd(&counts[qs[cur].out_slot], s);
    }
}

// Single-query form of k_enumerate: the descriptor travels as a kernel
// parameter (no descriptor copy) and all device state (queue counters, count,
// status, deferred records, per-warp scratch) lives in one region the caller
// provides, so a count allocates nothing. With df.list set, heavy units are
// recorded for k_enumerate_split_one as in k_enumerate.
__global__ void __launch_bounds__(256, 3) k_enumerate_one(const __grid_constant__ KQ q,
                                                       int64_t total_units, int chunk,
                                                       unsigned long long* __restrict__ work,
                                                       unsigned long long* __restrict__ count,
                                                       int* __restrict__ status,
                                                       int32_t* __restrict__ scratch,
                                                       int64_t words_per_warp, DeferCtl df) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t* my = scratch + gwarp * words_per_warp;
    int32_t* sm = smem + (threadIdx.x >> 5) * kWarpSmemWords;
    WarpState ws;
    unsigned long long acc = 0;
    for (;;) {
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(work, (unsigned long long)chunk);
        start = __shfl_sync(kFull, start, 0);
        if ((int64_t)start >= total_units) break;
        int64_t end = (int64_t)start + chunk;
        if (end > total_units) end = total_units;
        for (int64_t u = (int64_t)start; u < end; ++u)
            process_unit(q, q.unit_lo + u, ws, my, sm, lane, acc, status, 0, -1, &df, u);
    }
    unsigned long long s = warp_sum(acc);
    if (lane == 0 && s) atomicAdd(count, s);
}

// Second pass of k_enumerate_one: chunk t of the deferred units, one per warp pop.
__global__ void __launch_bounds__(256, 3) k_enumerate_split_one(const __grid_constant__ KQ q,
                                                             const Deferred* __restrict__ dl,
                                                             const unsigned long long* __restrict__ dcount,
                                                             int64_t cap,
                                                             const int64_t* __restrict__ prefix,
                                                             unsigned long long* __restrict__ work,
                                                             unsigned long long* __restrict__ count,
                                                             int* __restrict__ status,
                                                             int32_t* __restrict__ scratch,
                                                             int64_t words_per_warp) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t* my = scratch + gwarp * words_per_warp;
    int32_t* sm = smem + (threadIdx.x >> 5) * kWarpSmemWords;
    const int64_t n = (int64_t)*dcount < cap ? (int64_t)*dcount : cap;
    const int64_t total = prefix[n];
    WarpState ws;
    unsigned long long acc = 0;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(work, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= total) break;
        int64_t lo = 0, hi = n - 1;  // last record with prefix <= t
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= (int64_t)t) lo = mid; else hi = mid - 1;
        }
        const Deferred rec = dl[lo];
        const int64_t c0 = ((int64_t)t - prefix[lo]) * rec.chunk;
        process_unit(q, q.unit_lo + rec.unit, ws, my, sm, lane, acc, status, c0, c0 + rec.chunk);
    }
    unsigned long long s = warp_sum(acc);
    if (lane == 0 && s) atomicAdd(count, s);
}

// Merged program: several plans over one unit space (GzMerged). One warp per
// unit binds (e0, e1), runs the shared loop-1 operations (mq) once, then each
// plan's own loops (pq[p]). Per-plan counts gather in the warp's counters in
// its scratch (cnt_off words in) and are added to counts[] once at the end. A
// plan's heavy unit is deferred with its position in the group; the split pass
// then runs only the shared operations that plan reads (its mask).
__device__ __forceinline__ void bind_shared(const KQ& m, int64_t unit, uint64_t mask, WarpState& ws,
                                            int32_t* my, int lane, int* status) {
    const int32_t e0 = m.usrc[unit];
    ws.emb[0] = e0;
    ws.emb[1] = m.ucol[unit];
    ws.itp[1] = unit - m.urp[e0];
    unsigned long long none = 0;  // the shared operations write buffers, they count nothing
    const GzProg& P = m.prog;
    for (int i = P.level_begin[1]; i < P.level_end[1]; ++i)
        if ((mask >> i) & 1ull) exec_op(m, P.ops[i], ws, my, lane, none, status);
}

__global__ void __launch_bounds__(256, 3) k_enumerate_merged(const KQ* __restrict__ mq,
                                                          const KQ* __restrict__ pq, int np,
                                                          int64_t total_units, int chunk,
                                                          unsigned long long* __restrict__ work,
                                                          unsigned long long* __restrict__ counts,
                                                          int* __restrict__ status,
                                                          int32_t* __restrict__ scratch,
                                                          int64_t words_per_warp, int64_t cnt_off,
                                                          DeferCtl df) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t* my = scratch + gwarp * words_per_warp;
    unsigned long long* wc = reinterpret_cast<unsigned long long*>(my + cnt_off);
    int32_t* sm = smem + (threadIdx.x >> 5) * kWarpSmemWords;
    for (int p = lane; p < np; p += 32) wc[p] = 0;
    __syncwarp();
    const KQ& m = mq[0];
    WarpState ws;
    for (;;) {
        unsigned long long start = 0;
        if (lane == 0) start = atomicAdd(work, (unsigned long long)chunk);
        start = __shfl_sync(kFull, start, 0);
        if ((int64_t)start >= total_units) break;
        int64_t end = (int64_t)start + chunk;
        if (end > total_units) end = total_units;
        for (int64_t u = (int64_t)start; u < end; ++u) {
            const int64_t unit = m.unit_lo + u;
            bind_shared(m, unit, m.shared_mask, ws, my, lane, status);
            for (int p = 0; p < np; ++p) {
                unsigned long long acc = 0;
                process_unit(pq[p], unit, ws, my, sm, lane, acc, status, 0, -1, &df, u);
                if (__any_sync(kFull, acc != 0)) {
                    const unsigned long long t = warp_sum(acc);
                    if (lane == 0) wc[p] += t;
                }
            }
        }
    }
    __syncwarp();
    if (lane == 0)
        for (int p = 0; p < np; ++p)
            if (wc[p]) atomicAdd(&counts[pq[p].out_slot], wc[p]);
}

// Second pass of a merged launch: chunk t of the deferred (unit, plan) records.
__global__ void __launch_bounds__(256, 3) k_enumerate_merged_split(const KQ* __restrict__ mq,
                                                                const KQ* __restrict__ pq,
                                                                const Deferred* __restrict__ dl,
                                                                const unsigned long long* __restrict__ dcount,
                                                                int64_t cap,
                                                                const int64_t* __restrict__ prefix,
                                                                unsigned long long* __restrict__ work,
                                                                unsigned long long* __restrict__ counts,
                                                                int* __restrict__ status,
                                                                int32_t* __restrict__ scratch,
                                                                int64_t words_per_warp) {
    extern __shared__ int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int32_t* my = scratch + gwarp * words_per_warp;
    int32_t* sm = smem + (threadIdx.x >> 5) * kWarpSmemWords;
    const int64_t n = (int64_t)*dcount < cap ? (int64_t)*dcount : cap;
    const int64_t total = prefix[n];
    const KQ& m = mq[0];
    WarpState ws;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(work, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= total) break;
        int64_t lo = 0, hi = n - 1;  // last record with prefix <= t
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= (int64_t)t) lo = mid; else hi = mid - 1;
        }
        const Deferred rec = dl[lo];
        const int64_t c0 = ((int64_t)t - prefix[lo]) * rec.chunk;
        const int64_t unit = m.unit_lo + rec.unit;
        const KQ& q = pq[rec.plan];
        bind_shared(m, unit, q.shared_mask, ws, my, lane, status);
        unsigned long long acc = 0;
        process_unit(q, unit, ws, my, sm, lane, acc, status, c0, c0 + rec.chunk);
        const unsigned long long sum = warp_sum(acc);
        if (lane == 0 && sum) atomicAdd(&counts[q.out_slot], sum);
    }
}

void fill_kq(const Query& Q, const LaunchCfg& cfg, KQ& k, uint64_t* words_out) {
    memset(&k, 0, sizeof(KQ));
    k.split_min = Q.split_min > 0 ? Q.split_min : cfg.split_min;
    k.split_chunk = Q.split_chunk > 0 ? Q.split_chunk : cfg.split_chunk;
    if (k.split_min <= 0 || k.split_chunk <= 0) {
        int64_t smin = 0, sch = 0;
        auto_split(*Q.prog, Q.unit_hi - Q.unit_lo, resident_warps(cfg), &smin, &sch);
        if (k.split_min <= 0) k.split_min = smin;
        if (k.split_chunk <= 0) k.split_chunk = sch;
    }
    if (k.split_chunk < 1) k.split_chunk = 1;
    k.prog = *Q.prog;
    const GzView& v = *Q.view;
    k.rp = v.rp; k.col = v.col; k.drp = v.dag_rp; k.dcol = v.dag_col;
    if (Q.prog->unit_dag) { k.usrc = v.dag_src; k.ucol = v.dag_col; k.urp = v.dag_rp; }
    else { k.usrc = v.src; k.ucol = v.col; k.urp = v.rp; }
    k.unit_lo = Q.unit_lo;
    k.unit_count = Q.unit_hi - Q.unit_lo;
    k.min_root_out = Q.min_root_out;
    k.out_slot = 0;
    *words_out = scratch_layout(*Q.prog, *Q.g, v, &k);
}

// Dynamic shared memory of a CTA of bw warps, and the limit raised once per
// device for each enumeration kernel (8 warps, above the 48 KB default).
inline size_t cta_smem(int bw) { return (size_t)bw * kWarpSmemWords * 4; }
std::atomic<unsigned long long> g_attr_enum{0}, g_attr_split{0}, g_attr_one{0}, g_attr_split_one{0};
std::atomic<unsigned long long> g_attr_merged{0}, g_attr_merged_split{0};

cudaError_t enum_attrs() {
    const int b = (int)cta_smem(8);
    cudaError_t e = smem_attr_once(k_enumerate, b, g_attr_enum);
    if (e == cudaSuccess) e = smem_attr_once(k_enumerate_split, b, g_attr_split);
    if (e == cudaSuccess) e = smem_attr_once(k_enumerate_one, b, g_attr_one);
    if (e == cudaSuccess) e = smem_attr_once(k_enumerate_split_one, b, g_attr_split_one);
    return e;
}

// SM count and resident CTAs per SM of k_enumerate for each block size, per
// device, looked up once (the occupancy query costs microseconds per call).
struct OccKey {
    int dev, bw;
    bool operator<(const OccKey& o) const { return dev != o.dev ? dev < o.dev : bw < o.bw; }
};
std::mutex g_occ_mu;
std::map<OccKey, std::pair<int, int>> g_occ;

gz_status grid_shape(int bw, int* sms_out, int* per_sm_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "count: cudaGetDevice");
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find(OccKey{dev, bw});
        if (it != g_occ.end()) {
            *sms_out = it->second.first;
            *per_sm_out = it->second.second;
            return GZ_OK;
        }
    }
    e = enum_attrs();
    if (e != cudaSuccess) return cuda_fail(e, "count: kernel shared-memory attribute");
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enumerate, bw * 32, cta_smem(bw));
    if (e != cudaSuccess) return cuda_fail(e, "count: occupancy");
    if (per_sm < 1) per_sm = 1;
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ[OccKey{dev, bw}] = {sms, per_sm};
    *sms_out = sms;
    *per_sm_out = per_sm;
    return GZ_OK;
}

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Deferred-record capacity of a launch over `units` work units.
inline int64_t defer_cap(int64_t units) { return std::min<int64_t>(units, (int64_t)1 << 20); }

}  // namespace

// A unit goes to the split pass from split_min loop-2 candidates on and is cut
// into work items of split_chunk candidates; every item recomputes loop 1. A
// query with many units per resident warp keeps few, coarse items (512, 256):
// its heavy units end while the others still run. A query with few units per
// warp (a narrow root range, a small graph) ends on the critical path of its
// heaviest units, so it cuts them finely: to single candidates when each
// loop-2 candidate carries work that grows with its degree (a flattened last
// loop that streams N(c) against fixed lists, or loops below loop 2), to items
// of 64 from 64 candidates on for k = 4 patterns whose last loop intersects
// with a fixed operand. Measured on GB300 on the oracle's sampled R-MAT 22
// ranges (against (512, 256): tailed triangle 18x, chordal 5-cycle 9x, diamond
// 1.8x, c4 1.2x faster) and on full R-MAT 16 and 18 counts (where (512, 256)
// is the fastest or within noise of it).
constexpr int64_t kNarrowUnitsPerWarp = 64;

void auto_split(const GzProg& p, int64_t units, int warps, int64_t* split_min, int64_t* split_chunk) {
    if (units < kNarrowUnitsPerWarp * (int64_t)std::max(warps, 1)) {
        const bool per_candidate_heavy = p.flat == 2 || p.k >= 5;
        *split_min = per_candidate_heavy ? 4 : 64;
        *split_chunk = per_candidate_heavy ? 1 : 64;
    } else {
        *split_min = 512;
        *split_chunk = 256;
    }
}

// Bytes of a single-query region before its scratch: the counters, then (with
// splitting) the deferred records and the chunk prefix.
uint64_t one_meta_bytes(const Query& Q, bool split) {
    if (!split || Q.prog->k < 4) return kRegionHeader;
    const int64_t cap = defer_cap(Q.unit_hi - Q.unit_lo);
    return kRegionHeader + align256(sizeof(Deferred) * cap) + align256(sizeof(int64_t) * (cap + 1));
}

// Counts one query with every piece of device state inside `region`:
// one_meta_bytes(Q, split) bytes of counters (pass-1 queue, count, status,
// pass-2 queue, deferred-record count) and deferred records, then scratch_bytes
// of per-warp scratch. Launches fewer warps when the scratch would not hold a
// full grid. Allocates nothing. Synchronous: the count and status are read back
// into pinned (16 bytes of page-locked host memory) or, when it is NULL, host
// locals. split = false runs no second pass (every unit in the first).
gz_status count_one_in_region(const Query& Q, const LaunchCfg& cfg, cudaStream_t s, void* region,
                              uint64_t scratch_bytes, bool split, uint64_t* out_count,
                              unsigned long long* pinned) {
    KQ k;
    uint64_t words = 0;
    fill_kq(Q, cfg, k, &words);
    const int64_t total = Q.unit_hi - Q.unit_lo;
    *out_count = 0;
    if (total <= 0) return GZ_OK;
    split = split && Q.prog->k >= 4;
    int bw = cfg.block_warps, sms = 0, per_sm = 0;
    gz_status st = grid_shape(bw, &sms, &per_sm);
    if (st != GZ_OK) return st;
    int64_t warps = (int64_t)sms * per_sm * bw;
    if (cfg.blocks > 0) warps = (int64_t)cfg.blocks * bw;
    if (words > 0) {
        const int64_t fit = (int64_t)(scratch_bytes / (words * sizeof(int32_t)));
        if (fit < 1) {
            set_error("count: %llu bytes of scratch per warp exceed the %llu-byte region",
                      (unsigned long long)(words * 4), (unsigned long long)scratch_bytes);
            return GZ_EOVERFLOW;
        }
        if (fit < warps) warps = fit;
    }
    if (warps < bw) bw = (int)warps;
    const int blocks = (int)(warps / bw);
    char* base = reinterpret_cast<char*>(region);
    unsigned long long* hdr = reinterpret_cast<unsigned long long*>(region);
    int* status = reinterpret_cast<int*>(hdr + 2);
    const uint64_t meta = one_meta_bytes(Q, split);
    int32_t* scratch = reinterpret_cast<int32_t*>(base + meta);
    const int64_t cap = split ? defer_cap(total) : 0;
    Deferred* dl = split ? reinterpret_cast<Deferred*>(base + kRegionHeader) : nullptr;
    int64_t* prefix = split ? reinterpret_cast<int64_t*>(base + kRegionHeader + align256(sizeof(Deferred) * cap))
                            : nullptr;
    const int chunk = cfg.chunk > 0 ? cfg.chunk : 1;
    cudaError_t e = cudaMemsetAsync(region, 0, kRegionHeader, s);
    if (e == cudaSuccess) {
        DeferCtl df{dl, hdr + 4, cap};
        k_enumerate_one<<<blocks, bw * 32, cta_smem(bw), s>>>(k, total, chunk, hdr, hdr + 1, status, scratch,
                                                             (int64_t)words, df);
        GZ_COUNT_LAUNCH();
        if (split) {
            k_split_scan<<<1, 1024, 0, s>>>(dl, hdr + 4, cap, prefix);
            GZ_COUNT_LAUNCH();
            k_enumerate_split_one<<<blocks, bw * 32, cta_smem(bw), s>>>(k, dl, hdr + 4, cap, prefix, hdr + 3,
                                                                       hdr + 1, status, scratch, (int64_t)words);
            GZ_COUNT_LAUNCH();
        }
        e = cudaGetLastError();
    }
    unsigned long long local[2] = {0, 0};
    unsigned long long* h = pinned ? pinned : local;  // pinned: an asynchronous 16-byte read-back
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, hdr + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "count (region)");
    if ((int)h[1] != 0) {
        set_error("count: a scratch buffer overflowed (planner capacity bug)");
        return GZ_EOVERFLOW;
    }
    *out_count = h[0];
    return GZ_OK;
}

uint64_t scratch_words_per_warp(const GzProg& p, const gz_graph& g, const GzView& v) {
    return scratch_layout(p, g, v, nullptr);
}

int resident_warps(const LaunchCfg& cfg) {
    int sms = 0, per_sm = 0;
    if (grid_shape(cfg.block_warps, &sms, &per_sm) != GZ_OK) {
        sms = 1;
        per_sm = 1;
    }
    const int blocks = cfg.blocks > 0 ? cfg.blocks : sms * per_sm;
    return blocks * cfg.block_warps;
}

// Device bytes count_launch needs beside the scratch: the query descriptors,
// four counters, and (when some query has k >= 4) the deferred records and
// their chunk prefix.
uint64_t launch_meta_bytes(const Query* qs, int nq) {
    if (nq <= 0) return 0;
    int64_t total = 0;
    bool split = false;
    for (int i = 0; i < nq; ++i) {
        total += qs[i].unit_hi - qs[i].unit_lo;
        split = split || qs[i].prog->k >= 4;
    }
    const int64_t cap = split ? defer_cap(total) : 0;
    return align256(sizeof(KQ) * nq) + 256 + align256(sizeof(Deferred) * cap) +
           align256(sizeof(int64_t) * (cap + 1));
}

// Builds the per-query descriptors, then one persistent launch. d_counts[nq] must
// be zeroed by the caller (on stream s); scratch must hold resident_warps(cfg) *
// max words per warp int32 words; meta must hold launch_meta_bytes(qs, nq) bytes
// (256-byte aligned). Allocates nothing.
gz_status count_launch(const Query* qs, int nq, const LaunchCfg& cfg, cudaStream_t s,
                       unsigned long long* d_counts, void* scratch, uint64_t scratch_bytes,
                       int* d_status, void* meta, uint64_t meta_bytes) {
    if (nq <= 0) return GZ_OK;
    std::vector<KQ> h(nq);
    int64_t total = 0;
    uint64_t words = 0;
    for (int i = 0; i < nq; ++i) {
        const Query& Q = qs[i];
        KQ& k = h[i];
        uint64_t w = 0;
        fill_kq(Q, cfg, k, &w);
        k.unit_begin = total;
        k.out_slot = Q.out_slot >= 0 ? Q.out_slot : i;
        total += k.unit_count;
        if (w > words) words = w;
    }
    if (total == 0) return GZ_OK;
    const int warps = resident_warps(cfg);
    if ((uint64_t)warps * words * sizeof(int32_t) > scratch_bytes) {
        set_error("count: scratch too small (%llu bytes needed)",
                  (unsigned long long)((uint64_t)warps * words * 4));
        return GZ_ENOMEM;
    }
    if (meta_bytes < launch_meta_bytes(qs, nq)) {
        set_error("count: launch metadata region too small");
        return GZ_ENOMEM;
    }
    // meta: queries | 4 counters (pass-1 queue, pass-2 queue, records) |
    // deferred records [cap] | chunk prefix [cap + 1]
    bool split = false;
    for (int i = 0; i < nq; ++i) split = split || qs[i].prog->k >= 4;
    const int64_t cap = split ? defer_cap(total) : 0;
    char* base = reinterpret_cast<char*>(meta);
    const uint64_t qbytes = align256(sizeof(KQ) * nq);
    KQ* d = reinterpret_cast<KQ*>(base);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(base + qbytes);
    Deferred* dl = reinterpret_cast<Deferred*>(base + qbytes + 256);
    int64_t* prefix = reinterpret_cast<int64_t*>(base + qbytes + 256 + align256(sizeof(Deferred) * cap));
    cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(KQ) * nq, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, 32, s);
    if (e == cudaSuccess) {
        int blocks = warps / cfg.block_warps;
        if (cfg.grid_frac < 1.0) blocks = std::max(1, (int)(blocks * cfg.grid_frac));
        DeferCtl df{split ? dl : nullptr, work + 2, cap};
        k_enumerate<<<blocks, cfg.block_warps * 32, cta_smem(cfg.block_warps), s>>>(
            d, nq, total, cfg.chunk > 0 ? cfg.chunk : 1, work, d_counts, d_status,
            reinterpret_cast<int32_t*>(scratch), (int64_t)words, df);
        GZ_COUNT_LAUNCH();
        if (split) {
            k_split_scan<<<1, 1024, 0, s>>>(dl, work + 2, cap, prefix);
            GZ_COUNT_LAUNCH();
            k_enumerate_split<<<blocks, cfg.block_warps * 32, cta_smem(cfg.block_warps), s>>>(
                d, nq, dl, work + 2, cap, prefix, work + 1, d_counts, d_status,
                reinterpret_cast<int32_t*>(scratch), (int64_t)words);
            GZ_COUNT_LAUNCH();
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "enumerate launch");
    return GZ_OK;
}

// Scratch layout of a merged launch (per warp): the shared buffers, then the
// largest own region of any plan (its buffers and, for a fixed-operand last
// loop, its hash table), then one uint64 counter per plan. Fills the shared
// descriptor and the plans' buffer offsets when mk / pk are given.
static uint64_t merged_layout(const GzMerged& m, const gz_graph& g, const GzView& v, KQ* mk, KQ* pk,
                              uint64_t* cnt_off) {
    auto cap_of = [&](int dag) { return (uint64_t)(dag ? v.max_out : g.max_deg); };
    const int ns = m.shared.nbuf;
    uint64_t off = 0;
    int64_t soff[GZ_MAXBUF], scap[GZ_MAXBUF];
    for (int b = 0; b < ns; ++b) {
        const uint64_t cap = cap_of(m.shared.buf_dag[b]);
        soff[b] = (int64_t)off;
        scap[b] = (int64_t)cap;
        if (mk) { mk->buf_off[b] = soff[b]; mk->buf_cap[b] = scap[b]; }
        off += (cap + 31) & ~31ull;
    }
    const uint64_t shared_words = off;
    uint64_t own_max = 0;
    for (size_t i = 0; i < m.progs.size(); ++i) {
        const GzProg& q = m.progs[i];
        KQ* k = pk ? pk + i : nullptr;
        uint64_t po = shared_words;
        for (int b = 0; b < q.nbuf; ++b) {
            if (b < ns) {
                if (k) { k->buf_off[b] = soff[b]; k->buf_cap[b] = scap[b]; }
                continue;
            }
            const uint64_t cap = cap_of(q.buf_dag[b]);
            if (k) { k->buf_off[b] = (int64_t)po; k->buf_cap[b] = (int64_t)cap; }
            po += (cap + 31) & ~31ull;
        }
        int lg = 0;
        const uint64_t capmax = (uint64_t)g.max_deg;
        if (q.flat == 1 && capmax > (uint64_t)kStageWords)
            while ((1ull << lg) < 2 * capmax && lg < kGlobalHashLog2) ++lg;
        if (k) {
            k->hash_off = (int64_t)po;
            k->hash_log2 = lg;
        }
        if (lg) po += 1ull << lg;
        own_max = std::max(own_max, po - shared_words);
    }
    const uint64_t co = (shared_words + own_max + 1) & ~1ull;  // uint64 counters, 8-byte aligned
    if (cnt_off) *cnt_off = co;
    return (co + 2 * m.progs.size() + 1) & ~1ull;  // even: every warp's region 8-byte aligned
}

// The shared operations plan q reads: those writing the buffers its operations
// and candidate lists use, closed over the shared operations' own inputs.
static uint64_t shared_mask_of(const GzProg& sh, const GzProg& q) {
    const int ns = sh.nbuf;
    uint64_t need = 0;  // bit b: shared buffer b is read
    for (int i = 0; i < q.nops; ++i)
        if (q.ops[i].left_buf >= 0 && q.ops[i].left_buf < ns) need |= 1ull << q.ops[i].left_buf;
    for (int d = 0; d < GZ_MAX_K; ++d)
        if (q.cand_buf[d] >= 0 && q.cand_buf[d] < ns) need |= 1ull << q.cand_buf[d];
    uint64_t mask = 0;
    for (int i = sh.nops - 1; i >= 0; --i)  // writers come before readers
        if ((need >> sh.ops[i].dst) & 1ull) {
            mask |= 1ull << i;
            if (sh.ops[i].left_buf >= 0) need |= 1ull << sh.ops[i].left_buf;
        }
    return mask;
}

uint64_t merged_scratch_words(const GzMerged& m, const gz_graph& g, const GzView& v) {
    return merged_layout(m, g, v, nullptr, nullptr, nullptr);
}

uint64_t merged_meta_bytes(const GzMerged& m, int64_t units) {
    bool split = false;
    for (const GzProg& q : m.progs) split = split || q.k >= 4;
    const int64_t cap = split ? defer_cap(units) : 0;
    return align256(sizeof(KQ) * (m.progs.size() + 1)) + 256 + align256(sizeof(Deferred) * cap) +
           align256(sizeof(int64_t) * (cap + 1));
}

gz_status count_merged(const GzMerged& m, const gz_graph* g, const GzView* v, const LaunchCfg& cfg,
                       cudaStream_t s, unsigned long long* d_counts, int* d_status, void* scratch,
                       uint64_t scratch_bytes, void* meta, uint64_t meta_bytes) {
    const int np = (int)m.progs.size();
    if (np == 0) return GZ_OK;
    const int64_t units = m.unit_dag ? v->dag_nnz : g->nnz;
    if (units <= 0) return GZ_OK;
    std::vector<KQ> h(np + 1);
    for (int i = 0; i <= np; ++i) {
        KQ& k = h[i];
        memset(&k, 0, sizeof(KQ));
        k.prog = i == 0 ? m.shared : m.progs[i - 1];
        k.rp = v->rp; k.col = v->col; k.drp = v->dag_rp; k.dcol = v->dag_col;
        if (m.unit_dag) { k.usrc = v->dag_src; k.ucol = v->dag_col; k.urp = v->dag_rp; }
        else { k.usrc = v->src; k.ucol = v->col; k.urp = v->rp; }
        k.unit_lo = 0;
        k.unit_count = units;
        // a merged split item re-runs the shared loop-1 operations its plan
        // reads, so narrow launches split less finely than single programs:
        // (128, 64), measured on R-MAT 12 motif-4/5 sets against (512, 256),
        // (64, 16) and (16, 4)
        int64_t smin = cfg.split_min, sch = cfg.split_chunk;
        const bool narrow = units < kNarrowUnitsPerWarp * (int64_t)resident_warps(cfg);
        if (smin <= 0) smin = narrow ? 128 : 512;
        if (sch <= 0) sch = narrow ? 64 : 256;
        k.split_min = smin;
        k.split_chunk = sch > 0 ? sch : 1;
        k.out_slot = i == 0 ? 0 : m.plan_index[i - 1];
        k.merge_pos = i == 0 ? 0 : i - 1;
        k.shared_mask = i == 0 ? (m.shared.nops >= 64 ? ~0ull : (1ull << m.shared.nops) - 1)
                               : shared_mask_of(m.shared, m.progs[i - 1]);
    }
    uint64_t cnt_off = 0;
    const uint64_t words = merged_layout(m, *g, *v, &h[0], h.data() + 1, &cnt_off);
    const int warps = resident_warps(cfg);
    if ((uint64_t)warps * words * sizeof(int32_t) > scratch_bytes) {
        set_error("merged count: scratch too small (%llu bytes needed)",
                  (unsigned long long)((uint64_t)warps * words * 4));
        return GZ_ENOMEM;
    }
    if (meta_bytes < merged_meta_bytes(m, units)) {
        set_error("merged count: launch metadata region too small");
        return GZ_ENOMEM;
    }
    bool split = false;
    for (const GzProg& q : m.progs) split = split || q.k >= 4;
    const int64_t cap = split ? defer_cap(units) : 0;
    char* base = reinterpret_cast<char*>(meta);
    const uint64_t qbytes = align256(sizeof(KQ) * (np + 1));
    KQ* d = reinterpret_cast<KQ*>(base);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(base + qbytes);
    Deferred* dl = reinterpret_cast<Deferred*>(base + qbytes + 256);
    int64_t* prefix = reinterpret_cast<int64_t*>(base + qbytes + 256 + align256(sizeof(Deferred) * cap));
    cudaError_t e = enum_attrs();
    if (e == cudaSuccess) e = smem_attr_once(k_enumerate_merged, (int)cta_smem(8), g_attr_merged);
    if (e == cudaSuccess) e = smem_attr_once(k_enumerate_merged_split, (int)cta_smem(8), g_attr_merged_split);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h.data(), sizeof(KQ) * (np + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, 32, s);
    if (e == cudaSuccess) {
        int blocks = warps / cfg.block_warps;
        if (cfg.grid_frac < 1.0) blocks = std::max(1, (int)(blocks * cfg.grid_frac));
        DeferCtl df{split ? dl : nullptr, work + 2, cap};
        // a merged unit carries every plan's work: one unit per queue pop
        k_enumerate_merged<<<blocks, cfg.block_warps * 32, cta_smem(cfg.block_warps), s>>>(
            d, d + 1, np, units, 1, work, d_counts, d_status, reinterpret_cast<int32_t*>(scratch),
            (int64_t)words, (int64_t)cnt_off, df);
        GZ_COUNT_LAUNCH();
        if (split) {
            k_split_scan<<<1, 1024, 0, s>>>(dl, work + 2, cap, prefix);
            GZ_COUNT_LAUNCH();
            k_enumerate_merged_split<<<blocks, cfg.block_warps * 32, cta_smem(cfg.block_warps), s>>>(
                d, d + 1, dl, work + 2, cap, prefix, work + 1, d_counts, d_status,
                reinterpret_cast<int32_t*>(scratch), (int64_t)words);
            GZ_COUNT_LAUNCH();
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "merged launch");
    return GZ_OK;
}

}  // namespace gz
