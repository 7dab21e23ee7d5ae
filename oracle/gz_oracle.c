/*
 * gz_oracle.c - the CPU oracle for vertex-induced pattern counting (GraphZero,
 * Mawhirter et al., arXiv 1911.12877).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the bench's CPU-baseline leg do.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, written plainly and slowly:
 *
 *  Oracle A (definition, tiny graphs)
 *    orc_count_brute_induced: #{U subset of V, |U| = k : G[U] isomorphic to P},
 *      trying every k-subset and every bijection onto P (vertex-induced matching,
 *      Sec. 2.1: black pattern edges must exist, red ones must be absent).
 *    orc_count_brute_injective: #{injective phi : V(P) -> V(G) preserving both
 *      edges and non-edges}; equals the induced count times |Aut(P)| (Sec. 4.1).
 *
 *  Planner pieces (Sec. 4, Sec. 5, Appendix)
 *    orc_automorphisms: Aut(P) by trying all k! permutations (Sec. 4.2).
 *    orc_restrictions: Algorithm 1 (restriction generation) and the Theorem 2
 *      reduction to one bound per schedule position (map child -> parent).
 *    orc_valid_schedules_brute: Algorithm 2 (all permutations, keep the valid).
 *    orc_distinct_schedules: Algorithm 4 (orbit pruning by stabilizers).
 *    orc_cost: the performance model of Sec. 5.4 and the Appendix.
 *
 *  Oracle B (the method on CPU)
 *    orc_count_nested: the nested loops of Sec. 4 with one bound per loop
 *      (Theorem 2) and bounded sorted-list set operations (Sec. 6). Each level's
 *      candidate set is rebuilt from the predecessors' neighbor lists. It also
 *      counts E, the list elements that bounded linear scans of those lists
 *      consume: for every partial embedding at every level d >= 1, the sum over
 *      all predecessors j < d of |N(e_j) intersect [0, bound_d)|.
 *    orc_reindex: the orientation relabelling of Sec. 6 (higher degree gets a
 *      smaller id; ties by original id, ascending).
 *
 *  Bitset work measure (for the roofline of bitset clique kernels)
 *    orc_clique_bitset_work: the 32-bit word operations of the oriented
 *      k-clique loops written over per-root bitsets (see its comment); also
 *      returns the clique count the walk finds, as a check.
 *
 *  Motifs (Sec. 7.1-7.2)
 *    orc_connected_patterns: every connected k-vertex graph up to isomorphism,
 *      by brute force over edge subsets and all k! relabellings.
 *
 * Readings where the paper is silent (the same list is kept in the design notes):
 *  - restriction (S[i], S[j]) in L means id(e_j) < id(e_i) (Theorem 1);
 *  - a level skips candidates equal to an already matched vertex;
 *  - Algorithm 4 removes vertices already scheduled from valid_next, and its
 *    "processed" marks are local to each recursive call; loops run in ascending
 *    label order;
 *  - cost model: n = 1000, p = 5/999; loop d runs n p^{#black} (1-p)^{#red}
 *    iterations per outer iteration (loop 0 runs n); the restriction pass
 *    probability up to loop d is prod_i 1/z_i, z_i = size of i's subtree in the
 *    restriction forest cut to loops <= d; cost = sum_d (prod_{j<=d} iters_j) *
 *    P_d; ties go to the first schedule in Algorithm 4 order.
 *
 * Mutation switch (orc_set_mutation) plants one known mistake at a time so the
 * tests can show the pins catch it. 0 = correct oracle.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXK 8
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ECAP -3

enum {
    MUT_NONE = 0,
    MUT_DROP_RED = 1,      /* forget the set subtraction of red predecessors */
    MUT_NO_BOUND = 2,      /* drop every restriction */
    MUT_NO_EXCLUDE = 3,    /* do not skip already matched vertices */
    MUT_BOUND_LE = 4,      /* bound taken inclusive (<=) */
    MUT_ALG1_NOSTAB = 5,   /* Algorithm 1 never shrinks the automorphism list */
    MUT_THM2_FIRST = 6,    /* Theorem 2 keeps the smallest z instead of the largest */
    MUT_AUT_NEXT_ONLY = 7, /* automorphism test only checks pairs (i, i+1) */
    MUT_REINDEX_ASC = 8,   /* orientation sorts degrees ascending */
    MUT_E_FULL = 9,        /* E counts whole lists, ignoring the bound */
    MUT_COST_NO_DIFF = 10, /* cost model drops the (1-p) factor of set differences */
    MUT_COST_EXP = 11,     /* cost model raises p to #black + 1 */
    MUT_COST_PRODUCT = 12  /* cost model multiplies the loops' costs instead of summing */
};

static int g_mut = 0;
void orc_set_mutation(int m) { g_mut = m; }

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- permutations */

/* Next permutation in lexicographic order; returns 0 after the last one. */
static int next_perm(int32_t* a, int k) {
    int i = k - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = k - 1;
    while (a[j] <= a[i]) --j;
    int32_t t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; ++l, --r) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

static int pattern_ok(int k, const uint8_t* adj) {
    if (k < 2 || k > ORC_MAXK) return 0;
    for (int i = 0; i < k; ++i) {
        if (adj[i * k + i]) return 0;
        for (int j = 0; j < k; ++j)
            if ((adj[i * k + j] != 0) != (adj[j * k + i] != 0)) return 0;
    }
    /* connected */
    int seen = 1, stack[ORC_MAXK], sp = 0;
    stack[sp++] = 0;
    while (sp) {
        int v = stack[--sp];
        for (int u = 0; u < k; ++u)
            if (adj[v * k + u] && !(seen >> u & 1)) { seen |= 1 << u; stack[sp++] = u; }
    }
    return seen == (1 << k) - 1;
}

/*
 * Aut(P): every permutation x of the labels with adj(i, j) == adj(x(i), x(j))
 * for all pairs (Sec. 4.2: all permutations are tried and the edge-preserving
 * ones kept). Writes up to cap permutations (k entries each); returns |Aut|.
 */
int orc_automorphisms(int k, const uint8_t* adj, int32_t* out, int cap) {
    if (!pattern_ok(k, adj)) return ORC_EINVAL;
    int32_t p[ORC_MAXK];
    for (int i = 0; i < k; ++i) p[i] = i;
    int cnt = 0;
    do {
        int ok = 1;
        for (int i = 0; i < k && ok; ++i)
            for (int j = i + 1; j < k; ++j) {
                if (g_mut == MUT_AUT_NEXT_ONLY && j != i + 1) continue;
                if ((adj[i * k + j] != 0) != (adj[p[i] * k + p[j]] != 0)) { ok = 0; break; }
            }
        if (ok) {
            if (cnt < cap && out) memcpy(out + (size_t)cnt * k, p, sizeof(int32_t) * k);
            ++cnt;
        }
    } while (next_perm(p, k));
    return cnt;
}

static int32_t* all_auts(int k, const uint8_t* adj, int* na) {
    int n = orc_automorphisms(k, adj, NULL, 0);
    if (n <= 0) { *na = n; return NULL; }
    int32_t* a = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * k);
    if (!a) { *na = ORC_ENOMEM; return NULL; }
    orc_automorphisms(k, adj, a, n);
    *na = n;
    return a;
}

static int schedule_valid(int k, const uint8_t* adj, const int32_t* order) {
    int used = 0;
    for (int i = 0; i < k; ++i) {
        int v = order[i];
        if (v < 0 || v >= k || (used >> v & 1)) return 0;
        if (i > 0) {
            int conn = 0;
            for (int j = 0; j < i; ++j) conn |= adj[v * k + order[j]] != 0;
            if (!conn) return 0;
        }
        used |= 1 << v;
    }
    return 1;
}

/*
 * Algorithm 1 for schedule `order` (labels), plus the Theorem 2 reduction.
 * pairs_out (optional, 2*cap label pairs) receives the full partial order L:
 * (v, x(v)) for every x in the current stabilizer that moves v. bp_out[i]
 * (schedule positions) is the one parent kept per position: Algorithm 1 visits
 * v in schedule order and overwrites map[x(v)] = v, so the latest, i.e. the
 * largest z, survives (Theorem 2). -1 = no bound. Returns |L| or an error.
 */
int orc_restrictions(int k, const uint8_t* adj, const int32_t* order, int32_t* bp_out,
                     int32_t* pairs_out, int cap) {
    if (!pattern_ok(k, adj) || !schedule_valid(k, adj, order)) return ORC_EINVAL;
    int na;
    int32_t* aut = all_auts(k, adj, &na);
    if (!aut) return na < 0 ? na : ORC_ENOMEM;
    int pos[ORC_MAXK];
    for (int i = 0; i < k; ++i) pos[order[i]] = i;
    int map_label[ORC_MAXK];
    for (int i = 0; i < k; ++i) map_label[i] = -1;
    uint8_t inL[ORC_MAXK][ORC_MAXK];
    memset(inL, 0, sizeof(inL));
    int npairs = 0;
    for (int s = 0; s < k; ++s) {
        int v = order[s];
        int keep = 0;
        for (int a = 0; a < na; ++a) {
            const int32_t* x = aut + (size_t)a * k;
            if (x[v] == v) {
                if (keep != a) memmove(aut + (size_t)keep * k, x, sizeof(int32_t) * k);
                ++keep;
            } else {
                int w = x[v];
                if (!inL[v][w]) {
                    inL[v][w] = 1;
                    if (pairs_out && npairs < cap) { pairs_out[2 * npairs] = v; pairs_out[2 * npairs + 1] = w; }
                    ++npairs;
                }
                if (g_mut == MUT_THM2_FIRST) { if (map_label[w] < 0) map_label[w] = v; }
                else map_label[w] = v;
                if (g_mut == MUT_ALG1_NOSTAB) ++keep; /* keeps the list unchanged */
            }
        }
        if (g_mut != MUT_ALG1_NOSTAB) na = keep;
    }
    free(aut);
    if (bp_out)
        for (int i = 0; i < k; ++i)
            bp_out[i] = map_label[order[i]] < 0 ? -1 : pos[map_label[order[i]]];
    return npairs;
}

/* Algorithm 2: every permutation of the labels that is a valid schedule. */
int orc_valid_schedules_brute(int k, const uint8_t* adj, int32_t* out, int cap) {
    if (!pattern_ok(k, adj)) return ORC_EINVAL;
    int32_t p[ORC_MAXK];
    for (int i = 0; i < k; ++i) p[i] = i;
    int cnt = 0;
    do {
        if (schedule_valid(k, adj, p)) {
            if (out && cnt < cap) memcpy(out + (size_t)cnt * k, p, sizeof(int32_t) * k);
            ++cnt;
        }
    } while (next_perm(p, k));
    return cnt;
}

typedef struct {
    int k;
    const uint8_t* adj;
    int32_t* out;
    int cap;
    int cnt;
} a4_ctx;

/* One call of Algorithm 4's recursive procedure. */
static void a4_rec(a4_ctx* c, int32_t* sched, int len, const int32_t* aut, int na, int valid_next) {
    int k = c->k;
    if (len == k) {
        if (c->out && c->cnt < c->cap) memcpy(c->out + (size_t)c->cnt * k, sched, sizeof(int32_t) * k);
        c->cnt++;
        return;
    }
    int iterate = len == 0 ? (1 << k) - 1 : valid_next;
    int processed = 0; /* local to this call */
    int32_t* stab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(na > 0 ? na : 1) * k);
    for (int v = 0; v < k; ++v) {
        if (!(iterate >> v & 1) || (processed >> v & 1)) continue;
        int ns = 0;
        for (int a = 0; a < na; ++a) {
            const int32_t* x = aut + (size_t)a * k;
            if (x[v] == v) memcpy(stab + (size_t)ns++ * k, x, sizeof(int32_t) * k);
            else processed |= 1 << x[v];
        }
        int nb = 0;
        for (int u = 0; u < k; ++u) nb |= (c->adj[v * k + u] != 0) << u;
        int in_sched = 1 << v;
        for (int i = 0; i < len; ++i) in_sched |= 1 << sched[i];
        sched[len] = v;
        a4_rec(c, sched, len + 1, stab, ns, (valid_next | nb) & ~in_sched);
    }
    free(stab);
}

/* Algorithm 4: the distinct schedules, in generation order. Returns how many. */
int orc_distinct_schedules(int k, const uint8_t* adj, int32_t* out, int cap) {
    if (!pattern_ok(k, adj)) return ORC_EINVAL;
    int na;
    int32_t* aut = all_auts(k, adj, &na);
    if (!aut) return na < 0 ? na : ORC_ENOMEM;
    a4_ctx c = {k, adj, out, cap, 0};
    int32_t sched[ORC_MAXK];
    a4_rec(&c, sched, 0, aut, na, 0);
    free(aut);
    return c.cnt;
}

/*
 * Restriction pass probability of loops 0..d (Appendix): prod over i <= d of
 * 1/z_i where z_i counts the positions j <= d with e_j forced below or equal
 * to e_i, i.e. i's subtree in the forest of bound parents, cut at d.
 */
double orc_restriction_probability(int k, const int32_t* bp, int d) {
    double pr = 1.0;
    for (int i = 0; i <= d && i < k; ++i) {
        int z = 0;
        for (int j = 0; j <= d; ++j) {
            int a = j;
            while (a >= 0 && a != i) a = bp[a];
            if (a == i) ++z;
        }
        pr /= (double)z;
    }
    return pr;
}

/* Performance model of Sec. 5.4 for one schedule (labels). */
double orc_cost(int k, const uint8_t* adj, const int32_t* order) {
    int32_t bp[ORC_MAXK];
    if (orc_restrictions(k, adj, order, bp, NULL, 0) < 0) return -1.0;
    const double n = 1000.0, p = 5.0 / 999.0;
    double prod = 1.0, cost = 0.0;
    for (int d = 0; d < k; ++d) {
        double iters = n;
        if (d > 0) {
            int nb = 0, nr = 0;
            for (int j = 0; j < d; ++j) {
                if (adj[order[d] * k + order[j]]) ++nb; else ++nr;
            }
            if (g_mut == MUT_COST_NO_DIFF) nr = 0;
            if (g_mut == MUT_COST_EXP) ++nb;
            iters = n * pow(p, (double)nb) * pow(1.0 - p, (double)nr);
        }
        prod *= iters;
        if (g_mut == MUT_COST_PRODUCT)
            cost = (d == 0 ? 1.0 : cost) * prod * orc_restriction_probability(k, bp, d);
        else
            cost += prod * orc_restriction_probability(k, bp, d);
    }
    return cost;
}

/* The schedule the model picks: the cheapest of Algorithm 4's, first on ties. */
int orc_choose_schedule(int k, const uint8_t* adj, int32_t* order_out, double* cost_out) {
    int ns = orc_distinct_schedules(k, adj, NULL, 0);
    if (ns <= 0) return ns < 0 ? ns : ORC_EINVAL;
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)ns * k);
    if (!s) return ORC_ENOMEM;
    orc_distinct_schedules(k, adj, s, ns);
    int best = 0;
    double bc = orc_cost(k, adj, s);
    for (int i = 1; i < ns; ++i) {
        double c = orc_cost(k, adj, s + (size_t)i * k);
        if (c < bc * (1.0 - 1e-12)) { bc = c; best = i; }
    }
    memcpy(order_out, s + (size_t)best * k, sizeof(int32_t) * k);
    if (cost_out) *cost_out = bc;
    free(s);
    return 0;
}

/* --------------------------------------------------------------- Oracle A */

static int g_has_edge(const int64_t* rp, const int32_t* col, int32_t u, int32_t v) {
    for (int64_t i = rp[u]; i < rp[u + 1]; ++i) if (col[i] == v) return 1;
    return 0;
}

/* Dense adjacency for a tiny graph (n <= 64). */
static uint8_t* dense(int64_t n, const int64_t* rp, const int32_t* col) {
    uint8_t* m = (uint8_t*)calloc((size_t)(n * n > 0 ? n * n : 1), 1);
    if (!m) return NULL;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t i = rp[v]; i < rp[v + 1]; ++i) m[v * n + col[i]] = 1;
    return m;
}

/* #{k-subsets U : G[U] isomorphic to P}; tiny graphs only (n <= 64). */
int orc_count_brute_induced(int k, const uint8_t* adj, int64_t n, const int64_t* rp,
                            const int32_t* col, uint64_t* out) {
    if (!pattern_ok(k, adj) || n < 0 || n > 64) return ORC_EINVAL;
    *out = 0;
    if (n < k) return 0;
    uint8_t* g = dense(n, rp, col);
    if (!g) return ORC_ENOMEM;
    int32_t U[ORC_MAXK];
    for (int i = 0; i < k; ++i) U[i] = i;
    uint64_t cnt = 0;
    for (;;) {
        int32_t p[ORC_MAXK];
        for (int i = 0; i < k; ++i) p[i] = i;
        int match = 0;
        do {
            int ok = 1;
            for (int i = 0; i < k && ok; ++i)
                for (int j = i + 1; j < k; ++j)
                    if ((adj[i * k + j] != 0) != (g[U[p[i]] * n + U[p[j]]] != 0)) { ok = 0; break; }
            if (ok) { match = 1; break; }
        } while (next_perm(p, k));
        cnt += (uint64_t)match;
        int i = k - 1;
        while (i >= 0 && U[i] == n - k + i) --i;
        if (i < 0) break;
        ++U[i];
        for (int j = i + 1; j < k; ++j) U[j] = U[j - 1] + 1;
    }
    free(g);
    *out = cnt;
    return 0;
}

/* #{injective phi preserving edges and non-edges}; tiny graphs only. */
int orc_count_brute_injective(int k, const uint8_t* adj, int64_t n, const int64_t* rp,
                              const int32_t* col, uint64_t* out) {
    if (!pattern_ok(k, adj) || n < 0 || n > 64) return ORC_EINVAL;
    *out = 0;
    if (n < k) return 0;
    uint8_t* g = dense(n, rp, col);
    if (!g) return ORC_ENOMEM;
    int32_t phi[ORC_MAXK];
    for (int i = 0; i < k; ++i) phi[i] = 0;
    uint64_t cnt = 0;
    for (;;) {
        int ok = 1;
        for (int i = 0; i < k && ok; ++i)
            for (int j = i + 1; j < k; ++j) {
                if (phi[i] == phi[j]) { ok = 0; break; }
                if ((adj[i * k + j] != 0) != (g[phi[i] * n + phi[j]] != 0)) { ok = 0; break; }
            }
        cnt += (uint64_t)ok;
        int i = k - 1;
        while (i >= 0 && phi[i] == n - 1) { phi[i] = 0; --i; }
        if (i < 0) break;
        ++phi[i];
    }
    free(g);
    *out = cnt;
    return 0;
}

/* --------------------------------------------------------------- Oracle B */

typedef struct {
    int k;
    int black[ORC_MAXK][ORC_MAXK]; /* black[d][j]: pattern edge between positions d and j */
    int bp[ORC_MAXK];
    const int64_t* rp;
    const int32_t* col;
} nplan;

static int prepare(nplan* pl, int k, const uint8_t* adj, const int32_t* order) {
    if (orc_restrictions(k, adj, order, pl->bp, NULL, 0) < 0) return ORC_EINVAL;
    pl->k = k;
    for (int d = 0; d < k; ++d)
        for (int j = 0; j < k; ++j) pl->black[d][j] = adj[order[d] * k + order[j]] != 0;
    return 0;
}

static inline int below(int32_t u, int32_t bound, int bounded) {
    if (!bounded) return 1;
    if (g_mut == MUT_BOUND_LE) return u <= bound;
    return u < bound;
}

/* Number of elements of sorted L[0, len) below bound (all of them if unbounded). */
static int64_t count_below(const int32_t* L, int64_t len, int32_t bound, int bounded) {
    if (!bounded) return len;
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (L[mid] < bound) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * E of the last loop without building its sets: every c in S_{k-2} (already
 * built, matched vertices removed) is one partial embedding of the last loop,
 * which adds sum_{j<k-1} |N(e_j) intersect [0, bound_{k-1})| with e_{k-2} = c.
 */
static void last_level_elems(const nplan* pl, int32_t* emb, const int32_t* S, int64_t n,
                             uint64_t* el) {
    const int k = pl->k, d = k - 1;
    const int bounded = pl->bp[d] >= 0 && g_mut != MUT_NO_BOUND;
    for (int64_t i = 0; i < n; ++i) {
        emb[k - 2] = S[i];
        int32_t bound = pl->bp[d] >= 0 ? emb[pl->bp[d]] : 0;
        for (int j = 0; j < d; ++j) {
            const int32_t* L = pl->col + pl->rp[emb[j]];
            int64_t len = pl->rp[emb[j] + 1] - pl->rp[emb[j]];
            *el += (uint64_t)count_below(L, len, bound, bounded);
        }
    }
}

/* One level of the nested loops: build S_d from scratch, then recurse or count.
 * With elems_only set, the last loop only adds its E (no count is produced). */
static void nested_level(const nplan* pl, int d, int32_t* emb, int32_t** buf, int32_t* tmp,
                         uint64_t* cnt, uint64_t* el, int elems_only) {
    const int k = pl->k;
    int bounded = pl->bp[d] >= 0 && g_mut != MUT_NO_BOUND;
    int32_t bound = pl->bp[d] >= 0 ? emb[pl->bp[d]] : 0;
    /* E: the bounded part of every predecessor's list */
    for (int j = 0; j < d; ++j) {
        const int32_t* L = pl->col + pl->rp[emb[j]];
        int64_t len = pl->rp[emb[j] + 1] - pl->rp[emb[j]];
        if (g_mut == MUT_E_FULL) { *el += (uint64_t)len; continue; }
        for (int64_t i = 0; i < len && below(L[i], bound, bounded); ++i) ++*el;
    }
    int j0 = -1;
    for (int j = 0; j < d; ++j) if (pl->black[d][j]) { j0 = j; break; }
    int32_t* S = buf[d];
    int64_t n = 0;
    {
        const int32_t* L = pl->col + pl->rp[emb[j0]];
        int64_t len = pl->rp[emb[j0] + 1] - pl->rp[emb[j0]];
        for (int64_t i = 0; i < len && below(L[i], bound, bounded); ++i) S[n++] = L[i];
    }
    for (int j = 0; j < d; ++j) {
        if (j == j0) continue;
        const int32_t* L = pl->col + pl->rp[emb[j]];
        int64_t len = pl->rp[emb[j] + 1] - pl->rp[emb[j]];
        int black = pl->black[d][j];
        if (!black && g_mut == MUT_DROP_RED) continue;
        /* two-pointer merge of sorted S with sorted L */
        int64_t a = 0, b = 0, w = 0;
        while (a < n) {
            while (b < len && L[b] < S[a]) ++b;
            int found = b < len && L[b] == S[a];
            if (found == black) tmp[w++] = S[a];
            ++a;
        }
        memcpy(S, tmp, sizeof(int32_t) * (size_t)w);
        n = w;
    }
    if (g_mut != MUT_NO_EXCLUDE) {
        int64_t w = 0;
        for (int64_t i = 0; i < n; ++i) {
            int dup = 0;
            for (int j = 0; j < d; ++j) dup |= S[i] == emb[j];
            if (!dup) S[w++] = S[i];
        }
        n = w;
    }
    if (d == k - 1) { *cnt += (uint64_t)n; return; }
    if (elems_only && d == k - 2) { last_level_elems(pl, emb, S, n, el); return; }
    for (int64_t i = 0; i < n; ++i) {
        emb[d] = S[i];
        nested_level(pl, d + 1, emb, buf, tmp, cnt, el, elems_only);
    }
}

/*
 * Oracle B: count instances of P (labels adj, schedule `order`) whose first
 * scheduled vertex lies in [root_lo, root_hi), and the element count E of
 * those roots. threads <= 0 uses the OpenMP default.
 */
static int nested_run(int k, const uint8_t* adj, const int32_t* order, int64_t n,
                      const int64_t* rp, const int32_t* col, int64_t root_lo, int64_t root_hi,
                      int threads, uint64_t* count_out, uint64_t* elems_out, int elems_only);

int orc_count_nested(int k, const uint8_t* adj, const int32_t* order, int64_t n,
                     const int64_t* rp, const int32_t* col, int64_t root_lo, int64_t root_hi,
                     int threads, uint64_t* count_out, uint64_t* elems_out) {
    return nested_run(k, adj, order, n, rp, col, root_lo, root_hi, threads, count_out, elems_out, 0);
}

/*
 * E only (the same value orc_count_nested reports), skipping the construction
 * of the last loop's sets: their E needs only the bounded list lengths. For
 * workloads whose last loop is too large for the plain count.
 */
int orc_elems_nested(int k, const uint8_t* adj, const int32_t* order, int64_t n,
                     const int64_t* rp, const int32_t* col, int64_t root_lo, int64_t root_hi,
                     int threads, uint64_t* elems_out) {
    uint64_t c = 0;
    if (k < 3) return nested_run(k, adj, order, n, rp, col, root_lo, root_hi, threads, &c, elems_out, 0);
    return nested_run(k, adj, order, n, rp, col, root_lo, root_hi, threads, &c, elems_out, 1);
}

static int nested_run(int k, const uint8_t* adj, const int32_t* order, int64_t n,
                      const int64_t* rp, const int32_t* col, int64_t root_lo, int64_t root_hi,
                      int threads, uint64_t* count_out, uint64_t* elems_out, int elems_only) {
    nplan pl;
    if (!pattern_ok(k, adj) || prepare(&pl, k, adj, order) < 0) return ORC_EINVAL;
    if (root_lo < 0) root_lo = 0;
    if (root_hi > n) root_hi = n;
    pl.rp = rp; pl.col = col;
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) if (rp[v + 1] - rp[v] > maxdeg) maxdeg = rp[v + 1] - rp[v];
    uint64_t cnt = 0, el = 0;
    int err = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel reduction(+ : cnt, el)
    {
        int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)(maxdeg + 1) * (k + 1));
        int32_t* buf[ORC_MAXK];
        if (!mem) {
#pragma omp atomic write
            err = 1;
        } else {
            for (int d = 0; d < k; ++d) buf[d] = mem + (size_t)d * (maxdeg + 1);
            int32_t* tmp = mem + (size_t)k * (maxdeg + 1);
            int32_t emb[ORC_MAXK];
#pragma omp for schedule(dynamic, 16)
            for (int64_t v = root_lo; v < root_hi; ++v) {
                emb[0] = (int32_t)v;
                if (elems_only && k - 2 == 0) {
                    /* loop 1 is the last loop: its one partial embedding is (e_0) */
                    int bounded = pl.bp[1] >= 0 && g_mut != MUT_NO_BOUND;
                    el += (uint64_t)count_below(col + rp[v], rp[v + 1] - rp[v], (int32_t)v, bounded);
                } else {
                    nested_level(&pl, 1, emb, buf, tmp, &cnt, &el, elems_only);
                }
            }
            free(mem);
        }
    }
    if (err) return ORC_ENOMEM;
    *count_out = cnt;
    if (elems_out) *elems_out = el;
    return 0;
}

/*
 * E by brute force (tiny graphs): walk every tuple (e_0..e_{d-1}) of V^d that
 * satisfies levels 1..d-1 by direct adjacency tests, distinctness and the one
 * bound per level, and add sum_{j<d} |N(e_j) intersect [0, bound_d)|.
 */
int orc_elems_brute(int k, const uint8_t* adj, const int32_t* order, int64_t n,
                    const int64_t* rp, const int32_t* col, uint64_t* out) {
    nplan pl;
    if (!pattern_ok(k, adj) || prepare(&pl, k, adj, order) < 0 || n > 64) return ORC_EINVAL;
    uint8_t* g = dense(n, rp, col);
    if (!g) return ORC_ENOMEM;
    uint64_t el = 0;
    for (int d = 1; d < k; ++d) {
        int32_t e[ORC_MAXK];
        uint64_t total = 1;
        for (int i = 0; i < d; ++i) total *= (uint64_t)n;
        for (uint64_t code = 0; code < total; ++code) {
            uint64_t c = code;
            for (int i = 0; i < d; ++i) { e[i] = (int32_t)(c % (uint64_t)n); c /= (uint64_t)n; }
            int ok = 1;
            for (int t = 1; t < d && ok; ++t) {
                for (int j = 0; j < t; ++j) {
                    if (e[t] == e[j]) { ok = 0; break; }
                    if ((g[e[t] * n + e[j]] != 0) != (pl.black[t][j] != 0)) { ok = 0; break; }
                }
                if (ok && pl.bp[t] >= 0 && !(e[t] < e[pl.bp[t]])) ok = 0;
            }
            if (!ok) continue;
            for (int j = 0; j < d; ++j)
                for (int64_t i = rp[e[j]]; i < rp[e[j] + 1]; ++i)
                    if (pl.bp[d] < 0 || col[i] < e[pl.bp[d]]) ++el;
        }
    }
    free(g);
    *out = el;
    return 0;
}

/* ------------------------------------------------------------- orientation */

static const int64_t* g_sort_deg;
static int cmp_rank(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    int64_t dx = g_sort_deg[x], dy = g_sort_deg[y];
    if (dx != dy) {
        if (g_mut == MUT_REINDEX_ASC) return dx < dy ? -1 : 1;
        return dx > dy ? -1 : 1; /* higher degree first */
    }
    return (x > y) - (x < y); /* ties: original id ascending */
}
static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Sec. 6 reindexing: new_id(v) = rank of v by (degree descending, original id
 * ascending). Writes the relabelled CSR (lists re-sorted) and new_id[].
 */
int orc_reindex(int64_t n, const int64_t* rp, const int32_t* col, int64_t* rp_out,
                int32_t* col_out, int32_t* new_id) {
    int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!deg || !order) { free(deg); free(order); return ORC_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) { deg[v] = rp[v + 1] - rp[v]; order[v] = (int32_t)v; }
    g_sort_deg = deg;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_rank);
    for (int64_t r = 0; r < n; ++r) new_id[order[r]] = (int32_t)r;
    rp_out[0] = 0;
    for (int64_t r = 0; r < n; ++r) rp_out[r + 1] = rp_out[r] + deg[order[r]];
    for (int64_t r = 0; r < n; ++r) {
        int32_t v = order[r];
        int32_t* dst = col_out + rp_out[r];
        for (int64_t i = rp[v]; i < rp[v + 1]; ++i) dst[i - rp[v]] = new_id[col[i]];
        qsort(dst, (size_t)deg[v], sizeof(int32_t), cmp_i32);
    }
    free(deg); free(order);
    return 0;
}

/* Edge test used by the tests' structural checks. */
int orc_has_edge(const int64_t* rp, const int32_t* col, int32_t u, int32_t v) {
    return g_has_edge(rp, col, u, v);
}

/* -------------------------------------------------- bitset work measure */

/*
 * Work measure of the oriented k-clique count in bitset form. It is used to
 * state a roofline for kernels that keep each root's candidate sets as
 * bitsets; it is not part of the method, and no count the tests compare comes
 * from it.
 *
 * On the degree-reindexed graph (Sec. 6) a k-clique's schedule bounds each
 * loop by the one before it, so e_1, e_2, ... all lie in the root's out-list
 * O = N(e_0) intersect [0, e_0), sorted. Relative to O, row(a) is the bitset
 * {b < a : O[b] in N(O[a])}. Loop 2's candidate set for (e_1, e_2) = (O[a],
 * O[b]) is row(a) AND row(b); each deeper loop ANDs the row of the index just
 * chosen, and the last loop counts the set's bits. A set whose newest row is
 * row(lim) holds bits below lim only, so it spans ceil(lim / 32) 32-bit words.
 * One "word operation" produces one such word (the AND of the rows in it, then
 * either a popcount or a walk over its bits). words_out sums, over every pair
 * (a, b in row(a)) and every deeper partial clique, the words of the set it
 * builds; building the rows and the loop over a are not included. count_out
 * is the number of k-cliques the walk finds, which checks the walk against the
 * plain count. Roots with |O| < k - 1 are skipped (they hold no k-clique).
 * Graph: the reindexed CSR; roots in [root_lo, root_hi); 4 <= k <= 8.
 */
static void bits_level(const uint32_t* rows, int64_t W, const uint32_t* set, int32_t lim,
                       int depth, uint32_t* scratch, uint64_t* words, uint64_t* cnt) {
    const int64_t nw = ((int64_t)lim + 31) / 32;
    *words += (uint64_t)nw;
    if (depth == 1) {
        for (int64_t w = 0; w < nw; ++w) *cnt += (uint64_t)__builtin_popcount(set[w]);
        return;
    }
    uint32_t* next = scratch;
    for (int64_t w = 0; w < nw; ++w) {
        uint32_t bits = set[w];
        while (bits) {
            const int32_t c = (int32_t)(w * 32 + __builtin_ctz(bits));
            bits &= bits - 1;
            const uint32_t* rc = rows + (size_t)c * W;
            const int64_t cw = ((int64_t)c + 31) / 32;
            for (int64_t x = 0; x < cw; ++x) next[x] = set[x] & rc[x];
            bits_level(rows, W, next, c, depth - 1, scratch + W, words, cnt);
        }
    }
}

int orc_clique_bitset_work(int k, int64_t n, const int64_t* rp, const int32_t* col,
                           int64_t root_lo, int64_t root_hi, int threads, uint64_t* count_out,
                           uint64_t* words_out) {
    if (k < 4 || k > ORC_MAXK) return ORC_EINVAL;
    if (root_lo < 0) root_lo = 0;
    if (root_hi > n) root_hi = n;
    int64_t maxout = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = 0;
        for (int64_t i = rp[v]; i < rp[v + 1] && col[i] < v; ++i) ++d;
        if (d > maxout) maxout = d;
    }
    const int64_t Wmax = (maxout + 31) / 32 + 1;
    uint64_t cnt = 0, words = 0;
    int err = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel reduction(+ : cnt, words)
    {
        uint32_t* rows = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(maxout + 1) * Wmax);
        uint32_t* scratch = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(k + 1) * Wmax);
        if (!rows || !scratch) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t v = root_lo; v < root_hi; ++v) {
                const int32_t* O = col + rp[v];
                int64_t d = 0;
                while (rp[v] + d < rp[v + 1] && O[d] < v) ++d;
                if (d < k - 1) continue;
                const int64_t W = (d + 31) / 32;
                memset(rows, 0, sizeof(uint32_t) * (size_t)d * W);
                /* row(a): merge O[0, a) with the out-list of O[a] (both sorted) */
                for (int64_t a = 1; a < d; ++a) {
                    const int32_t u = O[a];
                    int64_t i = rp[u], b = 0;
                    while (i < rp[u + 1] && col[i] < u && b < a) {
                        if (col[i] < O[b]) ++i;
                        else if (col[i] > O[b]) ++b;
                        else { rows[a * W + b / 32] |= 1u << (b % 32); ++i; ++b; }
                    }
                }
                uint32_t* set = scratch;
                for (int64_t a = 1; a < d; ++a) {
                    const uint32_t* ra = rows + a * W;
                    for (int64_t wb = 0; wb < (a + 31) / 32; ++wb) {
                        uint32_t bits = ra[wb];
                        while (bits) {
                            const int32_t b = (int32_t)(wb * 32 + __builtin_ctz(bits));
                            bits &= bits - 1;
                            const uint32_t* rb = rows + (size_t)b * W;
                            for (int64_t x = 0; x < (b + 31) / 32; ++x) set[x] = ra[x] & rb[x];
                            bits_level(rows, W, set, b, k - 3, scratch + Wmax, &words, &cnt);
                        }
                    }
                }
            }
        }
        free(rows);
        free(scratch);
    }
    if (err) return ORC_ENOMEM;
    *count_out = cnt;
    *words_out = words;
    return 0;
}

/* -------------------------------------------------------------- motifs */

/* Adjacency string of graph m (k x k) relabelled by p: s[i*k + j] = m[p[i]][p[j]]. */
static void relabel(int k, const uint8_t* m, const int32_t* p, uint8_t* s) {
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) s[i * k + j] = m[p[i] * k + p[j]];
}

/*
 * Every connected graph on k vertices up to isomorphism (the motif patterns of
 * Sec. 7.1-7.2), plainly: each edge subset of K_k that is connected is put in its
 * canonical form, the lexicographically largest adjacency string over all k!
 * relabellings, and kept if that form is new. Writes up to cap canonical
 * adjacencies (k*k bytes each) in order of discovery; returns how many.
 */
int orc_connected_patterns(int k, uint8_t* out, int cap) {
    if (k < 2 || k > 6) return ORC_EINVAL;
    const int ne = k * (k - 1) / 2;
    int ei[15], ej[15], t = 0;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) { ei[t] = i; ej[t] = j; ++t; }
    uint8_t* forms = (uint8_t*)malloc((size_t)200 * k * k);
    if (!forms) return ORC_ENOMEM;
    int nf = 0;
    uint8_t m[36], best[36], cur[36];
    for (long e = 0; e < (1L << ne); ++e) {
        memset(m, 0, sizeof(m));
        for (int b = 0; b < ne; ++b)
            if (e >> b & 1) m[ei[b] * k + ej[b]] = m[ej[b] * k + ei[b]] = 1;
        if (!pattern_ok(k, m)) continue; /* connected (and symmetric, loop-free) */
        int32_t p[ORC_MAXK];
        for (int i = 0; i < k; ++i) p[i] = i;
        int have = 0;
        do {
            relabel(k, m, p, cur);
            if (!have || memcmp(cur, best, (size_t)k * k) > 0) { memcpy(best, cur, (size_t)k * k); have = 1; }
        } while (next_perm(p, k));
        int dup = 0;
        for (int f = 0; f < nf && !dup; ++f) dup = memcmp(forms + (size_t)f * k * k, best, (size_t)k * k) == 0;
        if (dup) continue;
        if (nf >= 200) { free(forms); return ORC_ECAP; }
        memcpy(forms + (size_t)nf * k * k, best, (size_t)k * k);
        if (out && nf < cap) memcpy(out + (size_t)nf * k * k, best, (size_t)k * k);
        ++nf;
    }
    free(forms);
    return nf;
}

/* Canonical form (as above) of one k-vertex graph, written to out (k*k bytes). */
int orc_canonical_form(int k, const uint8_t* adj, uint8_t* out) {
    if (k < 1 || k > ORC_MAXK) return ORC_EINVAL;
    int32_t p[ORC_MAXK];
    for (int i = 0; i < k; ++i) p[i] = i;
    uint8_t cur[ORC_MAXK * ORC_MAXK];
    int have = 0;
    do {
        relabel(k, adj, p, cur);
        if (!have || memcmp(cur, out, (size_t)k * k) > 0) { memcpy(out, cur, (size_t)k * k); have = 1; }
    } while (next_perm(p, k));
    return 0;
}
