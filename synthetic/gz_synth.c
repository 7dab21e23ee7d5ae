/*
 * gz_synth.c - seeded synthetic graph generators (Erdos-Renyi and R-MAT).
 *
 * This module only builds inputs. It holds none of the counting method's
 * arithmetic (no patterns, restrictions, orientation or set operations). Both
 * the CUDA path and the CPU oracle read the graphs it writes, so their inputs
 * are identical by construction.
 *
 * Output format: an undirected simple graph as CSR, row_ptr int64[n+1] and
 * col int32[nnz], every list sorted ascending, no duplicates, no self-loops,
 * symmetric (u in N(v) <=> v in N(u)).
 *
 * Randomness: one counter-based generator, splitmix64's finaliser applied to
 * (seed, stream, counter), so every draw is a pure function of its indices and
 * the result does not depend on the thread count or the machine.
 *
 * The R-MAT recipe follows Chakrabarti, Zhan and Faloutsos (SDM 2004): each
 * of ef * 2^scale samples picks one of four quadrants per bit level with
 * probabilities (a, b, c, d), no noise. A seeded random relabelling of the
 * vertex ids follows (as Graph500 does) so that low ids are not hubs, then the
 * edge list is symmetrised, self-loops dropped, duplicates removed and each
 * list sorted. Isolated vertices are kept (n = 2^scale).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GZS_OK 0
#define GZS_EINVAL -1
#define GZS_ENOMEM -2

/* splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014). */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* One draw of the counter-based stream: a pure function of its three indices. */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return mix64(mix64(seed ^ mix64(stream + 0x632BE59BD9B4E019ULL)) + ctr);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unif(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Builds a symmetric simple CSR from an undirected edge list (src[i], dst[i]).
 * Self-loops are dropped and duplicates merged. On success *row_ptr_out and
 * *col_out are malloc'd and owned by the caller (free with gzs_free).
 */
static int build_csr(int64_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                     int64_t** row_ptr_out, int32_t** col_out, int64_t* nnz_out) {
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return GZS_ENOMEM;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; ++i) {
        int32_t u = src[i], v = dst[i];
        if (u == v) continue;
        __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
    }
    int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!off) { free(deg); return GZS_ENOMEM; }
    off[0] = 0;
    for (int64_t v = 0; v < n; ++v) off[v + 1] = off[v] + deg[v];
    int64_t total = off[n];
    int32_t* buf = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!buf) { free(deg); free(off); return GZS_ENOMEM; }
    memcpy(deg, off, (size_t)n * sizeof(int64_t)); /* deg[] becomes the fill cursor */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; ++i) {
        int32_t u = src[i], v = dst[i];
        if (u == v) continue;
        int64_t pu = __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
        int64_t pv = __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
        buf[pu] = v;
        buf[pv] = u;
    }
    /* sort and deduplicate each list in place; deg[v] = unique count */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t v = 0; v < n; ++v) {
        int32_t* l = buf + off[v];
        int64_t len = off[v + 1] - off[v];
        if (len > 1) qsort(l, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t w = 0;
        for (int64_t i = 0; i < len; ++i)
            if (w == 0 || l[i] != l[w - 1]) l[w++] = l[i];
        deg[v] = w;
    }
    int64_t* rp = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!rp) { free(deg); free(off); free(buf); return GZS_ENOMEM; }
    rp[0] = 0;
    for (int64_t v = 0; v < n; ++v) rp[v + 1] = rp[v] + deg[v];
    int64_t nnz = rp[n];
    int32_t* col = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!col) { free(deg); free(off); free(buf); free(rp); return GZS_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v)
        memcpy(col + rp[v], buf + off[v], (size_t)deg[v] * sizeof(int32_t));
    free(deg); free(off); free(buf);
    *row_ptr_out = rp; *col_out = col; *nnz_out = nnz;
    return GZS_OK;
}

void gzs_free(void* p) { free(p); }

int gzs_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * G(n, p): every unordered pair {i, j}, i < j, is an edge independently with
 * probability p. Pair (i, j) uses counter i * n + j of stream 1. O(n^2) work,
 * meant for n up to a few tens of thousands.
 */
int gzs_erdos_renyi(int64_t n, double p, uint64_t seed, int64_t** row_ptr, int32_t** col,
                    int64_t* nnz) {
    if (n < 0 || n > (1LL << 20) || !(p >= 0.0 && p <= 1.0)) return GZS_EINVAL;
    int64_t cap = 1024, ne = 0;
    int32_t* s = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    int32_t* d = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    if (!s || !d) { free(s); free(d); return GZS_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            if (unif(draw(seed, 1, (uint64_t)(i * n + j))) < p) {
                if (ne == cap) {
                    cap *= 2;
                    int32_t* s2 = (int32_t*)realloc(s, (size_t)cap * sizeof(int32_t));
                    int32_t* d2 = (int32_t*)realloc(d, (size_t)cap * sizeof(int32_t));
                    if (!s2 || !d2) { free(s2 ? s2 : s); free(d2 ? d2 : d); return GZS_ENOMEM; }
                    s = s2; d = d2;
                }
                s[ne] = (int32_t)i; d[ne] = (int32_t)j; ++ne;
            }
        }
    }
    int rc = build_csr(n, ne, s, d, row_ptr, col, nnz);
    free(s); free(d);
    return rc;
}

/*
 * R-MAT with 2^scale vertices and ef * 2^scale samples. Sample t, bit level b
 * draws counter t * 64 + b of stream 2; the relabelling permutation is a
 * Fisher-Yates shuffle driven by stream 3.
 */
int gzs_rmat(int scale, int64_t ef, double a, double b, double c, uint64_t seed,
             int64_t** row_ptr, int32_t** col, int64_t* nnz) {
    if (scale < 1 || scale > 30 || ef < 0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0)
        return GZS_EINVAL;
    int64_t n = 1LL << scale;
    int64_t ns = ef * n;
    int32_t* s = (int32_t*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int32_t));
    int32_t* d = (int32_t*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int32_t));
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!s || !d || !perm) { free(s); free(d); free(perm); return GZS_ENOMEM; }
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < ns; ++t) {
        int64_t u = 0, v = 0;
        for (int lvl = 0; lvl < scale; ++lvl) {
            double r = unif(draw(seed, 2, (uint64_t)t * 64u + (uint64_t)lvl));
            int bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        s[t] = (int32_t)u; d[t] = (int32_t)v;
    }
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t j = draw(seed, 3, (uint64_t)i) % (uint64_t)(i + 1);
        int32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < ns; ++t) { s[t] = perm[s[t]]; d[t] = perm[d[t]]; }
    free(perm);
    int rc = build_csr(n, ns, s, d, row_ptr, col, nnz);
    free(s); free(d);
    return rc;
}

/* CSR from a caller-provided undirected edge list (small structured graphs). */
int gzs_from_edges(int64_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                   int64_t** row_ptr, int32_t** col, int64_t* nnz) {
    if (n < 0 || ne < 0) return GZS_EINVAL;
    for (int64_t i = 0; i < ne; ++i)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return GZS_EINVAL;
    return build_csr(n, ne, src, dst, row_ptr, col, nnz);
}
