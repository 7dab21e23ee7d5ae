// gz_clique.cu - k-clique counting (4 <= k <= 8) on the out-list view, the
// orientation special case of GraphZero's restrictions (Sec. 6): a clique's
// schedule bounds every loop by the previous one (e_0 > e_1 > ... > e_{k-1}),
// so all of e_1.. lie in O = N(e_0) intersect [0, e_0), the root's out-list.
//
// The nested loops keep their order and their bounds, but the sets they
// intersect are represented relative to O: row(a) is the bitset of indices
// b < a with O[b] in N(O[a]) (O is sorted, so O[b] < O[a] iff b < a, and the
// loop bound e_{j+1} < e_j becomes "bits below the current index"). Loop 2's
// set for (e_1, e_2) = (O[a], O[b]) is row(a) & row(b); each deeper loop ANDs
// one more row; the last loop is a popcount. Counts are exact.
//
//  - k_clique_small: one warp per root with |O| <= 32 (one 32-bit row per lane's
//    vertex, rows in shared memory).
//  - k_clique_rows: the rows of every root with 32 < |O| <= kCliqueMaxOut,
//    built once per out-list view into device memory and kept there; the
//    kernels below copy them into shared memory.
//  - k_clique_warp (K = 4, 5): one 512-thread CTA per root, its warps taking
//    the rows a of the root dynamically and the pairs (a, b) one per lane.
//  - k_clique_big (K >= 6): one 512-thread CTA per root or per part of a root
//    (roots with |O| >= kSplitD are split over several CTAs), rows in shared
//    memory with an odd word stride, the (a, b) edges of the local DAG spread
//    over all threads.
//  - k_clique_long: roots with kCliqueMaxOut < |O| <= kCliqueLongOut, rows in
//    device memory (k_clique_long_rows); longer roots are left to the caller.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <vector>

#include "gz_internal.h"

namespace gz {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kBigPop = 16;     // roots per queue slot of the big kernel; most are skipped
constexpr int kBigThreads = 512;  // threads of a big-kernel CTA (one root at a time)
constexpr int kHeavyD = 33;     // out-degree from which a root's rows are built once and cached
constexpr int kSplitD = 128;    // out-degree from which k_clique_big splits a root over several CTAs
constexpr uint64_t kHeavyRowWords = 1ull << 29;  // budget for prebuilt heavy rows (2 GiB)
constexpr uint64_t kLongRowWords = 1ull << 30;   // budget for long roots' global rows (4 GiB)

// Row stride (32-bit words) of the bitset rows of a root with d out-neighbours,
// kept in shared memory and in the prebuilt heavy rows: ceil(d / 32) words
// rounded up to whole 16-byte chunks, with an odd chunk count, so rows start on
// 16-byte boundaries (128-bit loads) and the same chunk of consecutive rows
// falls in different bank groups.
__host__ __device__ __forceinline__ int row_stride(int d) {
    const int chunks = (((d + 31) >> 5) + 3) >> 2;
    return (chunks | 1) << 2;
}

__device__ __forceinline__ bool has(const int32_t* __restrict__ R, int n, int32_t x) {
    int lo = 0, len = n;
    while (len > 0) {
        int half = len >> 1;
        if (__ldg(R + lo + half) < x) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo < n && __ldg(R + lo) == x;
}

// Index of x in sorted O[0, n) or -1 (shared memory).
__device__ __forceinline__ int index_of(const int32_t* O, int n, int32_t x) {
    int lo = 0, len = n;
    while (len > 0) {
        int half = len >> 1;
        if (O[lo + half] < x) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return (lo < n && O[lo] == x) ? lo : -1;
}

// Sum over the cliques that extend the set AND(rs[0..NR)) (bits < lim) by
// DEPTH more vertices, each below the previous one; DEPTH == 1 is a popcount.
// NR is a template parameter so the row pointers stay in registers and the
// AND over them unrolls; the popcount loop sums in 32 bits (at most lim).
template <int DEPTH, int NR>
__device__ __forceinline__ unsigned long long extend(const uint32_t* rows, int W,
                                                     const uint32_t* const* rs, int lim) {
    const int words = (lim + 31) >> 5;
    if constexpr (DEPTH == 1) {
        uint32_t cnt = 0;
        for (int w = 0; w < words; ++w) {
            uint32_t s = rs[0][w];
#pragma unroll
            for (int i = 1; i < NR; ++i) s &= rs[i][w];
            cnt += __popc(s);
        }
        return cnt;
    } else {
        unsigned long long cnt = 0;
        const uint32_t* rn[NR + 1];
#pragma unroll
        for (int i = 0; i < NR; ++i) rn[i] = rs[i];
        for (int w = 0; w < words; ++w) {
            uint32_t s = rs[0][w];
#pragma unroll
            for (int i = 1; i < NR; ++i) s &= rs[i][w];
            while (s) {
                const int c = (w << 5) + __ffs(s) - 1;
                s &= s - 1;
                rn[NR] = rows + (size_t)c * W;
                cnt += extend<DEPTH - 1, NR + 1>(rows, W, rn, c);
            }
        }
        return cnt;
    }
}

template <int K>
__device__ __forceinline__ unsigned long long count_pair(const uint32_t* rows, int W, int a, int b) {
    const uint32_t* rs[2] = {rows + (size_t)a * W, rows + (size_t)b * W};
    return extend<K - 3, 2>(rows, W, rs, b);
}

__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// Roots with 1 <= |O| <= 32: one warp per root, dynamic root queue.
// count4 (K = 5 only, else NULL): the fused K4 + K5 pass also adds each pair's
// K4 count |row(a) & row(b)| there.
template <int K>
__global__ void __launch_bounds__(kThreads) k_clique_small(const int64_t* __restrict__ drp,
                                                           const int32_t* __restrict__ dcol,
                                                           int64_t root_lo, int64_t root_hi,
                                                           unsigned long long* __restrict__ work,
                                                           unsigned long long* __restrict__ count,
                                                           unsigned long long* __restrict__ count4) {
    __shared__ uint32_t rows_s[kThreads / 32][32];
    __shared__ unsigned long long red[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* rows = rows_s[warp];
    unsigned long long acc = 0, acc4 = 0;
    const int dmin = count4 ? 3 : K - 1;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(work, 32ull);
        base = __shfl_sync(kFull, base, 0);
        if ((int64_t)(root_lo + base) >= root_hi) break;
        // 32 roots per pop; the warp walks them one at a time
        for (int r = 0; r < 32; ++r) {
            const int64_t v = root_lo + (int64_t)base + r;
            if (v >= root_hi) break;
            const int64_t ob = drp[v];
            const int d = (int)(drp[v + 1] - ob);
            if (d < dmin || d > 32) continue;
            const int32_t u = lane < d ? dcol[ob + lane] : 0;
            const int64_t ub = lane < d ? drp[u] : 0;
            const int du = lane < d ? (int)(drp[u + 1] - ub) : 0;
            uint32_t row = 0;
            for (int b = 0; b < d - 1; ++b) {
                const int32_t x = __shfl_sync(kFull, u, b);
                if (lane > b && lane < d && has(dcol + ub, du, x)) row |= 1u << b;
            }
            rows[lane] = row;
            __syncwarp();
            if (lane < d) {
                uint32_t bits = row;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    acc += count_pair<K>(rows, 1, lane, b);
                    if (count4) acc4 += __popc(row & rows[b]);
                }
            }
            __syncwarp();
        }
    }
    unsigned long long s = block_sum(acc, red);
    if (threadIdx.x == 0 && s) atomicAdd(count, s);
    if (count4) {
        __syncthreads();  // red is reused
        s = block_sum(acc4, red);
        if (threadIdx.x == 0 && s) atomicAdd(count4, s);
    }
}

// Builds row(a), a in [1, d), of the root whose out-list O[0, d) is in shared
// memory into rows (stride Ws, zeroed): one warp per a streams the shorter of
// O[0, a) and N'(O[a]) and looks each element up in the other, so a root costs
// about sum_a min(a, |N'(O[a])|) lookups. Lookups in O are binary searches in
// shared memory; lookups in N'(O[a]) are too when stage (per warp, kCliqueMaxOut
// words, or NULL) is given: the warp first copies N'(O[a]) there (coalesced),
// else they are binary searches in global memory.
__device__ __forceinline__ void build_rows(const int64_t* __restrict__ drp,
                                           const int32_t* __restrict__ dcol, const int32_t* O,
                                           int d, uint32_t* rows, int Ws, int lane, int warp,
                                           int nwarps, int32_t* stage) {
    for (int a = warp + 1; a < d; a += nwarps) {
        const int32_t u = O[a];
        const int64_t ub = drp[u];
        const int du = (int)(drp[u + 1] - ub);
        uint32_t* ra = rows + (size_t)a * Ws;
        if (du < a) {
            for (int i = lane; i < du; i += 32) {
                const int b = index_of(O, a, __ldg(dcol + ub + i));
                if (b >= 0) atomicOr(ra + (b >> 5), 1u << (b & 31));
            }
        } else if (stage && du <= kCliqueMaxOut) {
            for (int i = lane; i < du; i += 32) stage[i] = __ldg(dcol + ub + i);
            __syncwarp();
            for (int b0 = 0; b0 < a; b0 += 32) {
                const int b = b0 + lane;
                const bool in = b < a && index_of(stage, du, O[b]) >= 0;
                const uint32_t m = __ballot_sync(kFull, in);
                if (lane == 0) ra[b0 >> 5] = m;
            }
            __syncwarp();
        } else {
            for (int b0 = 0; b0 < a; b0 += 32) {
                const int b = b0 + lane;
                const bool in = b < a && has(dcol + ub, du, O[b]);
                const uint32_t m = __ballot_sync(kFull, in);
                if (lane == 0) ra[b0 >> 5] = m;
            }
        }
    }
}

// Rows of every cached root, built once per out-list view into global memory:
// row a of root hr[i].x goes to grows + hr[i].z + a * row_stride(d), every word
// of it written (padding included), so the buffer needs no clearing. One CTA per
// root at a time, roots handed out by the counter *next. O is indexed by an
// open-addressing hash in shared memory (2 * kCliqueMaxOut slots of
// (vertex id << 32 | position); load <= 1/2). The warps take rows a from a
// shared counter, largest first; a warp assembles row(a) in its own small
// shared buffer, streaming the out-list of O[a] and probing the hash (one probe
// per entry) when that list is not much longer than a, else looking each O[b],
// b < a, up in it by binary search, then writes the row out. Shared memory per
// CTA stays small (hash, O, one row per warp), so many CTAs share an SM.
constexpr int kRowsThreads = 256;
constexpr int kRowBufWords = 36;  // >= row_stride(kCliqueMaxOut)
static_assert(kRowBufWords >= (((kCliqueMaxOut / 32 + 3) / 4) | 1) * 4, "row buffer too small");

__global__ void __launch_bounds__(kRowsThreads) k_clique_rows(const int64_t* __restrict__ drp,
                                                              const int32_t* __restrict__ dcol,
                                                              const int4* __restrict__ hr, int nh,
                                                              unsigned long long* __restrict__ next,
                                                              uint32_t* __restrict__ grows) {
    __shared__ unsigned long long hx[2 * kCliqueMaxOut];
    __shared__ int32_t O[kCliqueMaxOut];
    __shared__ uint32_t rbuf_s[kRowsThreads / 32][kRowBufWords];
    __shared__ int s_h, s_next;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* rbuf = rbuf_s[warp];
    constexpr unsigned kMask = 2 * kCliqueMaxOut - 1;
    for (;;) {
        if (threadIdx.x == 0) {
            s_h = (int)atomicAdd(next, 1ull);
            s_next = 0;
        }
        __syncthreads();
        const int h = s_h;
        if (h >= nh) break;
        const int64_t v = hr[h].x;
        const int64_t ob = drp[v];
        const int d = (int)(drp[v + 1] - ob);
        const int Ws = row_stride(d);
        uint32_t* dst = grows + (uint32_t)hr[h].z;
        for (int i = threadIdx.x; i < 2 * kCliqueMaxOut; i += kRowsThreads) hx[i] = ~0ull;
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += kRowsThreads) {
            const int32_t x = dcol[ob + i];
            O[i] = x;
            const unsigned long long kv = ((unsigned long long)(uint32_t)x << 32) | (uint32_t)i;
            unsigned sl = ((uint32_t)x * 0x9E3779B1u) >> 21;  // 11 bits: 2048 slots
            while (atomicCAS(&hx[sl], ~0ull, kv) != ~0ull) sl = (sl + 1) & kMask;
        }
        __syncthreads();
        // the next row and its out-list bounds are fetched one row ahead, so
        // those loads overlap the current row's work
        int a = -1;
        int64_t ub = 0, ue = 0;
        {
            int m = 0;
            if (lane == 0) m = atomicAdd(&s_next, 1);
            a = d - 1 - __shfl_sync(kFull, m, 0);
            if (a >= 0) {
                ub = drp[O[a]];
                ue = drp[O[a] + 1];
            }
        }
        while (a >= 0) {
            int m = 0;
            if (lane == 0) m = atomicAdd(&s_next, 1);
            const int an = d - 1 - __shfl_sync(kFull, m, 0);
            int64_t ubn = 0, uen = 0;
            if (an >= 0) {
                ubn = drp[O[an]];
                uen = drp[O[an] + 1];
            }
            for (int w = lane; w < Ws; w += 32) rbuf[w] = 0u;
            __syncwarp();
            const int du = (int)(ue - ub);
            if (du <= 4 * a) {
                // stream N'(O[a]) with four loads in flight per lane, probing
                // the hash of O once per entry
                for (int i0 = 0; i0 < du; i0 += 128) {
                    int32_t x[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int i = i0 + 32 * t + lane;
                        x[t] = i < du ? __ldg(dcol + ub + i) : -1;
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (x[t] < 0) continue;
                        unsigned sl = ((uint32_t)x[t] * 0x9E3779B1u) >> 21;
                        int b = -1;
                        for (;;) {
                            const unsigned long long e = hx[sl];
                            if (e == ~0ull) break;
                            if ((int32_t)(e >> 32) == x[t]) { b = (int)(uint32_t)e; break; }
                            sl = (sl + 1) & kMask;
                        }
                        if (b >= 0 && b < a) atomicOr(rbuf + (b >> 5), 1u << (b & 31));
                    }
                }
            } else {
                // N'(O[a]) is long: look each O[b], b < a, up in it. Sample k of
                // the list (lane k, one load) is entry p(k) = min(k gap, du - 1),
                // gap = ceil(du / 32); with k samples <= x, x can only sit in
                // [p(k - 1), p(k - 1) + gap), which a bisection searches.
                const int gap = (du + 31) >> 5;
                const int32_t samp = __ldg(dcol + ub + min(lane * gap, du - 1));
                for (int b0 = 0; b0 < a; b0 += 32) {
                    const int b = b0 + lane;
                    const int32_t x = b < a ? O[b] : INT32_MAX;
                    int k = 0;  // samples <= x (samples are nondecreasing)
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t y = __shfl_sync(kFull, samp, k + step - 1);
                        if (y <= x) k += step;
                    }
                    if (__shfl_sync(kFull, samp, k) <= x) ++k;  // k <= 31 before, may reach 32
                    bool in = false;
                    if (b < a && k > 0) {
                        const int lo = min((k - 1) * gap, du - 1);
                        in = has(dcol + ub + lo, min(gap, du - lo), x);
                    }
                    const uint32_t msk = __ballot_sync(kFull, in);
                    if (lane == 0) rbuf[b0 >> 5] = msk;
                }
            }
            __syncwarp();
            for (int w = lane; w < Ws; w += 32) dst[(size_t)a * Ws + w] = rbuf[w];
            __syncwarp();
            a = an;
            ub = ubn;
            ue = uen;
        }
        __syncthreads();
    }
}

// Roots with 32 < |O| <= max_out: one CTA per root, or per part of a heavy
// root. Shared memory: rows [max_out * Wsmax] words (row stride Ws = W | 1 for
// the current root, odd so that threads reading word w of different rows hit
// different banks; prebuilt rows, stored with row_stride(d), are re-strided on
// the copy), O [max_out], pre [max_out + 1].
//
// Rows come from build_rows or, for a part of a heavy root, are copied from the
// rows k_clique_rows built once for that root. pre[a] counts the local DAG
// edges (a, b), b < a, before row a; edge p is then one work item: a thread
// finds its (a, b) and runs the remaining K - 3 loops over row(a) & row(b).
// Consecutive threads take consecutive edges (same a, neighbouring b), so row(a)
// reads are broadcasts and row(b) reads fall in distinct banks. A heavy root's
// parts take interleaved blocks of kBigThreads edges.
template <int K>
__global__ void __launch_bounds__(kBigThreads) k_clique_big(const int64_t* __restrict__ drp,
                                                         const int32_t* __restrict__ dcol,
                                                         int64_t root_lo, int64_t root_hi,
                                                         int max_out, int heavy_d,
                                                         const int4* __restrict__ heavy,
                                                         int nheavy,
                                                         const uint32_t* __restrict__ grows,
                                                         unsigned long long* __restrict__ work,
                                                         unsigned long long* __restrict__ count) {
    extern __shared__ uint32_t sm[];
    __shared__ unsigned long long red[kBigThreads / 32];
    __shared__ int64_t s_root;
    const int Wsmax = ((max_out + 31) >> 5) | 1;
    uint32_t* rows = sm;
    int32_t* O = reinterpret_cast<int32_t*>(sm + (size_t)max_out * Wsmax);
    int32_t* pre = O + max_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = kBigThreads / 32;
    unsigned long long acc = 0;
    const int64_t nchunks = (root_hi - root_lo + kBigPop - 1) / kBigPop;
    for (;;) {
        // queue slots: [0, nheavy) one part of a heavy root each (heaviest first),
        // then chunks of kBigPop consecutive roots (heavy ones skipped there)
        if (threadIdx.x == 0) s_root = (int64_t)atomicAdd(work, 1ull);
        __syncthreads();
        const int64_t slot = s_root;
        __syncthreads();
        if (slot >= nheavy + nchunks) break;
        int64_t v0, nr;
        int part = 0, parts = 1;
        const uint32_t* src = nullptr;  // prebuilt rows of a heavy root
        if (slot < nheavy) {
            const int4 h = heavy[slot];
            v0 = h.x;
            nr = 1;
            part = h.y & 0xffff;
            parts = h.y >> 16;
            src = grows + (uint32_t)h.z;
        } else {
            v0 = root_lo + (slot - nheavy) * kBigPop;
            nr = kBigPop;
        }
      for (int r = 0; r < nr; ++r) {
        const int64_t v = v0 + r;
        if (v >= root_hi) break;
        const int64_t ob = drp[v];
        const int d = (int)(drp[v + 1] - ob);
        if (d <= 32 || d > max_out || (slot >= nheavy && d >= heavy_d)) continue;
        const int Ws = ((d + 31) >> 5) | 1;
        for (int i = threadIdx.x; i < d; i += kBigThreads) O[i] = dcol[ob + i];
        if (src) {
            const int Wg = row_stride(d);
            for (int i = threadIdx.x; i < d * Ws; i += kBigThreads) {
                const int a = i / Ws, w = i - a * Ws;
                rows[i] = w < Wg ? __ldg(src + (size_t)a * Wg + w) : 0u;
            }
            __syncthreads();
        } else {
            for (int i = threadIdx.x; i < d * Ws; i += kBigThreads) rows[i] = 0;
            __syncthreads();
            build_rows(drp, dcol, O, d, rows, Ws, lane, warp, nwarps, nullptr);
            __syncthreads();
        }
        // pre[a] = number of local edges (a, b), b < a, before row a
        if (warp == 0) {
            int run = 0;
            for (int a0 = 0; a0 < d; a0 += 32) {
                const int a = a0 + lane;
                int c = 0;
                if (a < d)
                    for (int w = 0, wa = (a + 31) >> 5; w < wa; ++w) c += __popc(rows[(size_t)a * Ws + w]);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                if (a < d) pre[a] = run + incl - c;
                run += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) pre[d] = run;
        }
        __syncthreads();
        const int pairs = pre[d];
        for (int blk = part; blk * kBigThreads < pairs; blk += parts) {
            const int p = blk * kBigThreads + threadIdx.x;
            if (p >= pairs) continue;
            int lo = 0, hi = d - 1;  // last a with pre[a] <= p
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= p) lo = mid; else hi = mid - 1;
            }
            const int a = lo;
            int j = p - pre[a];
            const uint32_t* ra = rows + (size_t)a * Ws;
            int b = -1;
            for (int w = 0; w < Ws; ++w) {
                uint32_t m = ra[w];
                const int c = __popc(m);
                if (j < c) {
                    for (int i = 0; i < j; ++i) m &= m - 1;
                    b = (w << 5) + __ffs(m) - 1;
                    break;
                }
                j -= c;
            }
            acc += count_pair<K>(rows, Ws, a, b);
        }
        __syncthreads();
      }
    }
    unsigned long long s = block_sum(acc, red);
    if (threadIdx.x == 0 && s) atomicAdd(count, s);
}

// K = 4 and K = 5 on roots with 32 < |O| <= max_out: k_clique_warp. The rows
// sit in shared memory as in k_clique_big, but the work is spread by warps, not
// by CTA-wide pair indices. One CTA takes one root at a time (heavy roots
// first, heaviest first, with their prebuilt rows; no root is split over CTAs:
// on the skewed graphs measured the largest root holds a fifth of one SM's
// share of the work). The CTA's warps pop the root's rows a from a counter in
// shared memory, largest a first, and walk the pairs (a, b in row(a)) one pair
// per lane: for K = 5, 32 consecutive pairs at a time, a group running on into
// the next row the warp pops (k5_rows_packed); for K = 4, whose pairs are cheap,
// lane l simply takes bit l of each word of row(a). Then the lane counts its
// pair:
//  - K = 4: |row(a) & row(b)| below b;
//  - K = 5: with S = row(a) & row(b) (bits below b) held in registers, the sum
//    over c in S of |S & row(c)|, row(c) holding bits below c only.
// Rows are read as 16-byte chunks (row_stride keeps them aligned). Warps never
// wait for each other inside a root.
constexpr int kWarpCta = 512;
constexpr int kWarpCtaWarps = kWarpCta / 32;

// Position of the k-th set bit (0-based) of m; requires k < popc(m).
__device__ __forceinline__ int select_bit(uint32_t m, int k) {
    int pos = 0;
    int c = __popc(m & 0xffffu);
    if (k >= c) { k -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xffu);
    if (k >= c) { k -= c; m >>= 8; pos += 8; }
    c = __popc(m & 0xfu);
    if (k >= c) { k -= c; m >>= 4; pos += 4; }
    c = __popc(m & 0x3u);
    if (k >= c) { k -= c; m >>= 2; pos += 2; }
    if (k >= (int)(m & 1u)) pos += 1;
    return pos;
}

// The popcounts run on the SM's quarter-rate XU pipe, so only words below b
// (row(b) is zero above them) are counted.
__device__ __forceinline__ uint32_t k4_pair(const uint4* __restrict__ rows4, int Ws4, int a, int b) {
    const uint4* ra = rows4 + (size_t)a * Ws4;
    const uint4* rb = rows4 + (size_t)b * Ws4;
    const int nw = (b + 31) >> 5;
    uint32_t cnt = 0;
    int q = 0;
    for (; 4 * q + 4 <= nw; ++q) {
        const uint4 A = ra[q], B = rb[q];
        cnt += __popc(A.x & B.x) + __popc(A.y & B.y) + __popc(A.z & B.z) + __popc(A.w & B.w);
    }
    const int rest = nw - 4 * q;
    if (rest > 0) {
        const uint4 A = ra[q], B = rb[q];
        cnt += __popc(A.x & B.x);
        if (rest > 1) cnt += __popc(A.y & B.y);
        if (rest > 2) cnt += __popc(A.z & B.z);
    }
    return cnt;
}

// Words of S (from word 0) that take the dense walk when they are dense, and
// the bit count above which a warp counts a word as dense.
constexpr int kDenseWords = 2;
constexpr int kDenseMin = 15;

// WM: a multiple of 4 with WM >= ceil(b / 32); S is unrolled into WM registers.
// Every lane of the warp calls it (b = 0 gives an empty S and no loads).
// F4: also add |S| to k4 (the pair's K4 count: S holds the vertices that close
// a 4-clique with (root, a, b)), for the fused K4 + K5 pass.
template <int WM, bool F4>
__device__ __forceinline__ uint32_t k5_pair(const uint4* __restrict__ rows4, int Ws4, int a, int b,
                                            uint32_t& k4) {
    const uint4* ra = rows4 + (size_t)a * Ws4;
    const uint4* rb = rows4 + (size_t)b * Ws4;
    const int nq = (b + 127) >> 7;
    uint32_t S[WM];
#pragma unroll
    for (int q = 0; q < WM / 4; ++q) {
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        if (q < nq) {
            const uint4 A = ra[q], B = rb[q];
            x = make_uint4(A.x & B.x, A.y & B.y, A.z & B.z, A.w & B.w);
            if constexpr (F4) k4 += __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w);
        }
        S[4 * q] = x.x;
        S[4 * q + 1] = x.y;
        S[4 * q + 2] = x.z;
        S[4 * q + 3] = x.w;
    }
    // c runs over the bits of S word w (highest first, one count-leading-zeros
    // each); row(c) is zero above word w, so exactly w + 1 words are counted
    // (the guards are compile-time constants of the unrolled loops). Words 0..3
    // hold most candidates on skewed graphs (low local index = high degree);
    // there row(c) is one 16-byte chunk, loaded one candidate ahead so that the
    // load of the next row overlaps the popcounts of this one.
    uint32_t cnt = 0;
    const uint32_t* rows32 = reinterpret_cast<const uint32_t*>(rows4);
    const int Ws = Ws4 * 4;
#pragma unroll
    for (int w = 0; w < 4 && w < WM; ++w) {
        if (w < kDenseWords) {
            // Dense word (some lane's S word holds more than kDenseMin bits):
            // the lanes walk all 32 candidates c = 32 w + j in lockstep, with no
            // bit search; row(c) is at one address for every lane (a broadcast
            // load), read only by lanes whose S has bit c (so c < b < d).
            const unsigned mx = __reduce_max_sync(kFull, (unsigned)__popc(S[w]));
            if (mx > (unsigned)kDenseMin) {
#pragma unroll
                for (int j = (w == 0 ? 1 : 0); j < 32; ++j) {
                    if ((S[w] >> j) & 1u) {
                        const uint32_t* rc = rows32 + (size_t)(32 * w + j) * Ws;
                        if (w == 0) {
                            cnt += __popc(S[0] & rc[0]);
                        } else if (w == 1) {
                            const uint2 r = *reinterpret_cast<const uint2*>(rc);
                            cnt += __popc(S[0] & r.x) + __popc(S[1] & r.y);
                        } else {
                            const uint4 r = *reinterpret_cast<const uint4*>(rc);
                            cnt += __popc(S[0] & r.x) + __popc(S[1] & r.y) + __popc(S[2] & r.z);
                            if (w == 3) cnt += __popc(S[3] & r.w);
                        }
                    }
                }
                continue;
            }
        }
        uint32_t bits = S[w];
        if (!bits) continue;
        int hb = 31 - __clz(bits);
        bits ^= 1u << hb;
        uint4 r = rows4[(size_t)((w << 5) + hb) * Ws4];
        while (bits) {
            hb = 31 - __clz(bits);
            bits ^= 1u << hb;
            const uint4 nx = rows4[(size_t)((w << 5) + hb) * Ws4];
            cnt += __popc(S[0] & r.x);
            if (w >= 1) cnt += __popc(S[1] & r.y);
            if (w >= 2) cnt += __popc(S[2] & r.z);
            if (w >= 3) cnt += __popc(S[3] & r.w);
            r = nx;
        }
        cnt += __popc(S[0] & r.x);
        if (w >= 1) cnt += __popc(S[1] & r.y);
        if (w >= 2) cnt += __popc(S[2] & r.z);
        if (w >= 3) cnt += __popc(S[3] & r.w);
    }
#pragma unroll
    for (int w = 4; w < WM; ++w) {
        uint32_t bits = S[w];
        while (bits) {
            const int hb = 31 - __clz(bits);
            bits ^= 1u << hb;
            const uint4* rc = rows4 + (size_t)((w << 5) + hb) * Ws4;
#pragma unroll
            for (int q = 0; q <= w / 4; ++q) {
                const uint4 r = rc[q];
                cnt += __popc(S[4 * q] & r.x);
                if (4 * q + 1 <= w) cnt += __popc(S[4 * q + 1] & r.y);
                if (4 * q + 2 <= w) cnt += __popc(S[4 * q + 2] & r.z);
                if (4 * q + 3 <= w) cnt += __popc(S[4 * q + 3] & r.w);
            }
        }
    }
    return cnt;
}

// nw: words of the widest pair among the warp's active lanes (the same for all
// lanes, so the warp runs one instantiation of k5_pair).
template <bool F4>
__device__ __forceinline__ uint32_t k5_pair_any(const uint4* rows4, int Ws4, int a, int b, int nw, uint32_t& k4) {
    if (nw <= 8) return k5_pair<8, F4>(rows4, Ws4, a, b, k4);
    if (nw <= 16) return k5_pair<16, F4>(rows4, Ws4, a, b, k4);
    if (nw <= 24) return k5_pair<24, F4>(rows4, Ws4, a, b, k4);
    return k5_pair<32, F4>(rows4, Ws4, a, b, k4);
}

// K = 5 walk of one root's rows by one warp. The 32 lanes take 32 consecutive
// pairs (a, b) in the order: rows a popped from *next (largest a first), bits b
// of row(a) ascending. A group that exhausts its row continues with the next
// row the warp pops, so lanes idle only at the end of the root's rows (rows
// with fewer than 32 bits are the common case on skewed graphs). A lane finds
// its b from the popcount prefix of row(a)'s words (one word per lane) by a
// shuffle search. All loop control is warp-uniform. F4: K4 counts too (acc4).
template <bool F4>
__device__ __forceinline__ void k5_rows_packed(const uint32_t* rows, const uint4* rows4, int Ws, int Ws4,
                                               int d, int lane, int* next, unsigned long long& acc,
                                               unsigned long long& acc4) {
    int cur_a = 0, cur_j = 0, cur_total = 0;  // row being drawn, pairs taken, its pairs
    uint32_t word = 0;                        // this lane's word of row(cur_a)
    int incl = 0;                             // popcount of row(cur_a)'s words 0..lane
    bool drained = false;
    for (;;) {
        int my_a = -1, my_b = 0, filled = 0;
        while (filled < 32) {
            if (cur_j == cur_total) {
                if (drained) break;
                int m = 0;
                if (lane == 0) m = atomicAdd(next, 1);
                m = __shfl_sync(kFull, m, 0);
                const int a = d - 1 - m;
                if (a < 1) {
                    drained = true;
                    break;
                }
                cur_a = a;
                cur_j = 0;
                word = lane < ((a + 31) >> 5) ? rows[(size_t)a * Ws + lane] : 0u;
                incl = __popc(word);
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                cur_total = __shfl_sync(kFull, incl, 31);
                continue;
            }
            const int take = min(32 - filled, cur_total - cur_j);
            const bool mine = lane >= filled && lane < filled + take;
            const int j = mine ? cur_j + lane - filled : 0;  // this lane's bit of row(cur_a), in order
            int wlo = 0, whi = 31;                           // first word whose inclusive count exceeds j
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int mid = (wlo + whi) >> 1;
                const int x = __shfl_sync(kFull, incl, mid);
                if (x > j) whi = mid; else wlo = mid + 1;
            }
            const uint32_t ww = __shfl_sync(kFull, word, wlo);
            const int before = __shfl_sync(kFull, incl, wlo) - __popc(ww);
            if (mine) {
                my_a = cur_a;
                my_b = (wlo << 5) + select_bit(ww, j - before);
            }
            filled += take;
            cur_j += take;
        }
        if (filled == 0) break;
        // idle lanes (the root's last group) count the empty pair (a, 0)
        if (my_a < 0) my_a = my_b = 0;
        const int nw = __reduce_max_sync(kFull, (unsigned)((my_b + 31) >> 5));
        uint32_t k4 = 0;
        acc += k5_pair_any<F4>(rows4, Ws4, my_a, my_b, nw, k4);
        if constexpr (F4) acc4 += k4;
    }
}

// F4 (K = 5 only): the fused K4 + K5 pass; the K4 count goes to *count4.
template <int K, bool F4 = false>
__global__ void __launch_bounds__(kWarpCta, 2) k_clique_warp(const int64_t* __restrict__ drp,
                                                          const int32_t* __restrict__ dcol,
                                                          int64_t root_lo, int64_t root_hi,
                                                          int max_out, int heavy_d,
                                                          const int4* __restrict__ heavy,
                                                          int nheavy,
                                                          const uint32_t* __restrict__ grows,
                                                          unsigned long long* __restrict__ work,
                                                          unsigned long long* __restrict__ count,
                                                          unsigned long long* __restrict__ count4) {
    static_assert(K == 4 || K == 5, "k_clique_warp counts K4 and K5");
    static_assert(!F4 || K == 5, "the fused pass is the K5 walk");
    extern __shared__ __align__(16) uint32_t smw[];
    __shared__ unsigned long long red[kWarpCtaWarps];
    __shared__ int64_t s_slot;
    __shared__ int s_next;
    const int Wsmax = row_stride(max_out);
    uint32_t* rows = smw;
    int32_t* O = reinterpret_cast<int32_t*>(smw + (size_t)max_out * Wsmax);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long acc = 0, acc4 = 0;
    const int64_t nchunks = (root_hi - root_lo + kBigPop - 1) / kBigPop;
    for (;;) {
        // queue slots: [0, nheavy) one heavy root each (heaviest first), then
        // chunks of kBigPop consecutive roots (heavy ones skipped there)
        if (threadIdx.x == 0) s_slot = (int64_t)atomicAdd(work, 1ull);
        __syncthreads();
        const int64_t slot = s_slot;
        __syncthreads();
        if (slot >= nheavy + nchunks) break;
        int64_t v0, nr;
        const uint32_t* src = nullptr;  // prebuilt rows of a heavy root
        if (slot < nheavy) {
            const int4 h = heavy[slot];
            v0 = h.x;
            nr = 1;
            src = grows + (uint32_t)h.z;
        } else {
            v0 = root_lo + (slot - nheavy) * kBigPop;
            nr = kBigPop;
        }
        for (int r = 0; r < nr; ++r) {
            const int64_t v = v0 + r;
            if (v >= root_hi) break;
            const int64_t ob = drp[v];
            const int d = (int)(drp[v + 1] - ob);
            if (d <= 32 || d > max_out || (slot >= nheavy && d >= heavy_d)) continue;
            const int Ws = row_stride(d);
            if (src) {
                const uint4* s4 = reinterpret_cast<const uint4*>(src);
                uint4* r4 = reinterpret_cast<uint4*>(rows);
                for (int i = threadIdx.x; i < d * (Ws >> 2); i += kWarpCta) r4[i] = __ldg(s4 + i);
            } else {
                for (int i = threadIdx.x; i < d; i += kWarpCta) O[i] = dcol[ob + i];
                for (int i = threadIdx.x; i < d * Ws; i += kWarpCta) rows[i] = 0;
                __syncthreads();
                build_rows(drp, dcol, O, d, rows, Ws, lane, warp, kWarpCtaWarps, nullptr);
            }
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
            const uint4* rows4 = reinterpret_cast<const uint4*>(rows);
            const int Ws4 = Ws >> 2;
            if constexpr (K == 5) {
                k5_rows_packed<F4>(rows, rows4, Ws, Ws4, d, lane, &s_next, acc, acc4);
            } else {
                for (;;) {
                    int m = 0;
                    if (lane == 0) m = atomicAdd(&s_next, 1);
                    m = __shfl_sync(kFull, m, 0);
                    const int a = d - 1 - m;  // largest rows first
                    if (a < 1) break;
                    // rows are dense on the heavy roots, so lane l takes bit l of
                    // each word w of row(a) (b = 32 w + l): b needs no search and
                    // all active lanes count the same w + 1 words
                    for (int w = 0, nwa = (a + 31) >> 5; w < nwa; ++w) {
                        const uint32_t bits = rows[(size_t)a * Ws + w];
                        if ((bits >> lane) & 1u) acc += k4_pair(rows4, Ws4, a, (w << 5) + lane);
                    }
                }
            }
            __syncthreads();
        }
    }
    unsigned long long s = block_sum(acc, red);
    if (threadIdx.x == 0 && s) atomicAdd(count, s);
    if constexpr (F4) {
        __syncthreads();  // red is reused
        s = block_sum(acc4, red);
        if (threadIdx.x == 0 && s) atomicAdd(count4, s);
    }
}

// Roots whose out-list is too long for shared-memory rows (kCliqueMaxOut <
// |O| <= kCliqueLongOut): rows live in global memory, where k_clique_long_rows
// builds them (one CTA per root, O in shared memory, rows zeroed by the host),
// and k_clique_long walks their local DAG edges as k_clique_big does, reading
// the rows through the L1/L2 caches. lr[i] = (root, part | parts << 16, word
// offset of the root's rows); the offsets of the build list have parts = 1.
__global__ void __launch_bounds__(kThreads) k_clique_long_rows(const int64_t* __restrict__ drp,
                                                               const int32_t* __restrict__ dcol,
                                                               const int4* __restrict__ lr, int nl,
                                                               uint32_t* __restrict__ grows) {
    extern __shared__ uint32_t sm[];
    int32_t* O = reinterpret_cast<int32_t*>(sm);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int h = blockIdx.x; h < nl; h += gridDim.x) {
        const int64_t v = lr[h].x;
        const int64_t ob = drp[v];
        const int d = (int)(drp[v + 1] - ob);
        const int Ws = ((d + 31) >> 5) | 1;
        for (int i = threadIdx.x; i < d; i += kThreads) O[i] = dcol[ob + i];
        __syncthreads();
        build_rows(drp, dcol, O, d, grows + (uint32_t)lr[h].z, Ws, lane, warp, kThreads / 32, nullptr);
        __syncthreads();
    }
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_clique_long(const int64_t* __restrict__ drp,
                                                          const int4* __restrict__ lr, int nl,
                                                          const uint32_t* __restrict__ grows,
                                                          unsigned long long* __restrict__ work,
                                                          unsigned long long* __restrict__ count) {
    extern __shared__ uint32_t sm[];
    int32_t* pre = reinterpret_cast<int32_t*>(sm);  // [kCliqueLongOut + 1]
    __shared__ unsigned long long red[kThreads / 32];
    __shared__ int64_t s_slot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = kThreads / 32;
    unsigned long long acc = 0;
    for (;;) {
        if (threadIdx.x == 0) s_slot = (int64_t)atomicAdd(work, 1ull);
        __syncthreads();
        const int64_t slot = s_slot;
        __syncthreads();
        if (slot >= nl) break;
        const int4 h = lr[slot];
        const int part = h.y & 0xffff, parts = h.y >> 16;
        const int d = (int)(drp[h.x + 1] - drp[h.x]);
        const int Ws = ((d + 31) >> 5) | 1;
        const uint32_t* rows = grows + (uint32_t)h.z;
        // pre[a + 1] = popcount of row a (warp per row), then an inclusive scan
        for (int a = warp; a < d; a += nwarps) {
            int c = 0;
            for (int w = lane, wa = (a + 31) >> 5; w < wa; w += 32) c += __popc(rows[(size_t)a * Ws + w]);
            for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
            if (lane == 0) pre[a + 1] = c;
        }
        __syncthreads();
        if (warp == 0) {
            int run = 0;
            if (lane == 0) pre[0] = 0;
            for (int a0 = 1; a0 <= d; a0 += 32) {
                const int a = a0 + lane;
                const int c = a <= d ? pre[a] : 0;
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                if (a <= d) pre[a] = run + incl;
                run += __shfl_sync(kFull, incl, 31);
            }
        }
        __syncthreads();
        const int pairs = pre[d];
        for (int blk = part; (int64_t)blk * kThreads < pairs; blk += parts) {
            const int p = blk * kThreads + threadIdx.x;
            if (p >= pairs) continue;
            int lo = 0, hi = d - 1;  // last a with pre[a] <= p
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= p) lo = mid; else hi = mid - 1;
            }
            const int a = lo;
            int j = p - pre[a];
            const uint32_t* ra = rows + (size_t)a * Ws;
            int b = -1;
            for (int w = 0; w < Ws; ++w) {
                uint32_t m = ra[w];
                const int c = __popc(m);
                if (j < c) {
                    for (int i = 0; i < j; ++i) m &= m - 1;
                    b = (w << 5) + __ffs(m) - 1;
                    break;
                }
                j -= c;
            }
            acc += count_pair<K>(rows, Ws, a, b);
        }
        __syncthreads();
    }
    unsigned long long s = block_sum(acc, red);
    if (threadIdx.x == 0 && s) atomicAdd(count, s);
}

// Roots with out-degree >= kHeavyD (one pass to count, one to fill).
// Ordered collection of the roots with out-degree >= heavy_d: per-tile counts,
// a one-CTA scan of the tile counts, then each tile writes its roots in id
// order at its offset, so the list comes out sorted by root with no host sort.
constexpr int kCollectThreads = 256;
constexpr int kCollectPer = 16;  // consecutive vertices per thread
constexpr int kCollectTile = kCollectThreads * kCollectPer;

__device__ __forceinline__ int block_excl_scan(int c, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int x = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        int wi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - x;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    return warp_tot[warp] + incl - c;
}

__global__ void __launch_bounds__(kCollectThreads) k_heavy_counts(const int64_t* __restrict__ drp, int64_t n,
                                                                  int heavy_d, int* __restrict__ tile_cnt) {
    __shared__ int warp_tot[kCollectThreads / 32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kCollectTile + (int64_t)threadIdx.x * kCollectPer;
    int c = 0;
    for (int i = 0; i < kCollectPer; ++i) {
        const int64_t v = base + i;
        if (v < n && drp[v + 1] - drp[v] >= heavy_d) ++c;
    }
    block_excl_scan(c, warp_tot, &total);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = total;
}

// off[i] = tiles' counts before tile i, off[ntiles] = all (one CTA).
__global__ void __launch_bounds__(1024) k_heavy_scan(const int* __restrict__ cnt, int64_t ntiles,
                                                     int64_t* __restrict__ off) {
    __shared__ int64_t part[1024];
    const int64_t per = (ntiles + 1023) / 1024;
    const int64_t b = threadIdx.x * per, e = b + per < ntiles ? b + per : ntiles;
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const int64_t x = part[i];
            part[i] = run;
            run += x;
        }
        off[ntiles] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        off[i] = run;
        run += cnt[i];
    }
}

__global__ void __launch_bounds__(kCollectThreads) k_heavy_fill(const int64_t* __restrict__ drp, int64_t n,
                                                                int heavy_d, const int64_t* __restrict__ off,
                                                                int2* __restrict__ out) {
    __shared__ int warp_tot[kCollectThreads / 32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kCollectTile + (int64_t)threadIdx.x * kCollectPer;
    int c = 0;
    for (int i = 0; i < kCollectPer; ++i) {
        const int64_t v = base + i;
        if (v < n && drp[v + 1] - drp[v] >= heavy_d) ++c;
    }
    int64_t pos = off[blockIdx.x] + block_excl_scan(c, warp_tot, &total);
    for (int i = 0; i < kCollectPer; ++i) {
        const int64_t v = base + i;
        if (v < n) {
            const int64_t d = drp[v + 1] - drp[v];
            if (d >= heavy_d) out[pos++] = make_int2((int)v, (int)d);
        }
    }
}

// Fills v.heavy (sorted by root id) once per out-list build.
gz_status gather_heavy(GzView& v, int64_t n, cudaStream_t s) {
    if (v.heavy_built) return GZ_OK;
    v.heavy.clear();
    if (n <= 0 || v.max_out < kHeavyD) {
        v.heavy_built = true;
        return GZ_OK;
    }
    const int64_t ntiles = (n + kCollectTile - 1) / kCollectTile;
    // tile counts | offsets [ntiles + 1]
    const size_t cbytes = (sizeof(int) * ntiles + 15) & ~(size_t)15;
    char* buf = nullptr;
    cudaError_t e = gz_malloc_async(&buf, cbytes + sizeof(int64_t) * (ntiles + 1), s);
    if (e != cudaSuccess) return cuda_fail(e, "clique: heavy roots");
    int* cnt = reinterpret_cast<int*>(buf);
    int64_t* off = reinterpret_cast<int64_t*>(buf + cbytes);
    int64_t h = 0;
    k_heavy_counts<<<(unsigned)ntiles, kCollectThreads, 0, s>>>(v.dag_rp, n, kHeavyD, cnt);
    GZ_COUNT_LAUNCH();
    k_heavy_scan<<<1, 1024, 0, s>>>(cnt, ntiles, off);
    GZ_COUNT_LAUNCH();
    e = cudaMemcpyAsync(&h, off + ntiles, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int2* d_out = nullptr;
    std::vector<int2> tmp(h);
    if (e == cudaSuccess && h > 0) {
        e = gz_malloc_async(&d_out, sizeof(int2) * h, s);
        if (e == cudaSuccess) {
            k_heavy_fill<<<(unsigned)ntiles, kCollectThreads, 0, s>>>(v.dag_rp, n, kHeavyD, off, d_out);
            GZ_COUNT_LAUNCH();
            e = cudaMemcpyAsync(tmp.data(), d_out, sizeof(int2) * h, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(d_out, s);
    }
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_fail(e, "clique: heavy roots");
    v.heavy.reserve(h);
    for (const int2& x : tmp) v.heavy.emplace_back(x.x, x.y);
    v.heavy_built = true;
    return GZ_OK;
}

// Parts a heavy root is split into by k_clique_big: about its work (d^2 for
// K = 4, d^3 beyond) over that of a root of out-degree kSplitD, at most 64 and
// at most d. Parts
// copy the root's prebuilt rows, so a part costs little beyond its share.
int parts_for(int K, int d) {
    const double r = (double)d / kSplitD;
    const double w = K == 4 ? r * r : r * r * r;
    const int p = (int)std::ceil(w);
    return std::max(1, std::min(std::min(p, 64), d));
}

// Builds, once per out-list view, the bitset rows of every heavy root with at
// most mo out-neighbours into v.heavy_rows (kept until the view is rebuilt or
// the graph destroyed). Over kHeavyRowWords words in all, nothing is cached and
// heavy roots are not split.
gz_status build_heavy_rows(GzView& v, int mo, int sms, cudaStream_t s) {
    if (v.heavy_rows_built) return GZ_OK;
    v.heavy_rows_ok = false;
    v.slot_host.clear();
    v.heavy_off.assign(v.heavy.size(), UINT32_MAX);
    std::vector<int4> list;
    uint64_t words = 0;
    for (size_t i = 0; i < v.heavy.size(); ++i) {
        const int d = v.heavy[i].second;
        if (d > mo) continue;
        v.heavy_off[i] = (uint32_t)words;
        list.push_back(make_int4(v.heavy[i].first, 0, (int)words, 0));
        words += ((uint64_t)d * row_stride(d) + 3) & ~3ull;
    }
    v.heavy_rows_built = true;
    if (list.empty() || words > kHeavyRowWords) {
        v.heavy_off.assign(v.heavy.size(), UINT32_MAX);
        return GZ_OK;
    }
    int4* d_list = nullptr;
    cudaError_t e = cudaSuccess;
    if (words > v.heavy_rows_cap) {  // grow; rebuilds of the same view reuse the buffer
        cudaFree(v.heavy_rows);
        v.heavy_rows = nullptr;
        v.heavy_rows_cap = 0;
        e = gz_malloc(&v.heavy_rows, sizeof(uint32_t) * words);
        if (e == cudaSuccess) v.heavy_rows_cap = words;
    }
    // list | work counter
    const size_t lbytes = (sizeof(int4) * list.size() + 15) & ~(size_t)15;
    if (e == cudaSuccess) e = gz_malloc_async(&d_list, lbytes + 16, s);
    unsigned long long* d_next = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(d_list) + lbytes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_list, list.data(), sizeof(int4) * list.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, 16, s);
    if (e == cudaSuccess) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_rows, kRowsThreads, 0);
        const int rb = (int)std::min<size_t>(list.size(), (size_t)sms * std::max(1, per_sm));
        if (e == cudaSuccess) {
            k_clique_rows<<<rb, kRowsThreads, 0, s>>>(v.dag_rp, v.dag_col, d_list, (int)list.size(), d_next,
                                                      v.heavy_rows);
            GZ_COUNT_LAUNCH();
            e = cudaGetLastError();
        }
    }
    if (d_list) cudaFreeAsync(d_list, s);
    // the rows are complete before any stream (other batch slots included) uses them
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(v.heavy_rows);
        v.heavy_rows = nullptr;
        v.heavy_rows_cap = 0;
        v.heavy_off.assign(v.heavy.size(), UINT32_MAX);
        return cuda_fail(e, "clique: heavy rows");
    }
    v.heavy_rows_ok = true;
    // the heavy-root slots of k_clique_warp (one per cached root, heaviest
    // first: a counting sort by out-degree), kept on the device for counts over
    // all roots and on the host for root ranges
    std::vector<int> start(mo + 2, 0);
    for (size_t i = 0; i < v.heavy.size(); ++i)
        if (v.heavy_off[i] != UINT32_MAX) ++start[mo - v.heavy[i].second];
    for (int x = 0, run = 0; x <= mo + 1; ++x) {
        const int c = start[x];
        start[x] = run;
        run += c;
    }
    v.slot_host.assign(list.size(), make_int4(0, 0, 0, 0));
    for (size_t i = 0; i < v.heavy.size(); ++i)
        if (v.heavy_off[i] != UINT32_MAX)
            v.slot_host[start[mo - v.heavy[i].second]++] =
                make_int4(v.heavy[i].first, 1 << 16, (int)v.heavy_off[i], v.heavy[i].second);
    if ((int64_t)v.slot_host.size() > v.slot_cap) {
        cudaFree(v.slot_dev);
        v.slot_dev = nullptr;
        v.slot_cap = 0;
        e = gz_malloc(&v.slot_dev, sizeof(int4) * v.slot_host.size());
        if (e != cudaSuccess) return cuda_fail(e, "clique: heavy slots");
        v.slot_cap = (int64_t)v.slot_host.size();
    }
    e = cudaMemcpyAsync(v.slot_dev, v.slot_host.data(), sizeof(int4) * v.slot_host.size(),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "clique: heavy slots");
    return GZ_OK;
}

// Roots of [lo, hi) with kCliqueMaxOut < |O| <= kCliqueLongOut: rows built in
// global memory (at most kLongRowWords words; roots beyond that budget, and
// roots longer than kCliqueLongOut, are left to the caller's general kernel,
// see clique_long_cutoff), then their edges walked by k_clique_long.
template <int K>
gz_status launch_long(GzView& v, int64_t lo, int64_t hi, double frac, cudaStream_t s,
                      unsigned long long* d_count, unsigned long long* d_work) {
    std::vector<std::pair<int32_t, int32_t>> hr;
    auto it = std::lower_bound(v.heavy.begin(), v.heavy.end(), std::make_pair((int32_t)lo, INT32_MIN));
    for (; it != v.heavy.end() && it->first < hi; ++it)
        if (it->second > kCliqueMaxOut && it->second <= kCliqueLongOut) hr.push_back(*it);
    if (hr.empty()) return GZ_OK;
    std::stable_sort(hr.begin(), hr.end(), [](const std::pair<int32_t, int32_t>& a,
                                              const std::pair<int32_t, int32_t>& b) {
        return a.second > b.second;
    });
    std::vector<int4> build, ent;
    uint64_t words = 0;
    for (const auto& x : hr) {
        const uint64_t sz = (uint64_t)x.second * (((x.second + 31) / 32) | 1);
        if (words + sz > kLongRowWords) break;
        build.push_back(make_int4(x.first, 1 << 16, (int)words, 0));
        const int parts = std::min(64, std::max(1, (int)((uint64_t)x.second * x.second / (256 * 256))));
        for (int p = 0; p < parts; ++p) ent.push_back(make_int4(x.first, p | (parts << 16), (int)words, 0));
        words += (sz + 3) & ~3ull;
    }
    if (build.size() < hr.size()) {
        set_error("clique: long out-lists exceed the row budget");
        return GZ_ENOMEM;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int4* d_l = nullptr;
    uint32_t* grows = nullptr;
    cudaError_t e = gz_malloc_async(&d_l, sizeof(int4) * (build.size() + ent.size()), s);
    if (e == cudaSuccess) e = gz_malloc_async(&grows, sizeof(uint32_t) * words, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(grows, 0, sizeof(uint32_t) * words, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_l, build.data(), sizeof(int4) * build.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_l + build.size(), ent.data(), sizeof(int4) * ent.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const size_t smem = sizeof(int32_t) * (kCliqueLongOut + 1);
        cudaFuncSetAttribute(k_clique_long_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_clique_long<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int rb = (int)std::min<size_t>(build.size(), std::max<size_t>(1, (size_t)(sms * 4 * frac)));
        k_clique_long_rows<<<rb, kThreads, smem, s>>>(v.dag_rp, v.dag_col, d_l, (int)build.size(), grows);
        GZ_COUNT_LAUNCH();
        const int lb = (int)std::min<size_t>(ent.size(), std::max<size_t>(1, (size_t)(sms * 4 * frac)));
        k_clique_long<K><<<lb, kThreads, smem, s>>>(v.dag_rp, d_l + build.size(), (int)ent.size(), grows,
                                                     d_work, d_count);
        GZ_COUNT_LAUNCH();
        e = cudaGetLastError();
    }
    if (d_l) cudaFreeAsync(d_l, s);
    if (grows) cudaFreeAsync(grows, s);
    if (e != cudaSuccess) return cuda_fail(e, "clique: long roots");
    return GZ_OK;
}

// Grids are the resident CTAs on every SM, or the fraction frac of them (the
// request loop runs slow requests on part of the device).
inline int grid_part(int full, double frac) { return frac < 1.0 ? std::max(1, (int)(full * frac)) : full; }

// d_count4 (K = 5 only, else NULL): the fused K4 + K5 pass, which also adds the
// K4 count of the roots to *d_count4; the view must have no root longer than
// kCliqueMaxOut (those take the long-root kernels, which count one K).
template <int K>
gz_status launch_k(const GzView& v, int64_t n, int64_t lo, int64_t hi, double frac, cudaStream_t s,
                   unsigned long long* d_count, unsigned long long* d_work,
                   unsigned long long* d_count4 = nullptr) {
    if (d_count4 && (K != 5 || v.max_out > kCliqueMaxOut)) {
        set_error("fused K4 + K5 pass: needs K = 5 and out-lists of at most %d", kCliqueMaxOut);
        return GZ_EINVAL;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_small<K>, kThreads, 0);
    const int64_t nroots = hi - lo;
    int blocks = grid_part(sms * (per_sm > 0 ? per_sm : 1), frac);
    const int64_t need_small = (nroots + 32 * (kThreads / 32) - 1) / (32 * (kThreads / 32));
    if (need_small < blocks) blocks = (int)std::max<int64_t>(1, need_small);
    k_clique_small<K><<<blocks, kThreads, 0, s>>>(v.dag_rp, v.dag_col, lo, hi, d_work, d_count, d_count4);
    GZ_COUNT_LAUNCH();
    if (v.max_out <= 32) {
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? GZ_OK : cuda_fail(e, "clique launch");
    }
    const int mo = (int)std::min<int64_t>(v.max_out, kCliqueMaxOut);
    GzView& mv = const_cast<GzView&>(v);
    gz_status st = gather_heavy(mv, n, s);
    if (st != GZ_OK) return st;
    st = build_heavy_rows(mv, mo, sms, s);
    if (st != GZ_OK) return st;
    // heavy roots of [lo, hi) with cached rows, heaviest first: for K <= 5 the
    // view's slot list (on the device already when all roots are counted), for
    // K >= 6 each root split into parts_for(K, d) slots
    std::vector<int4> ent;
    const int4* d_slots = nullptr;
    int nslots = 0;
    if (K <= 5 && mv.heavy_rows_ok && lo <= 0 && hi >= n) {
        d_slots = mv.slot_dev;
        nslots = (int)mv.slot_host.size();
    } else if (mv.heavy_rows_ok) {
        // the cached roots of [lo, hi), found in the root-sorted list, then
        // heaviest first
        auto it = std::lower_bound(mv.heavy.begin(), mv.heavy.end(), std::make_pair((int32_t)lo, INT32_MIN));
        for (; it != mv.heavy.end() && it->first < hi; ++it) {
            const size_t i = (size_t)(it - mv.heavy.begin());
            if (mv.heavy_off[i] == UINT32_MAX) continue;
            const int d = it->second;
            const int parts = K <= 5 ? 1 : parts_for(K, d);
            for (int p = 0; p < parts; ++p) ent.push_back(make_int4(it->first, p | (parts << 16), (int)mv.heavy_off[i], d));
        }
        std::stable_sort(ent.begin(), ent.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
    }
    // without cached rows no root is split (the chunk slots then take them all)
    const int heavy_d = mv.heavy_rows_ok ? kHeavyD : mo + 1;
    const size_t smem = ((size_t)mo * (K <= 5 ? row_stride(mo) : (((mo + 31) / 32) | 1)) + 2 * (size_t)mo + 1) * 4;
    int4* d_ent = nullptr;
    cudaError_t e = cudaSuccess;
    if (!ent.empty()) {
        e = gz_malloc_async(&d_ent, sizeof(int4) * ent.size(), s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_ent, ent.data(), sizeof(int4) * ent.size(), cudaMemcpyHostToDevice, s);
        d_slots = d_ent;
        nslots = (int)ent.size();
    }
    if (e == cudaSuccess) {
        const int64_t slots = (int64_t)nslots + (nroots + kBigPop - 1) / kBigPop;
        if constexpr (K <= 5) {
            auto kern = k_clique_warp<K, false>;
            if constexpr (K == 5) {
                if (d_count4) kern = k_clique_warp<5, true>;
            }
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpCta, smem);
            int bb = grid_part(sms * (per_sm > 0 ? per_sm : 1), frac);
            if (slots < bb) bb = (int)std::max<int64_t>(1, slots);
            if (e == cudaSuccess) {
                kern<<<bb, kWarpCta, smem, s>>>(v.dag_rp, v.dag_col, lo, hi, mo, heavy_d, d_slots, nslots,
                                                mv.heavy_rows, d_work + 1, d_count, d_count4);
                GZ_COUNT_LAUNCH();
            }
        } else {
            e = cudaFuncSetAttribute(k_clique_big<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_big<K>, kBigThreads, smem);
            int bb = grid_part(sms * (per_sm > 0 ? per_sm : 1), frac);
            if (slots < bb) bb = (int)std::max<int64_t>(1, slots);
            if (e == cudaSuccess) {
                k_clique_big<K><<<bb, kBigThreads, smem, s>>>(v.dag_rp, v.dag_col, lo, hi, mo, heavy_d, d_slots,
                                                               nslots, mv.heavy_rows, d_work + 1, d_count);
                GZ_COUNT_LAUNCH();
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (d_ent) cudaFreeAsync(d_ent, s);
    if (e != cudaSuccess) return cuda_fail(e, "clique launch");
    if (v.max_out > kCliqueMaxOut) return launch_long<K>(mv, lo, hi, frac, s, d_count, d_work + 2);
    return GZ_OK;
}

}  // namespace

bool clique_eligible(const GzProg& p, const gz_plan& plan, const GzView& v) {
    if (plan.k < 4 || plan.k > 8 || !v.has_dag) return false;
    for (int i = 0; i < plan.k; ++i)
        for (int j = 0; j < plan.k; ++j)
            if (i != j && !plan.adj[i * plan.k + j]) return false;
    for (int i = 1; i < plan.k; ++i)
        if (plan.bp[i] != i - 1) return false;
    (void)p;
    return true;
}

// Builds the per-view state the clique kernels share between calls (the heavy
// root list and their cached rows) on stream s, synchronously, so that later
// launches on any stream may use it.
gz_status clique_prepare(const GzView& v, int64_t n, cudaStream_t s) {
    if (!v.has_dag || v.max_out <= 32) return GZ_OK;
    GzView& mv = const_cast<GzView&>(v);
    gz_status st = gather_heavy(mv, n, s);
    if (st != GZ_OK) return st;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return build_heavy_rows(mv, (int)std::min<int64_t>(v.max_out, kCliqueMaxOut), sms, s);
}

// Adds the cliques of the roots in [lo, hi) whose out-list holds at most
// kCliqueLongOut vertices to *d_count; longer roots are left to the caller.
// d_work holds kCliqueWork zeroed counters.
gz_status clique_launch(int k, const GzView& v, int64_t n, int64_t lo, int64_t hi, double frac, cudaStream_t s,
                        unsigned long long* d_count, unsigned long long* d_work) {
    if (hi <= lo) return GZ_OK;
    switch (k) {
        case 4: return launch_k<4>(v, n, lo, hi, frac, s, d_count, d_work);
        case 5: return launch_k<5>(v, n, lo, hi, frac, s, d_count, d_work);
        case 6: return launch_k<6>(v, n, lo, hi, frac, s, d_count, d_work);
        case 7: return launch_k<7>(v, n, lo, hi, frac, s, d_count, d_work);
        case 8: return launch_k<8>(v, n, lo, hi, frac, s, d_count, d_work);
    }
    set_error("clique kernel: k = %d unsupported", k);
    return GZ_EINVAL;
}

bool clique45_fusable(const GzView& v) { return v.has_dag && v.max_out <= kCliqueMaxOut; }

// The fused K4 + K5 pass: one walk over the pairs (a, b) of every root adds the
// pair's K5 count to *d_count5 and its K4 count |row(a) & row(b)| to *d_count4
// (the K4 loops are a prefix of the K5 loops). Requires clique45_fusable(v).
gz_status clique_launch45(const GzView& v, int64_t n, int64_t lo, int64_t hi, double frac, cudaStream_t s,
                          unsigned long long* d_count5, unsigned long long* d_count4, unsigned long long* d_work) {
    if (hi <= lo) return GZ_OK;
    return launch_k<5>(v, n, lo, hi, frac, s, d_count5, d_work, d_count4);
}

}  // namespace gz
