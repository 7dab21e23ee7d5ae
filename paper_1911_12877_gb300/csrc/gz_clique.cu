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
//  - k_clique_big: one 512-thread CTA per root with 32 < |O| <= kCliqueMaxOut,
//    rows in shared memory (odd word stride), then the (a, b) edges of the
//    local DAG spread over all threads. Roots with |O| >= kHeavyD are split
//    over several CTAs ("parts"); their rows are built once per out-list view
//    by k_clique_rows into device memory and copied by each part.
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
constexpr int kHeavyD = 128;    // out-degree from which a root is split over several CTAs
constexpr uint64_t kHeavyRowWords = 1ull << 29;  // budget for prebuilt heavy rows (2 GiB)
constexpr uint64_t kLongRowWords = 1ull << 30;   // budget for long roots' global rows (4 GiB)

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
template <int K>
__global__ void __launch_bounds__(kThreads) k_clique_small(const int64_t* __restrict__ drp,
                                                           const int32_t* __restrict__ dcol,
                                                           int64_t root_lo, int64_t root_hi,
                                                           unsigned long long* __restrict__ work,
                                                           unsigned long long* __restrict__ count) {
    __shared__ uint32_t rows_s[kThreads / 32][32];
    __shared__ unsigned long long red[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* rows = rows_s[warp];
    unsigned long long acc = 0;
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
            if (d < K - 1 || d > 32) continue;
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
                }
            }
            __syncwarp();
        }
    }
    unsigned long long s = block_sum(acc, red);
    if (threadIdx.x == 0 && s) atomicAdd(count, s);
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

// Rows of every heavy root, built once into global memory (one CTA per root,
// grid-stride), so the parts of a heavy root copy them instead of rebuilding.
// hr[i] = (root, unused, word offset of its rows in grows). Shared memory as in
// k_clique_big (rows, O).
__global__ void __launch_bounds__(kThreads) k_clique_rows(const int64_t* __restrict__ drp,
                                                          const int32_t* __restrict__ dcol,
                                                          const int4* __restrict__ hr, int nh,
                                                          int max_out,
                                                          uint32_t* __restrict__ grows) {
    extern __shared__ uint32_t sm[];
    const int Wsmax = ((max_out + 31) >> 5) | 1;
    uint32_t* rows = sm;
    int32_t* O = reinterpret_cast<int32_t*>(sm + (size_t)max_out * Wsmax);
    // index of O: open-addressing hash of (vertex id << 32 | position), 2 *
    // kCliqueMaxOut slots (load <= 1/2); 8-byte aligned after rows and O
    const size_t hoff = ((size_t)max_out * Wsmax + max_out + 1) & ~(size_t)1;
    unsigned long long* hx = reinterpret_cast<unsigned long long*>(sm + hoff);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t* stage = reinterpret_cast<int32_t*>(hx + 2 * kCliqueMaxOut) + (size_t)warp * kCliqueMaxOut;
    constexpr unsigned kMask = 2 * kCliqueMaxOut - 1;
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int64_t v = hr[h].x;
        const int64_t ob = drp[v];
        const int d = (int)(drp[v + 1] - ob);
        const int Ws = ((d + 31) >> 5) | 1;
        for (int i = threadIdx.x; i < 2 * kCliqueMaxOut; i += kThreads) hx[i] = ~0ull;
        for (int i = threadIdx.x; i < d * Ws; i += kThreads) rows[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += kThreads) {
            const int32_t x = dcol[ob + i];
            O[i] = x;
            const unsigned long long kv = ((unsigned long long)(uint32_t)x << 32) | (uint32_t)i;
            unsigned sl = ((uint32_t)x * 0x9E3779B1u) >> 21;  // 11 bits: 2048 slots
            while (atomicCAS(&hx[sl], ~0ull, kv) != ~0ull) sl = (sl + 1) & kMask;
        }
        __syncthreads();
        // row(a): stream N'(O[a]) and look each entry up in the index of O (one
        // probe instead of a binary search) when it is not much longer than a;
        // else stage it and binary-search it for each O[b], b < a
        for (int a = warp + 1; a < d; a += kThreads / 32) {
            const int32_t u = O[a];
            const int64_t ub = drp[u];
            const int du = (int)(drp[u + 1] - ub);
            uint32_t* ra = rows + (size_t)a * Ws;
            if (du <= 4 * a || du > kCliqueMaxOut) {
                for (int i = lane; i < du; i += 32) {
                    const int32_t x = __ldg(dcol + ub + i);
                    unsigned sl = ((uint32_t)x * 0x9E3779B1u) >> 21;
                    int b = -1;
                    for (;;) {
                        const unsigned long long e = hx[sl];
                        if (e == ~0ull) break;
                        if ((int32_t)(e >> 32) == x) { b = (int)(uint32_t)e; break; }
                        sl = (sl + 1) & kMask;
                    }
                    if (b >= 0 && b < a) atomicOr(ra + (b >> 5), 1u << (b & 31));
                }
            } else {
                for (int i = lane; i < du; i += 32) stage[i] = __ldg(dcol + ub + i);
                __syncwarp();
                for (int b0 = 0; b0 < a; b0 += 32) {
                    const int b = b0 + lane;
                    const bool in = b < a && index_of(stage, du, O[b]) >= 0;
                    const uint32_t m = __ballot_sync(kFull, in);
                    if (lane == 0) ra[b0 >> 5] = m;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        uint32_t* dst = grows + (uint32_t)hr[h].z;
        for (int i = threadIdx.x; i < d * Ws; i += kThreads) dst[i] = rows[i];
        __syncthreads();
    }
}

// Roots with 32 < |O| <= max_out: one CTA per root, or per part of a heavy
// root. Shared memory: rows [max_out * Wsmax] words (row stride Ws = W | 1 for
// the current root, odd so that threads reading word w of different rows hit
// different banks), O [max_out], pre [max_out + 1].
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
            for (int i = threadIdx.x; i < d * Ws; i += kBigThreads) rows[i] = __ldg(src + i);
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
__global__ void k_collect_heavy(const int64_t* __restrict__ drp, int64_t n, int heavy_d,
                                int2* __restrict__ out, unsigned long long* __restrict__ cnt,
                                int64_t cap) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = drp[v + 1] - drp[v];
        if (d >= heavy_d) {
            const unsigned long long i = atomicAdd(cnt, 1ull);
            if (out && (int64_t)i < cap) out[i] = make_int2((int)v, (int)d);
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
    unsigned long long* cnt = nullptr;
    cudaError_t e = gz_malloc_async(&cnt, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "clique: heavy roots");
    int64_t gb = (n + 255) / 256;
    const int grid = (int)std::min<int64_t>(gb, 152 * 16);
    unsigned long long h = 0;
    e = cudaMemsetAsync(cnt, 0, sizeof(h), s);
    if (e == cudaSuccess) {
        k_collect_heavy<<<grid, 256, 0, s>>>(v.dag_rp, n, kHeavyD, nullptr, cnt, 0);
        GZ_COUNT_LAUNCH();
        e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int2* d_out = nullptr;
    std::vector<int2> tmp(h);
    if (e == cudaSuccess && h > 0) {
        e = gz_malloc_async(&d_out, sizeof(int2) * h, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess) {
            k_collect_heavy<<<grid, 256, 0, s>>>(v.dag_rp, n, kHeavyD, d_out, cnt, (int64_t)h);
            GZ_COUNT_LAUNCH();
            e = cudaMemcpyAsync(tmp.data(), d_out, sizeof(int2) * h, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(d_out, s);
    }
    cudaFreeAsync(cnt, s);
    if (e != cudaSuccess) return cuda_fail(e, "clique: heavy roots");
    v.heavy.reserve(h);
    for (const int2& x : tmp) v.heavy.emplace_back(x.x, x.y);
    std::sort(v.heavy.begin(), v.heavy.end());
    v.heavy_built = true;
    return GZ_OK;
}

// Parts a heavy root is split into: about its work (d^2 for K = 4, d^3 beyond)
// over that of a root of out-degree kHeavyD, at most 64 and at most d. Parts
// copy the root's prebuilt rows, so a part costs little beyond its share.
int parts_for(int K, int d) {
    const double r = (double)d / kHeavyD;
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
    v.heavy_off.assign(v.heavy.size(), UINT32_MAX);
    std::vector<int4> list;
    uint64_t words = 0;
    for (size_t i = 0; i < v.heavy.size(); ++i) {
        const int d = v.heavy[i].second;
        if (d > mo) continue;
        v.heavy_off[i] = (uint32_t)words;
        list.push_back(make_int4(v.heavy[i].first, 0, (int)words, 0));
        words += ((uint64_t)d * (((d + 31) / 32) | 1) + 3) & ~3ull;
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
    if (e == cudaSuccess) e = gz_malloc_async(&d_list, sizeof(int4) * list.size(), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_list, list.data(), sizeof(int4) * list.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const size_t hoff = ((size_t)mo * (((mo + 31) / 32) | 1) + mo + 1) & ~(size_t)1;
        const size_t smem = (hoff + 2 * 2 * (size_t)kCliqueMaxOut + (size_t)(kThreads / 32) * kCliqueMaxOut) * 4;
        cudaFuncSetAttribute(k_clique_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_rows, kThreads, smem);
        const int rb = (int)std::min<size_t>(list.size(), (size_t)sms * std::max(1, per_sm));
        k_clique_rows<<<rb, kThreads, smem, s>>>(v.dag_rp, v.dag_col, d_list, (int)list.size(), mo,
                                                 v.heavy_rows);
        GZ_COUNT_LAUNCH();
        e = cudaGetLastError();
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
    return GZ_OK;
}

// Roots of [lo, hi) with kCliqueMaxOut < |O| <= kCliqueLongOut: rows built in
// global memory (at most kLongRowWords words; roots beyond that budget, and
// roots longer than kCliqueLongOut, are left to the caller's general kernel,
// see clique_long_cutoff), then their edges walked by k_clique_long.
template <int K>
gz_status launch_long(GzView& v, int64_t lo, int64_t hi, cudaStream_t s,
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
        const int rb = (int)std::min<size_t>(build.size(), (size_t)sms * 4);
        k_clique_long_rows<<<rb, kThreads, smem, s>>>(v.dag_rp, v.dag_col, d_l, (int)build.size(), grows);
        GZ_COUNT_LAUNCH();
        const int lb = (int)std::min<size_t>(ent.size(), (size_t)sms * 4);
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

template <int K>
gz_status launch_k(const GzView& v, int64_t n, int64_t lo, int64_t hi, cudaStream_t s,
                   unsigned long long* d_count, unsigned long long* d_work) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_small<K>, kThreads, 0);
    const int64_t nroots = hi - lo;
    int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need_small = (nroots + 32 * (kThreads / 32) - 1) / (32 * (kThreads / 32));
    if (need_small < blocks) blocks = (int)std::max<int64_t>(1, need_small);
    k_clique_small<K><<<blocks, kThreads, 0, s>>>(v.dag_rp, v.dag_col, lo, hi, d_work, d_count);
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
    // heavy roots of [lo, hi) with cached rows, heaviest first, each split into parts
    std::vector<int> hi_idx;
    auto it = std::lower_bound(mv.heavy.begin(), mv.heavy.end(), std::make_pair((int32_t)lo, INT32_MIN));
    for (; it != mv.heavy.end() && it->first < hi; ++it) {
        const size_t i = (size_t)(it - mv.heavy.begin());
        if (mv.heavy_rows_ok && mv.heavy_off[i] != UINT32_MAX) hi_idx.push_back((int)i);
    }
    std::stable_sort(hi_idx.begin(), hi_idx.end(), [&](int a, int b) {
        return mv.heavy[a].second > mv.heavy[b].second;
    });
    std::vector<int4> ent;
    for (int i : hi_idx) {
        const int parts = parts_for(K, mv.heavy[i].second);
        for (int p = 0; p < parts; ++p)
            ent.push_back(make_int4(mv.heavy[i].first, p | (parts << 16), (int)mv.heavy_off[i], 0));
    }
    // without cached rows no root is split (the chunk slots then take them all)
    const int heavy_d = mv.heavy_rows_ok ? kHeavyD : mo + 1;
    const size_t smem = ((size_t)mo * (((mo + 31) / 32) | 1) + 2 * (size_t)mo + 1) * 4;
    int4* d_ent = nullptr;
    cudaError_t e = cudaSuccess;
    if (!ent.empty()) {
        e = gz_malloc_async(&d_ent, sizeof(int4) * ent.size(), s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_ent, ent.data(), sizeof(int4) * ent.size(), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        cudaFuncSetAttribute(k_clique_big<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_big<K>, kBigThreads, smem);
        int bb = sms * (per_sm > 0 ? per_sm : 1);
        const int64_t slots = (int64_t)ent.size() + (nroots + kBigPop - 1) / kBigPop;
        if (slots < bb) bb = (int)std::max<int64_t>(1, slots);
        k_clique_big<K><<<bb, kBigThreads, smem, s>>>(v.dag_rp, v.dag_col, lo, hi, mo, heavy_d, d_ent,
                                                       (int)ent.size(), mv.heavy_rows, d_work + 1, d_count);
        GZ_COUNT_LAUNCH();
        e = cudaGetLastError();
    }
    if (d_ent) cudaFreeAsync(d_ent, s);
    if (e != cudaSuccess) return cuda_fail(e, "clique launch");
    if (v.max_out > kCliqueMaxOut) return launch_long<K>(mv, lo, hi, s, d_count, d_work + 2);
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
// d_work holds three zeroed counters.
gz_status clique_launch(int k, const GzView& v, int64_t n, int64_t lo, int64_t hi, cudaStream_t s,
                        unsigned long long* d_count, unsigned long long* d_work) {
    if (hi <= lo) return GZ_OK;
    switch (k) {
        case 4: return launch_k<4>(v, n, lo, hi, s, d_count, d_work);
        case 5: return launch_k<5>(v, n, lo, hi, s, d_count, d_work);
        case 6: return launch_k<6>(v, n, lo, hi, s, d_count, d_work);
        case 7: return launch_k<7>(v, n, lo, hi, s, d_count, d_work);
        case 8: return launch_k<8>(v, n, lo, hi, s, d_count, d_work);
    }
    set_error("clique kernel: k = %d unsupported", k);
    return GZ_EINVAL;
}

}  // namespace gz
