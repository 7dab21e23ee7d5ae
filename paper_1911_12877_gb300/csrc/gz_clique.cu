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
//  - k_clique_big: one CTA per root with 32 < |O| <= kCliqueMaxOut; rows built
//    cooperatively (each row streams the shorter of O[0, a) and N(O[a])),
//    then the (a, b) pairs of the local DAG are spread over all threads.
#include <algorithm>
#include <cstdio>

#include "gz_internal.h"

namespace gz {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

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

// Sum over the cliques that extend the set AND(rs[0..nr)) (bits < lim) by
// DEPTH more vertices, each below the previous one; DEPTH == 1 is a popcount.
template <int DEPTH>
__device__ unsigned long long extend(const uint32_t* rows, int W, const uint32_t** rs, int nr, int lim) {
    const int words = (lim + 31) >> 5;
    unsigned long long cnt = 0;
    if constexpr (DEPTH == 1) {
        for (int w = 0; w < words; ++w) {
            uint32_t s = rs[0][w];
            for (int i = 1; i < nr; ++i) s &= rs[i][w];
            cnt += __popc(s);
        }
    } else {
        for (int w = 0; w < words; ++w) {
            uint32_t s = rs[0][w];
            for (int i = 1; i < nr; ++i) s &= rs[i][w];
            while (s) {
                const int c = (w << 5) + __ffs(s) - 1;
                s &= s - 1;
                rs[nr] = rows + (size_t)c * W;
                cnt += extend<DEPTH - 1>(rows, W, rs, nr + 1, c);
            }
        }
    }
    return cnt;
}

template <int K>
__device__ __forceinline__ unsigned long long count_pair(const uint32_t* rows, int W, int a, int b) {
    const uint32_t* rs[K];
    rs[0] = rows + (size_t)a * W;
    rs[1] = rows + (size_t)b * W;
    return extend<K - 3>(rows, W, rs, 2, b);
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

// Roots with 32 < |O| <= max_out: one CTA per root. Shared memory layout:
// rows [max_out * W] words, O [max_out], pre [max_out + 1].
template <int K>
__global__ void __launch_bounds__(kThreads) k_clique_big(const int64_t* __restrict__ drp,
                                                         const int32_t* __restrict__ dcol,
                                                         int64_t root_lo, int64_t root_hi,
                                                         int max_out,
                                                         unsigned long long* __restrict__ work,
                                                         unsigned long long* __restrict__ count) {
    extern __shared__ uint32_t sm[];
    __shared__ unsigned long long red[kThreads / 32];
    __shared__ int64_t s_root;
    const int Wmax = (max_out + 31) >> 5;
    uint32_t* rows = sm;
    int32_t* O = reinterpret_cast<int32_t*>(sm + (size_t)max_out * Wmax);
    int32_t* pre = O + max_out;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = kThreads / 32;
    unsigned long long acc = 0;
    constexpr int kPop = 16;  // roots per queue pop; most of them are small and skipped
    for (;;) {
        if (threadIdx.x == 0) s_root = root_lo + (int64_t)atomicAdd(work, (unsigned long long)kPop);
        __syncthreads();
        const int64_t v0 = s_root;
        __syncthreads();
        if (v0 >= root_hi) break;
      for (int r = 0; r < kPop; ++r) {
        const int64_t v = v0 + r;
        if (v >= root_hi) break;
        const int64_t ob = drp[v];
        const int d = (int)(drp[v + 1] - ob);
        if (d <= 32 || d > max_out) continue;
        const int W = (d + 31) >> 5;
        for (int i = threadIdx.x; i < d; i += kThreads) O[i] = dcol[ob + i];
        for (int i = threadIdx.x; i < d * W; i += kThreads) rows[i] = 0;
        __syncthreads();
        // rows: warp per a; stream the shorter of O[0, a) and N(O[a])
        for (int a = warp + 1; a < d; a += nwarps) {
            const int32_t u = O[a];
            const int64_t ub = drp[u];
            const int du = (int)(drp[u + 1] - ub);
            uint32_t* ra = rows + (size_t)a * W;
            if (du < a) {
                for (int i = lane; i < du; i += 32) {
                    const int b = index_of(O, a, __ldg(dcol + ub + i));
                    if (b >= 0) atomicOr(ra + (b >> 5), 1u << (b & 31));
                }
            } else {
                for (int b0 = 0; b0 < a; b0 += 32) {
                    const int b = b0 + lane;
                    const bool in = b < a && has(dcol + ub, du, O[b]);
                    const uint32_t m = __ballot_sync(kFull, in);
                    if (lane == 0) ra[b0 >> 5] = m;
                }
            }
        }
        __syncthreads();
        // pre[a] = number of local edges (a, b), b < a, before row a
        if (warp == 0) {
            int run = 0;
            for (int a0 = 0; a0 < d; a0 += 32) {
                const int a = a0 + lane;
                int c = 0;
                if (a < d)
                    for (int w = 0; w < W; ++w) c += __popc(rows[(size_t)a * W + w]);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                if (a < d) pre[a] = run + incl - c;
                run += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) pre[d] = run;
        }
        __syncthreads();
        const int pairs = pre[d];
        for (int p = threadIdx.x; p < pairs; p += kThreads) {
            int lo = 0, hi = d - 1;  // last a with pre[a] <= p
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= p) lo = mid; else hi = mid - 1;
            }
            const int a = lo;
            int j = p - pre[a];
            const uint32_t* ra = rows + (size_t)a * W;
            int b = -1;
            for (int w = 0; w < W; ++w) {
                uint32_t m = ra[w];
                const int c = __popc(m);
                if (j < c) {
                    for (int i = 0; i < j; ++i) m &= m - 1;
                    b = (w << 5) + __ffs(m) - 1;
                    break;
                }
                j -= c;
            }
            acc += count_pair<K>(rows, W, a, b);
        }
        __syncthreads();
      }
    }
    unsigned long long s = block_sum(acc, red);
    if (threadIdx.x == 0 && s) atomicAdd(count, s);
}

template <int K>
gz_status launch_k(const GzView& v, int64_t lo, int64_t hi, cudaStream_t s, unsigned long long* d_count,
                   unsigned long long* d_work) {
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
    if (v.max_out > 32) {
        const int mo = (int)v.max_out;
        const size_t smem = ((size_t)mo * ((mo + 31) / 32) + 2 * (size_t)mo + 2) * 4;
        cudaFuncSetAttribute(k_clique_big<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clique_big<K>, kThreads, smem);
        int bb = sms * (per_sm > 0 ? per_sm : 1);
        if (nroots < bb) bb = (int)std::max<int64_t>(1, nroots);
        k_clique_big<K><<<bb, kThreads, smem, s>>>(v.dag_rp, v.dag_col, lo, hi, mo, d_work + 1, d_count);
        GZ_COUNT_LAUNCH();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clique launch");
    return GZ_OK;
}

}  // namespace

bool clique_eligible(const GzProg& p, const gz_plan& plan, const GzView& v) {
    if (plan.k < 4 || plan.k > 8 || !v.has_dag || v.max_out > kCliqueMaxOut) return false;
    for (int i = 0; i < plan.k; ++i)
        for (int j = 0; j < plan.k; ++j)
            if (i != j && !plan.adj[i * plan.k + j]) return false;
    for (int i = 1; i < plan.k; ++i)
        if (plan.bp[i] != i - 1) return false;
    (void)p;
    return true;
}

// d_count must be zeroed; d_work holds two zeroed counters.
gz_status clique_launch(int k, const GzView& v, int64_t lo, int64_t hi, cudaStream_t s,
                        unsigned long long* d_count, unsigned long long* d_work) {
    if (hi <= lo) return GZ_OK;
    switch (k) {
        case 4: return launch_k<4>(v, lo, hi, s, d_count, d_work);
        case 5: return launch_k<5>(v, lo, hi, s, d_count, d_work);
        case 6: return launch_k<6>(v, lo, hi, s, d_count, d_work);
        case 7: return launch_k<7>(v, lo, hi, s, d_count, d_work);
        case 8: return launch_k<8>(v, lo, hi, s, d_count, d_work);
    }
    set_error("clique kernel: k = %d unsupported", k);
    return GZ_EINVAL;
}

}  // namespace gz
