// gz_graph.cu - device graph construction: CSR validation, the orientation pass
// (Sec. 6: reindex by decreasing degree, ties by original id), and the out-list
// (DAG) view N(v) intersect [0, v) used by bounded set operations.
//
// Every step is a streaming pass over the CSR, so the orientation is HBM-bound.
// The only sort is a stable LSD radix sort written here (8-bit digits, per-tile
// histograms, warp match-based stable ranks).
#include <cstdio>
#include <cstring>
#include <vector>

#include "gz_internal.h"

namespace gz {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                     // keys per thread in a radix tile
constexpr int kTile = kThreads * kItems;       // 4096 keys per tile
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

inline int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1ll << 30)) b = 1ll << 30;
    return (int)b;
}

// ------------------------------------------------------------------ scans

// Block-wide exclusive scan of kScanTile int64 values; writes the tile total.
__global__ void scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                           int64_t n, int64_t* __restrict__ tile_sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    // warp inclusive scan of per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;  // inclusive per warp
    }
    __syncthreads();
    int64_t run = incl - s + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == kScanThreads - 1 && tile_sums) tile_sums[blockIdx.x] = run;
}

__global__ void add_tile_offsets(int64_t* __restrict__ out, int64_t n,
                                 const int64_t* __restrict__ offs) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t add = offs[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

// Exclusive scan of n int64 values (in may alias out). Returns the total in
// *total_dev if non-null (device pointer, written by the last step).
cudaError_t exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        GZ_COUNT_LAUNCH();
        return cudaGetLastError();
    }
    int64_t* sums = nullptr;
    cudaError_t e = gz_malloc_async(&sums, sizeof(int64_t) * tiles, s);
    if (e != cudaSuccess) return e;
    scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
    GZ_COUNT_LAUNCH();
    e = exclusive_scan(sums, sums, tiles, s);
    if (e == cudaSuccess) {
        add_tile_offsets<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, sums);
        GZ_COUNT_LAUNCH();
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, s);
    return e;
}

// ------------------------------------------------------------------ radix sort

// Per-tile digit histogram, digit-major: hist[d * ntiles + tile].
__global__ void radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                           int64_t* __restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += kThreads) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kThreads) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += kThreads) hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Stable scatter of one tile. Warp w owns items [w*512, (w+1)*512) of the tile
// and walks them in order, 32 at a time; __match_any_sync groups equal digits,
// so ranks follow item order within the warp, and warps are ordered by index.
// The tile is first reordered by digit in shared memory, then written out
// run by run: consecutive threads write consecutive slots of one digit's run,
// so the stores fill whole sectors instead of one or two words per bucket.
__global__ void radix_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                              uint32_t* __restrict__ okeys, uint32_t* __restrict__ ovals,
                              int64_t n, int shift, const int64_t* __restrict__ offs,
                              int64_t ntiles) {
    constexpr int kWarps = kThreads / 32;
    constexpr int kPerWarp = kTile / kWarps;  // 512
    constexpr int kSteps = kPerWarp / 32;     // 16
    __shared__ uint32_t cnt[kWarps][256];
    __shared__ int64_t base_off[256];
    __shared__ uint32_t tstart[256];          // first slot of each digit in the reordered tile
    __shared__ uint32_t sk[kTile], sv[kTile];
    for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&cnt[0][0])[i] = 0;
    for (int i = threadIdx.x; i < 256; i += kThreads) base_off[i] = offs[(int64_t)i * ntiles + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tbase = (int64_t)blockIdx.x * kTile;
    const int64_t wbase = tbase + (int64_t)warp * kPerWarp;
    uint32_t k[kSteps], v[kSteps], r[kSteps];
#pragma unroll
    for (int st = 0; st < kSteps; ++st) {
        int64_t idx = wbase + st * 32 + lane;
        bool ok = idx < n;
        k[st] = ok ? keys[idx] : 0u;
        v[st] = ok ? vals[idx] : 0u;
        uint32_t dg = ok ? ((k[st] >> shift) & 255u) : 256u + lane;  // invalid lanes never match
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        uint32_t below = peers & ((1u << lane) - 1u);
        uint32_t prior = ok ? cnt[warp][dg] : 0u;
        r[st] = prior + __popc(below);
        __syncwarp();
        int leader = 31 - __clz(peers);
        if (ok && lane == leader) cnt[warp][dg] = prior + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps per digit; the digit's tile total goes to tstart
    for (int d = threadIdx.x; d < 256; d += kThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
        tstart[d] = run;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 256 digit totals, 8 per lane
        uint32_t t[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            t[j] = tstart[lane * 8 + j];
            sum += t[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            tstart[lane * 8 + j] = run;
            run += t[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int st = 0; st < kSteps; ++st) {
        int64_t idx = wbase + st * 32 + lane;
        if (idx < n) {
            uint32_t dg = (k[st] >> shift) & 255u;
            uint32_t lp = tstart[dg] + cnt[warp][dg] + r[st];
            sk[lp] = k[st];
            sv[lp] = v[st];
        }
    }
    __syncthreads();
    const int tn = (int)min((int64_t)kTile, n - tbase);
    for (int i = threadIdx.x; i < tn; i += kThreads) {
        const uint32_t kk = sk[i];
        const uint32_t dg = (kk >> shift) & 255u;
        const int64_t pos = base_off[dg] + (int64_t)(i - (int)tstart[dg]);
        okeys[pos] = kk;
        ovals[pos] = sv[i];
    }
}

// Stable sort of (key, value) pairs by the low `bits` bits of key, ping-ponging
// between (k0, v0) and (k1, v1): *rk, *rv receive the pair that holds the
// result (no copy back), the other pair is scratch afterwards.
cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n,
                             int bits, cudaStream_t s, uint32_t** rk, uint32_t** rv) {
    *rk = k0;
    *rv = v0;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    int64_t ntiles = (n + kTile - 1) / kTile;
    int64_t* hist = nullptr;
    cudaError_t e = gz_malloc_async(&hist, sizeof(int64_t) * 256 * ntiles, s);
    if (e != cudaSuccess) return e;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        int shift = 8 * p;
        radix_hist<<<(unsigned)ntiles, kThreads, 0, s>>>(k0, n, shift, hist, ntiles);
        GZ_COUNT_LAUNCH();
        e = exclusive_scan(hist, hist, 256 * ntiles, s);
        if (e != cudaSuccess) break;
        radix_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(k0, v0, k1, v1, n, shift, hist, ntiles);
        GZ_COUNT_LAUNCH();
        e = cudaGetLastError();
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    *rk = k0;
    *rv = v0;
    cudaFreeAsync(hist, s);
    return e;
}

// ------------------------------------------------------------------ graph kernels

__global__ void k_degrees(const int64_t* __restrict__ rp, int64_t n, int64_t* __restrict__ deg,
                          unsigned long long* __restrict__ maxdeg) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t d = 0;
    if (v < n) {
        d = rp[v + 1] - rp[v];
        if (deg) deg[v] = d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        int64_t t = __shfl_down_sync(0xffffffffu, d, o);
        d = t > d ? t : d;
    }
    if ((threadIdx.x & 31) == 0 && d > 0) atomicMax(maxdeg, (unsigned long long)d);
}

// err[0]: bad row_ptr, err[1]: out of range, err[2]: self-loop, err[3]: unsorted/dup,
// err[4]: asymmetric. One warp per vertex.
__global__ void k_validate(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           int64_t n, int64_t nnz, int symmetric,
                           unsigned long long* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        int64_t b = rp[v], e = rp[v + 1];
        if (b < 0 || e < b || e > nnz) {
            if (lane == 0) atomicAdd(&err[0], 1ull);
            continue;
        }
        for (int64_t i = b + lane; i < e; i += 32) {
            int32_t u = col[i];
            if (u < 0 || u >= n) { atomicAdd(&err[1], 1ull); continue; }
            if (u == v) atomicAdd(&err[2], 1ull);
            if (i > b && col[i - 1] >= u) atomicAdd(&err[3], 1ull);
            if (symmetric) {
                int64_t lo = rp[u], hi = rp[u + 1];
                if (lo < 0 || hi < lo || hi > nnz) continue;
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if (col[mid] < v) lo = mid + 1; else hi = mid;
                }
                if (lo >= rp[u + 1] || col[lo] != v) atomicAdd(&err[4], 1ull);
            }
        }
    }
}

// key = max_deg - deg (so ascending key = descending degree), value = id.
__global__ void k_rank_keys(const int64_t* __restrict__ deg, int64_t n, int64_t maxdeg,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        keys[v] = (uint32_t)(maxdeg - deg[v]);
        vals[v] = (uint32_t)v;
    }
}

// order[r] = old id at rank r -> new_id[old] = r, and the new degree array.
__global__ void k_new_ids(const uint32_t* __restrict__ order, const int64_t* __restrict__ deg,
                          int64_t n, int32_t* __restrict__ new_id, int64_t* __restrict__ ndeg) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        uint32_t v = order[r];
        new_id[v] = (int32_t)r;
        ndeg[r] = deg[v];
    }
}

// Row r of the new CSR gets old row order[r]: key = new id of the neighbour,
// value = r. One warp per row, coalesced over the row.
__global__ void k_relabel_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const uint32_t* __restrict__ order, const int32_t* __restrict__ new_id,
                               const int64_t* __restrict__ nrp, int64_t n,
                               uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        uint32_t v = order[r];
        int64_t b = rp[v], len = rp[v + 1] - b, o = nrp[r];
        for (int64_t i = lane; i < len; i += 32) {
            keys[o + i] = (uint32_t)new_id[col[b + i]];
            vals[o + i] = (uint32_t)r;
        }
    }
}

// After sorting by neighbour id, segment w must hold only key w (symmetry).
__global__ void k_check_segments(const uint32_t* __restrict__ keys, const int64_t* __restrict__ nrp,
                                 int64_t n, unsigned long long* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < n; w += nwarps) {
        for (int64_t i = nrp[w] + lane; i < nrp[w + 1]; i += 32)
            if (keys[i] != (uint32_t)w) atomicAdd(bad, 1ull);
    }
}

// split[v] = |N(v) intersect [0, v)| (lists sorted): one warp per vertex. The
// largest split goes to *maxout by one atomic per warp (a per-vertex atomic on
// one address serialises in L2).
__global__ void k_split(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                        int64_t* __restrict__ split, unsigned long long* __restrict__ maxout) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t wmax = 0;
    for (int64_t v = warp; v < n; v += nwarps) {
        int64_t b = rp[v], e = rp[v + 1];
        int64_t cnt = 0;
        for (int64_t i = b + lane; i < e; i += 32) {
            bool lt = col[i] < v;
            unsigned m = __ballot_sync(__activemask(), lt);
            cnt += __popc(m);
            if (!__shfl_sync(__activemask(), lt ? 1 : 0, 31 - __clz(__activemask()))) break;
        }
        cnt = __shfl_sync(0xffffffffu, cnt, 0);
        if (lane == 0) split[v] = cnt;
        wmax = cnt > wmax ? cnt : wmax;
    }
    if (lane == 0 && wmax > 0) atomicMax(maxout, (unsigned long long)wmax);
}

__global__ void k_dag_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ drp, int64_t n, int32_t* __restrict__ dcol,
                           int32_t* __restrict__ dsrc) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        int64_t b = rp[v], o = drp[v], len = drp[v + 1] - o;
        for (int64_t i = lane; i < len; i += 32) {
            dcol[o + i] = col[b + i];
            dsrc[o + i] = (int32_t)v;
        }
    }
}

__global__ void k_src(const int64_t* __restrict__ rp, int64_t n, int32_t* __restrict__ src) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps)
        for (int64_t i = rp[v] + lane; i < rp[v + 1]; i += 32) src[i] = (int32_t)v;
}

inline int warp_grid(int64_t n) {
    int64_t b = (n * 32 + kThreads - 1) / kThreads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

int bits_for(uint64_t x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

}  // namespace

// Device-wide helpers used by the API layer.
gz_status max_degree(const int64_t* rp, int64_t n, int64_t* out, cudaStream_t s) {
    unsigned long long* d = nullptr;
    cudaError_t e = gz_malloc_async(&d, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
    if (n > 0) {
        k_degrees<<<grid_for(n, kThreads), kThreads, 0, s>>>(rp, n, nullptr, d);
        GZ_COUNT_LAUNCH();
    }
    unsigned long long h = 0;
    e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "max degree");
    *out = (int64_t)h;
    return GZ_OK;
}

gz_status validate_csr(const int64_t* rp, const int32_t* col, int64_t n, int64_t nnz,
                       bool symmetric, cudaStream_t s) {
    // row_ptr endpoints on the host
    int64_t ends[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&ends[0], rp, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ends[1], rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "validate: read row_ptr");
    if (ends[0] != 0 || ends[1] != nnz) {
        set_error("gz_load_csr: row_ptr[0] = %lld, row_ptr[n] = %lld, expected 0 and nnz = %lld",
                  (long long)ends[0], (long long)ends[1], (long long)nnz);
        return GZ_EINVAL;
    }
    if (n == 0) return GZ_OK;
    unsigned long long* err = nullptr;
    e = gz_malloc_async(&err, sizeof(unsigned long long) * 5, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaMemsetAsync(err, 0, sizeof(unsigned long long) * 5, s);
    k_validate<<<warp_grid(n), kThreads, 0, s>>>(rp, col, n, nnz, symmetric ? 1 : 0, err);
    GZ_COUNT_LAUNCH();
    unsigned long long h[5];
    e = cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "validate");
    const char* what[5] = {"row_ptr not monotone", "column id out of range", "self-loop",
                           "list not strictly increasing (unsorted or duplicate)",
                           "graph not symmetric"};
    for (int i = 0; i < 5; ++i)
        if (h[i]) {
            set_error("gz_load_csr: invalid CSR: %s (%llu entries)", what[i], h[i]);
            return GZ_EINVAL;
        }
    return GZ_OK;
}

gz_status build_dag(gz_graph* g, GzView* v, cudaStream_t s) {
    if (v->has_dag) return GZ_OK;
    const int64_t n = g->n;
    cudaError_t e;
    if (!v->dag_rp) {  // kept across rebuilds of the view (same n)
        e = gz_malloc(&v->dag_rp, sizeof(int64_t) * (n + 1));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc dag_rp");
    }
    unsigned long long* mx = nullptr;
    e = gz_malloc_async(&mx, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(v->dag_rp + n, 0, sizeof(int64_t), s);
    if (n > 0) {
        k_split<<<warp_grid(n), kThreads, 0, s>>>(v->rp, v->col, n, v->dag_rp, mx);
        GZ_COUNT_LAUNCH();
    }
    e = exclusive_scan(v->dag_rp, v->dag_rp, n + 1, s);
    int64_t dnnz = 0;
    unsigned long long hmx = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&dnnz, v->dag_rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(mx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "build dag: split");
    const int64_t need = dnnz > 0 ? dnnz : 1;
    if (need > v->dag_cap) {  // grow; a rebuild of the same view reuses the arrays
        cudaFree(v->dag_col);
        cudaFree(v->dag_src);
        v->dag_col = nullptr;
        v->dag_src = nullptr;
        v->dag_cap = 0;
        const size_t bytes = sizeof(int32_t) * (size_t)need;
        e = gz_malloc(&v->dag_col, bytes);
        if (e == cudaSuccess) e = gz_malloc(&v->dag_src, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc dag");
        v->dag_cap = need;
    }
    if (n > 0) {
        k_dag_fill<<<warp_grid(n), kThreads, 0, s>>>(v->rp, v->col, v->dag_rp, n, v->dag_col, v->dag_src);
        GZ_COUNT_LAUNCH();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "build dag: fill");
    v->dag_nnz = dnnz;
    v->max_out = (int64_t)hmx;
    v->has_dag = true;
    return GZ_OK;
}

gz_status build_src(gz_graph* g, GzView* v, cudaStream_t s) {
    if (v->src) return GZ_OK;
    cudaError_t e = gz_malloc(&v->src, sizeof(int32_t) * (size_t)(g->nnz > 0 ? g->nnz : 1));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc src");
    if (g->n > 0) {
        k_src<<<warp_grid(g->n), kThreads, 0, s>>>(v->rp, g->n, v->src);
        GZ_COUNT_LAUNCH();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "build src");
    return GZ_OK;
}

// Sec. 6 reindexing on the device. See the file comment for the steps.
gz_status orient(gz_graph* g, cudaStream_t s) {
    const int64_t n = g->n, nnz = g->nnz;
    if (n > (int64_t)INT32_MAX || nnz > ((int64_t)1 << 40)) {
        set_error("gz_orient: graph too large");
        return GZ_EOVERFLOW;
    }
    GzView& o = g->ori;
    cudaError_t e = cudaSuccess;
    if (g->oriented) {
        // the oriented view is rewritten in place: counts still running on other
        // streams may read it
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "gz_orient: wait for running counts");
    }
    if (!o.rp) {
        e = gz_malloc(&o.rp, sizeof(int64_t) * (n + 1));
        if (e == cudaSuccess) e = gz_malloc(&o.col, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        if (e == cudaSuccess) e = gz_malloc(&g->new_id, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc oriented CSR");
    }
    if (n == 0) {
        cudaMemsetAsync(o.rp, 0, sizeof(int64_t), s);
        g->oriented = true;
        return build_dag(g, &o, s);
    }
    const int64_t m2 = nnz > n ? nnz : n;
    uint32_t *k0 = nullptr, *v0 = nullptr, *k1 = nullptr, *v1 = nullptr;
    int64_t *deg = nullptr, *ndeg = nullptr;
    e = gz_malloc_async(&k0, sizeof(uint32_t) * m2, s);
    if (e == cudaSuccess) e = gz_malloc_async(&v0, sizeof(uint32_t) * m2, s);
    if (e == cudaSuccess) e = gz_malloc_async(&k1, sizeof(uint32_t) * m2, s);
    if (e == cudaSuccess) e = gz_malloc_async(&v1, sizeof(uint32_t) * m2, s);
    if (e == cudaSuccess) e = gz_malloc_async(&deg, sizeof(int64_t) * (n + 1), s);
    if (e == cudaSuccess) e = gz_malloc_async(&ndeg, sizeof(int64_t) * (n + 1), s);
    gz_status st = GZ_OK;
    unsigned long long* bad = nullptr;
    if (e == cudaSuccess) e = gz_malloc_async(&bad, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { st = cuda_fail(e, "gz_orient: temporaries"); goto done; }
    {
        cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
        // 1. degrees -> rank keys (max_deg - deg), stable sort by key
        k_degrees<<<grid_for(n, kThreads), kThreads, 0, s>>>(g->orig.rp, n, deg, bad);
        GZ_COUNT_LAUNCH();
        cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
        k_rank_keys<<<grid_for(n, kThreads), kThreads, 0, s>>>(deg, n, g->max_deg, k0, v0);
        GZ_COUNT_LAUNCH();
        uint32_t *rk = nullptr, *order = nullptr;
        e = radix_sort_pairs(k0, v0, k1, v1, n, bits_for((uint64_t)g->max_deg), s, &rk, &order);
        if (e != cudaSuccess) { st = cuda_fail(e, "gz_orient: rank sort"); goto done; }
        // 2. new ids and new row pointers (order: old id per rank)
        k_new_ids<<<grid_for(n, kThreads), kThreads, 0, s>>>(order, deg, n, g->new_id, ndeg);
        GZ_COUNT_LAUNCH();
        cudaMemsetAsync(ndeg + n, 0, sizeof(int64_t), s);
        e = exclusive_scan(ndeg, o.rp, n + 1, s);
        if (e != cudaSuccess) { st = cuda_fail(e, "gz_orient: row scan"); goto done; }
        // 3. relabel rows in rank order into the pair that does not hold the
        //    order, then stable sort by neighbour id (the order's pair is the
        //    scratch, overwritten only after the relabel, in stream order): each
        //    segment then lists its neighbours' ranks in ascending order.
        uint32_t* ak = order == v0 ? k1 : k0;
        uint32_t* av = order == v0 ? v1 : v0;
        uint32_t* bk = order == v0 ? k0 : k1;
        uint32_t* bv = order == v0 ? v0 : v1;
        k_relabel_rows<<<warp_grid(n), kThreads, 0, s>>>(g->orig.rp, g->orig.col, order,
                                                        g->new_id, o.rp, n, ak, av);
        GZ_COUNT_LAUNCH();
        uint32_t *sk = nullptr, *sv = nullptr;
        e = radix_sort_pairs(ak, av, bk, bv, nnz, bits_for((uint64_t)(n - 1)), s, &sk, &sv);
        if (e != cudaSuccess) { st = cuda_fail(e, "gz_orient: edge sort"); goto done; }
        k_check_segments<<<warp_grid(n), kThreads, 0, s>>>(sk, o.rp, n, bad);
        GZ_COUNT_LAUNCH();
        e = cudaMemcpyAsync(o.col, sv, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s);
        unsigned long long hbad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_fail(e, "gz_orient: relabel"); goto done; }
        if (hbad) {
            set_error("gz_orient: graph is not symmetric (%llu misplaced entries)", hbad);
            st = GZ_EINVAL;
            goto done;
        }
        // 4. out-list (DAG) view of the reindexed graph, rebuilt every time
        if (o.has_dag) {  // rebuilt below into the same allocations
            o.has_dag = false;
            o.heavy.clear();
            o.heavy_built = false;
            o.heavy_off.clear();
            o.heavy_rows_built = false;
            o.heavy_rows_ok = false;
        }
        if (o.src) { cudaFree(o.src); o.src = nullptr; }
        st = build_dag(g, &o, s);
        if (st == GZ_OK) g->oriented = true;
    }
done:
    cudaFreeAsync(k0, s); cudaFreeAsync(v0, s); cudaFreeAsync(k1, s); cudaFreeAsync(v1, s);
    cudaFreeAsync(deg, s); cudaFreeAsync(ndeg, s); cudaFreeAsync(bad, s);
    return st;
}

}  // namespace gz
