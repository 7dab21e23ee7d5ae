// gz_noalloc.cu - gz_count_noalloc: pattern counting without any device
// allocation, for callers that must not allocate at counting time: real-time
// loops that forbid allocator calls after start-up, and host applications whose
// own memory manager reserves the whole device. The paper has no counterpart;
// this is a deployment variant of the general enumeration kernel.
//
// All device state of a call (queue counter, count, status and the per-warp
// set-operation scratch) lives in one file-scope static device array of fixed
// size, loaded with the library and held by every GPU that uses it until the
// process exits. Every call reuses that array: calls whose kernels overlap on
// the GPU (on different streams, or from several host threads) race on it and
// must be serialised by the caller. The array's device address is looked up
// once per device and kept, so it goes stale if the device is reset.
#include <mutex>

#include "gz_internal.h"

namespace gz {
gz_status prepare_check(const gz_plan* p, const gz_graph* g, int use_orientation, Query& q);
}

using namespace gz;

namespace {

// Counters first (kRegionHeader bytes), then GZ_NOALLOC_SCRATCH_BYTES of scratch.
static __device__ __align__(256) unsigned char g_region[kRegionHeader + GZ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_region_addr[kMaxDevices] = {};

// Device address of g_region on the current device, looked up once per device.
// In host code g_region names a host-side shadow, not device memory, so its
// address must come from cudaGetSymbolAddress with the device current.
gz_status region_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "gz_count_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gz_count_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
        return GZ_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_region_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_region);
        if (e != cudaSuccess || !p) return cuda_fail(e, "gz_count_noalloc: cudaGetSymbolAddress");
        g_region_addr[dev] = p;
    }
    *out = g_region_addr[dev];
    return GZ_OK;
}

}  // namespace

extern "C" gz_status gz_count_noalloc(const gz_plan* p, const gz_graph* g, int use_orientation,
                                      void* stream, uint64_t* out_count) {
    if (!p || !g || !out_count) {
        set_error("gz_count_noalloc: NULL argument");
        return GZ_EINVAL;
    }
    *out_count = 0;
    Query q{};
    gz_status st = prepare_check(p, g, use_orientation, q);
    if (st != GZ_OK) return st;
    if (q.unit_hi <= q.unit_lo) return GZ_OK;
    const uint64_t words = scratch_words_per_warp(p->prog, *g, *q.view);
    if (words * sizeof(int32_t) > GZ_NOALLOC_SCRATCH_BYTES) {
        set_error("gz_count_noalloc: this plan needs %llu bytes of scratch per warp; the static "
                  "maximum is %llu bytes (use gz_count)",
                  (unsigned long long)(words * 4), (unsigned long long)GZ_NOALLOC_SCRATCH_BYTES);
        return GZ_EOVERFLOW;
    }
    void* region = nullptr;
    st = region_address(&region);
    if (st != GZ_OK) return st;
    LaunchCfg cfg;
    cfg.block_warps = 8;
    cfg.chunk = 4;
    return count_one_in_region(q, cfg, (cudaStream_t)stream, region, GZ_NOALLOC_SCRATCH_BYTES, false,
                               out_count);
}
