// tb_noalloc.cu -- the root cell, keys and radix sort of tb_build without any
// device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns the device's memory pool (a caching allocator that has
// reserved all free memory, so a fresh cudaMalloc fails or fragments it),
// code inside a latency-critical loop where cudaMalloc's implicit device
// synchronisation is not acceptable, or code that must not grow its
// footprint after start-up.  For them this file keeps the sort's scratch --
// the digit histograms, the look-back array, the second key / index buffer,
// the (x, y, z, m) records the key kernel writes and the queue of long sort
// runs -- in one file-scope device array of fixed size (about 15 MB);
// particle counts above TB_NOALLOC_MAX_N are refused.
//
// The array belongs to this file's CUDA module.  CUDA loads modules lazily
// by default, so a device reserves the array when the module is first used
// there: at the first call on that device, whose address lookup loads it.
// The kernels' modules load the same way at the first call that sorts
// (n >= 2).  Those first calls can therefore fail when the device's memory
// is already taken; a caller makes one call with n >= 2 at start-up, and
// from then on the device holds the array and the kernels until the process
// exits and no call allocates.
//
// The array is shared by every call on a device and keeps the last call's
// contents: each call clears the parts that must start at zero (the build
// record with its counters, and the look-back words of the tiles it sorts).
// Calls whose work overlaps on the GPU race on it, so callers must order
// them (one stream, or events between streams).
#include <cstring>
#include <mutex>

#include "tb_internal.h"

namespace tb {

namespace {

constexpr int64_t kNoAllocMaxN = TB_NOALLOC_MAX_N;
constexpr int kNoAllocRadixBits = 8;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// layout of the scratch array
constexpr size_t kOffInfo = 0;
constexpr size_t kOffHist = align256(kOffInfo + sizeof(DevInfo));
constexpr size_t kOffPart = align256(kOffHist + sizeof(uint32_t) * 16 * 2048);
constexpr size_t kOffLook = align256(kOffPart + sizeof(float) * 8 * 152 * 4);
// look-back: one 64-bit word per tile and digit; the smallest compiled tile
// of 8-bit digits holds 2048 keys
constexpr size_t kLookWords = ((kNoAllocMaxN + 2047) / 2048) * (size_t(1) << kNoAllocRadixBits);
constexpr size_t kOffKeys = align256(kOffLook + sizeof(uint64_t) * kLookWords);
constexpr size_t kOffPerm = align256(kOffKeys + sizeof(uint64_t) * kNoAllocMaxN);
constexpr size_t kOffXm = align256(kOffPerm + sizeof(int32_t) * kNoAllocMaxN);
constexpr size_t kOffRuns = align256(kOffXm + 16 * size_t(kNoAllocMaxN));
// queue of long sort runs (over 128 keys) and one flag byte per 2048 keys
constexpr size_t kRunsCap = kNoAllocMaxN / 128 + 2 + (kNoAllocMaxN / 2048 + 4) / 4 + 1;
constexpr size_t kScratchBytes = align256(kOffRuns + sizeof(int32_t) * kRunsCap);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of the array, looked up once per device with that device
// current (the host-side name is only a stand-in and must not be passed to
// a kernel)
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

tb_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return TB_OK;
    return e == cudaErrorMemoryAllocation ? TB_ENOMEM : TB_ECUDA;
}

}  // namespace

}  // namespace tb

using namespace tb;

extern "C" tb_status tb_keys_sorted_noalloc(const float *d_pos, int64_t n, uint64_t *d_pkey,
                                            int32_t *d_perm, double *h_root, tb_stream stream) {
    if (n < 0 || n > kNoAllocMaxN) return TB_EINVAL;
    if (n > 0 && (!d_pos || !d_pkey || !d_perm)) return TB_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_pos) & 3u) || (reinterpret_cast<uintptr_t>(d_pkey) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_perm) & 3u))
        return TB_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return status_of(e);

    Workspace ws;   // host-side view: device pointers into the scratch array
    ws.info = reinterpret_cast<DevInfo *>(base + kOffInfo);
    ws.hist = reinterpret_cast<uint32_t *>(base + kOffHist);
    ws.bbox_part = reinterpret_cast<float *>(base + kOffPart);
    ws.lookback = reinterpret_cast<uint64_t *>(base + kOffLook);
    ws.keys_alt = reinterpret_cast<uint64_t *>(base + kOffKeys);
    ws.perm_alt = reinterpret_cast<int32_t *>(base + kOffPerm);
    ws.xm = reinterpret_cast<float4 *>(base + kOffXm);
    ws.long_runs = reinterpret_cast<int32_t *>(base + kOffRuns);
    if (long_run_capacity(kNoAllocMaxN) > (int64_t)kRunsCap) return TB_ECUDA;

    // what must start at zero: the build record and its counters, and the
    // look-back words of this call's tiles.  The record is cleared, so every
    // call runs with the same look-back epoch and the words a larger earlier
    // call left would read as published; a tile only reads the words of
    // tiles before it, so clearing this call's tiles is enough.
    const SortCfg cfg = default_sort_cfg(kNoAllocRadixBits);
    const int64_t look_words = ((n + cfg.tile() - 1) / cfg.tile()) << cfg.radix_bits;
    if (look_words > (int64_t)kLookWords) return TB_ECUDA;
    if ((e = cudaMemsetAsync(ws.info, 0, sizeof(DevInfo), s)) != cudaSuccess) return status_of(e);
    if (look_words > 0 &&
        (e = cudaMemsetAsync(ws.lookback, 0, sizeof(uint64_t) * look_words, s)) != cudaSuccess)
        return status_of(e);
    if (n == 0) {
        if (h_root) {
            h_root[0] = h_root[1] = h_root[2] = 0.0;
            h_root[3] = 1.0;
        }
        return status_of(cudaStreamSynchronize(s));
    }
    const int passes = sort_plan(cfg).passes;
    if ((e = launch_root(d_pos, n, ws, passes << cfg.radix_bits, s)) != cudaSuccess)
        return status_of(e);
    uint64_t *ka = (passes & 1) ? ws.keys_alt : d_pkey;
    uint64_t *kb = (passes & 1) ? d_pkey : ws.keys_alt;
    int32_t *pa = (passes & 1) ? ws.perm_alt : d_perm;
    int32_t *pb = (passes & 1) ? d_perm : ws.perm_alt;
    if ((e = launch_keys(d_pos, nullptr, n, ka, ws, cfg, TB_KEYS_MORTON, s)) != cudaSuccess)
        return status_of(e);
    uint64_t *kout = nullptr;
    int32_t *pout = nullptr;
    if ((e = launch_sort(ka, kb, pa, pb, n, ws, cfg, kout, pout, s)) != cudaSuccess)
        return status_of(e);
    if (kout != d_pkey || pout != d_perm) return TB_ECUDA;

    // the call ends by reading the device status (and the root cube)
    DevInfo h;
    if ((e = cudaMemcpyAsync(&h, ws.info, sizeof(DevInfo), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return status_of(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return status_of(e);
    if (h_root) {
        for (int a = 0; a < 3; ++a) h_root[a] = (double)h.lo[a];
        h_root[3] = h.side;
    }
    if (h.status & kErrNonFinite) return TB_ENONFINITE;
    if (h.status & kErrTimeout) return TB_ETIMEOUT;
    return TB_OK;
}
