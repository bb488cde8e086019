// tb_runs.cu -- the last step of the key sort (Sec. 2.3 step 2).
//
// The global radix passes order the (key, index) pairs stably by the upper
// bits of the key, key >> shift0.  What is left is to order every run of equal
// upper bits by the low shift0 bits, stably.  With 40 upper bits the runs of
// the tree workloads are short (most have one element; in a 2^27-particle
// clustered set about one in a million is longer than 128), so each run is
// finished where it lies:
//   run_sort_kernel  : per tile of 2048 positions (plus 128 beyond it), one
//                      bit per position marks where a run starts (a warp
//                      ballot per 32 positions); every run that starts in the
//                      tile and holds at most 128 keys is ordered in place,
//                      each member going to its rank by
//                      (low bits, position); longer runs are queued, and each
//                      tile notes whether any of its keys is smaller than its
//                      predecessor in the same run (a descent);
//   long_run_kernel  : each queued run that contains a descent is sorted by
//                      its low bits by one block with the block-local LSD sort
//                      (3 passes of 8 bits); runs without one (for instance
//                      identical keys) are already in order.
// The outcome equals a stable sort of the whole keys: equal upper bits stay
// in index order from the passes, and the run step orders them by the rest.
#include "tb_runs.cuh"

namespace tb {

namespace {

constexpr int kRunThreads = 256;

// Queue of long runs and the per-tile descent flags, laid out in one buffer.
struct RunBuffers {
    int32_t *queue;      // [n / kRunMax + 2] start positions of long runs
    uint8_t *desc;       // [n / kRunTile + 1] tile holds a descent inside a run
};
__host__ __device__ inline int64_t run_queue_cap(int64_t n) { return n / kRunMax + 2; }
__host__ __device__ inline RunBuffers run_buffers(int32_t *base, int64_t n) {
    return {base, reinterpret_cast<uint8_t *>(base + run_queue_cap(n))};
}

__global__ void __launch_bounds__(kRunThreads)
    run_sort_kernel(uint64_t *__restrict__ keys, int32_t *__restrict__ vals, int64_t n, int shift0,
                    RunBuffers rb, DevInfo *info) {
    __shared__ RunSmem sm;
    const int64_t s = (int64_t)blockIdx.x * kRunTile;
    const bool desc = run_tile<kRunThreads>(keys, vals, 0, s, n, shift0, sm, [&](int64_t a) {
        rb.queue[atomicAdd(&info->misc_ctr[5], 1u)] = (int32_t)a;
    });
    if (threadIdx.x == 0) rb.desc[blockIdx.x] = desc ? 1 : 0;
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    long_run_kernel(uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v, int64_t n,
                    int shift0, RunBuffers rb, DevInfo *info) {
    extern __shared__ __align__(16) unsigned char raw[];
    CtaSortShared &sm = *reinterpret_cast<CtaSortShared *>(raw);
    __shared__ uint32_t s_q;
    __shared__ unsigned long long s_end;
    __shared__ int s_desc;
    const uint32_t nq = *(volatile uint32_t *)&info->misc_ctr[5];
    const int passes = (shift0 + kCtaRadixBits - 1) / kCtaRadixBits;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(&info->misc_ctr[6], 1u);
        __syncthreads();
        const uint32_t q = s_q;
        __syncthreads();
        if (q >= nq) return;
        const int64_t a = rb.queue[q];
        const uint64_t tp = keys[a] >> shift0;
        // the run's end: the first later position with other upper bits;
        // the first 4096 positions are scanned by the block, then binary search
        if (threadIdx.x == 0) { s_end = (unsigned long long)n; s_desc = 0; }
        __syncthreads();
        int64_t base = a + 1;
        for (int it = 0; it < 4 && base < n; ++it, base += kCtaThreads) {
            const int64_t p = base + threadIdx.x;
            if (p < n && (keys[p] >> shift0) != tp) atomicMin(&s_end, (unsigned long long)p);
            __syncthreads();
            const bool done = s_end < (unsigned long long)n;
            __syncthreads();
            if (done) break;
        }
        if (threadIdx.x == 0 && s_end == (unsigned long long)n && base < n) {
            int64_t lo = base, hi = n;                  // first position with top > tp
            while (lo < hi) {
                const int64_t m = (lo + hi) >> 1;
                if ((keys[m] >> shift0) <= tp) lo = m + 1; else hi = m;
            }
            s_end = (unsigned long long)lo;
        }
        __syncthreads();
        const int64_t len = (int64_t)s_end - a;
        // only a run with a descent needs sorting: look at the tile flags
        const int64_t t0 = (a + 1) / kRunTile, t1 = (a + len - 1) / kRunTile;
        for (int64_t t = t0 + threadIdx.x; t <= t1; t += kCtaThreads)
            if (rb.desc[t]) s_desc = 1;
        __syncthreads();
        if (s_desc) {
            cta_histograms(keys, a, len, 0, passes, sm);
            const int np = cta_lsd_sort(keys, vals, alt_k, alt_v, a, len, 0, passes, false, sm);
            if (np & 1)
                for (int64_t p = a + threadIdx.x; p < a + len; p += kCtaThreads) {
                    keys[p] = alt_k[p];
                    vals[p] = alt_v[p];
                }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_runs(uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v, int64_t n,
                        int shift0, int32_t *long_runs, Workspace &ws, cudaStream_t s) {
    const RunBuffers rb = run_buffers(long_runs, n);
    if (shift0 <= 0 || n <= 1) return cudaSuccess;
    if (shift0 > 32) return cudaErrorInvalidValue;   // the run step ranks the low bits as 32-bit words
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        cudaFuncSetAttribute(long_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(CtaSortShared));
    }
    const int64_t tiles = (n + kRunTile - 1) / kRunTile;
    run_sort_kernel<<<(unsigned)tiles, kRunThreads, 0, s>>>(keys, vals, n, shift0, rb, ws.info);
    ++g_launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long_run_kernel<<<152, kCtaThreads, sizeof(CtaSortShared), s>>>(keys, vals, alt_k, alt_v, n, shift0,
                                                                   rb, ws.info);
    ++g_launches;
    return cudaGetLastError();
}

// int32 words for the queue and the tile flags of n keys
int64_t long_run_capacity(int64_t n) {
    return run_queue_cap(n) + (n / kRunTile + 1 + 3) / 4 + 1;
}

}  // namespace tb
