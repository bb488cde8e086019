// tb_runs.cu -- the last step of the key sort (Sec. 2.3 step 2).
//
// The global radix passes order the (key, index) pairs stably by the upper
// bits of the key, key >> shift0.  What is left is to order every run of equal
// upper bits by the low shift0 bits, stably.  With 40 upper bits the runs of
// the tree workloads are short (most have one element, few more than a few
// dozen), so each run is finished where it lies:
//   run_sort_kernel  : per tile of 2048 positions (plus a look-ahead window of
//                      1024), every run that starts in the tile is found by
//                      binary search for its ends, and each member's place is
//                      its rank by (low bits, position) within the run; runs
//                      that outgrow the window are queued;
//   long_run_kernel  : each queued run is sorted by its low bits by one block
//                      with the block-local LSD sort (3 passes of 8 bits).
// The outcome equals a stable sort of the whole keys: equal upper bits stay
// in index order from the passes, and the run step orders them by the rest.
#include "tb_ctasort.cuh"

namespace tb {

namespace {

constexpr int kRunThreads = 256;
constexpr int kRunTile = 2048;
constexpr int kRunWin = 1024;
constexpr int kRunPer = (kRunTile + kRunWin + kRunThreads - 1) / kRunThreads;

__global__ void __launch_bounds__(kRunThreads)
    run_sort_kernel(uint64_t *__restrict__ keys, int32_t *__restrict__ vals, int64_t n, int shift0,
                    int32_t *__restrict__ long_runs, DevInfo *info) {
    __shared__ uint64_t sk[kRunTile + kRunWin + 1];
    const int64_t s = (int64_t)blockIdx.x * kRunTile;
    const int64_t e = min64(n, s + kRunTile), we = min64(n, e + kRunWin);
    const int64_t lo = s > 0 ? s - 1 : 0;   // shared index x holds position lo + x
    const int nw = (int)(we - lo);
    for (int x = threadIdx.x; x < nw; x += blockDim.x) sk[x] = keys[lo + x];
    __syncthreads();
    const uint64_t lowmask = (uint64_t(1) << shift0) - 1;
    auto top = [&](int64_t p) { return sk[p - lo] >> shift0; };
    int32_t dst[kRunPer];   // new position - s of the key at s + tid + i * threads, or -1
    int32_t val[kRunPer];
#pragma unroll
    for (int i = 0; i < kRunPer; ++i) {
        dst[i] = -1;
        const int64_t p = s + threadIdx.x + (int64_t)i * kRunThreads;
        if (p >= we) continue;
        const uint64_t tp = top(p);
        // most runs are single keys: no equal neighbour
        if ((p == 0 || top(p - 1) != tp) && (p + 1 >= we || top(p + 1) != tp)) continue;
        if (p >= e && top(e - 1) != tp) continue;             // run begins in a later tile
        // equal upper bits are contiguous, so the run's ends are found by
        // binary search in the window
        if (s > 0 && top(s - 1) == tp) continue;             // run began in an earlier tile
        int64_t a, b;
        {
            int64_t l = s, h = p;                             // first position with top == tp
            while (l < h) { const int64_t m = (l + h) >> 1; if (top(m) < tp) l = m + 1; else h = m; }
            a = l;
        }
        {
            int64_t l = p + 1, h = we;                        // first position with top > tp
            while (l < h) { const int64_t m = (l + h) >> 1; if (top(m) <= tp) l = m + 1; else h = m; }
            b = l;
        }
        if (b == we && we < n) {                              // may run past the window
            if (p == a) long_runs[atomicAdd(&info->misc_ctr[5], 1u)] = (int32_t)a;
            continue;
        }
        const uint64_t lp = sk[p - lo] & lowmask;
        int64_t r = 0;
        for (int64_t j = a; j < b; ++j) {
            const uint64_t lj = sk[j - lo] & lowmask;
            r += (lj < lp) || (lj == lp && j < p);
        }
        dst[i] = (int32_t)(a + r - s);
        val[i] = vals[p];
    }
    __syncthreads();   // every moved value is read before any is overwritten
#pragma unroll
    for (int i = 0; i < kRunPer; ++i) {
        if (dst[i] < 0) continue;
        const int64_t p = s + threadIdx.x + (int64_t)i * kRunThreads;
        keys[s + dst[i]] = sk[p - lo];
        vals[s + dst[i]] = val[i];
    }
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    long_run_kernel(uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v, int64_t n,
                    int shift0, const int32_t *long_runs, DevInfo *info) {
    extern __shared__ __align__(16) unsigned char raw[];
    CtaSortShared &sm = *reinterpret_cast<CtaSortShared *>(raw);
    __shared__ uint32_t s_q;
    __shared__ int64_t s_end;
    const uint32_t nq = *(volatile uint32_t *)&info->misc_ctr[5];
    const int passes = (shift0 + kCtaRadixBits - 1) / kCtaRadixBits;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(&info->misc_ctr[6], 1u);
        __syncthreads();
        const uint32_t q = s_q;
        __syncthreads();
        if (q >= nq) return;
        const int64_t a = long_runs[q];
        const uint64_t tp = keys[a] >> shift0;
        // the run's end: the first position after a whose upper bits differ
        if (threadIdx.x == 0) s_end = n;
        __syncthreads();
        for (int64_t base = a + 1; base < n; base += blockDim.x) {
            const int64_t p = base + threadIdx.x;
            if (p < n && (keys[p] >> shift0) != tp) atomicMin((unsigned long long *)&s_end, (unsigned long long)p);
            __syncthreads();
            const bool done = s_end < n;
            __syncthreads();
            if (done) break;
        }
        const int64_t len = s_end - a;
        cta_histograms(keys, a, len, 0, passes, sm);
        const int np = cta_lsd_sort(keys, vals, alt_k, alt_v, a, len, 0, passes, false, sm);
        if (np & 1)
            for (int64_t p = a + threadIdx.x; p < a + len; p += blockDim.x) {
                keys[p] = alt_k[p];
                vals[p] = alt_v[p];
            }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_runs(uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v, int64_t n,
                        int shift0, int32_t *long_runs, Workspace &ws, cudaStream_t s) {
    if (shift0 <= 0 || n <= 1) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(long_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(CtaSortShared));
        attr = true;
    }
    const int64_t tiles = (n + kRunTile - 1) / kRunTile;
    run_sort_kernel<<<(unsigned)tiles, kRunThreads, 0, s>>>(keys, vals, n, shift0, long_runs, ws.info);
    ++g_launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long_run_kernel<<<152, kCtaThreads, sizeof(CtaSortShared), s>>>(keys, vals, alt_k, alt_v, n, shift0,
                                                                   long_runs, ws.info);
    ++g_launches;
    return cudaGetLastError();
}

int64_t long_run_capacity(int64_t n) { return n / kRunWin + 2; }

}  // namespace tb
