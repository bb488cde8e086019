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
#include "tb_ctasort.cuh"

namespace tb {

namespace {

constexpr int kRunThreads = 256;
constexpr int kRunTile = 2048;
constexpr int kRunMax = 128;                                 // longest run ordered in place
constexpr int kRunSpan = kRunTile + kRunMax;                 // positions a tile loads
constexpr int kRunChunks = kRunSpan / 32 + 1;                // 32-position start masks (+ one past)
constexpr int kRunPer = kRunTile / kRunThreads;

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
    // sk[x + 2] = keys[s + x] for x in [-1, nw); sk[nw + 2] is a sentinel
    // whose upper bits differ from every key's (keys leave bit 63 clear)
    __shared__ __align__(16) uint64_t sk[kRunSpan + 4];
    __shared__ uint32_t smask[kRunChunks];   // bit l of chunk c: position 32 c + l starts a run
    __shared__ int16_t prv[kRunChunks];      // last chunk <= c holding a start, or -1
    __shared__ int16_t nxt[kRunChunks];      // first chunk >= c holding a start
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * kRunTile;
    const int te = (int)min64(kRunTile, n - s);
    const int nw = (int)min64(kRunSpan, n - s);
    if ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0) {
        const ulonglong2 *src2 = reinterpret_cast<const ulonglong2 *>(keys + s);
        ulonglong2 *dst2 = reinterpret_cast<ulonglong2 *>(sk + 2);
        for (int x = threadIdx.x; x < nw / 2; x += kRunThreads) dst2[x] = src2[x];
        if (threadIdx.x == 0 && (nw & 1)) sk[nw + 1] = keys[s + nw - 1];
    } else {
        for (int x = threadIdx.x; x < nw; x += kRunThreads) sk[x + 2] = keys[s + x];
    }
    if (threadIdx.x == 0) {
        sk[1] = s > 0 ? keys[s - 1] : ~0ull;
        sk[nw + 2] = ~0ull;
    }
    __syncthreads();
    const uint64_t lim = uint64_t(1) << shift0;   // equal upper bits <=> xor below lim
    const uint64_t lowm = lim - 1;
    // start masks; positions past the loaded ones count as starts
    bool multi = false;
    for (int c = warp; c < kRunChunks; c += kRunThreads / 32) {
        const int x = c * 32 + lane;
        const bool st = x >= nw || ((sk[x + 2] ^ sk[x + 1]) >= lim);
        const uint32_t m = __ballot_sync(0xffffffffu, st);
        if (lane == 0) smask[c] = m;
        multi |= (m != 0xffffffffu) && c * 32 <= te;   // includes position te (a run from te - 1)
    }
    // a tile of single-key runs is done
    if (!__syncthreads_or(multi)) {
        if (threadIdx.x == 0) rb.desc[blockIdx.x] = 0;
        return;
    }
    if (warp == 0) {
        // prv / nxt over the chunks, 32 at a time with ballots
        int carry = -1;
        for (int g = 0; g < kRunChunks; g += 32) {
            const int c = g + lane;
            const bool has = c < kRunChunks && smask[c] != 0;
            const uint32_t hm = __ballot_sync(0xffffffffu, has);
            const uint32_t le = hm & (0xffffffffu >> (31 - lane));
            const int p = le ? g + 31 - __clz(le) : carry;
            if (c < kRunChunks) prv[c] = (int16_t)p;
            carry = __shfl_sync(0xffffffffu, p, 31);
        }
        carry = kRunChunks - 1;   // the last chunk lies past the loaded span: all starts
        for (int g = ((kRunChunks - 1) / 32) * 32; g >= 0; g -= 32) {
            const int c = g + lane;
            const bool has = c < kRunChunks && smask[c] != 0;
            const uint32_t hm = __ballot_sync(0xffffffffu, has);
            const uint32_t ge = hm & (0xffffffffu << lane);
            const int q = ge ? g + __ffs(ge) - 1 : carry;
            if (c < kRunChunks) nxt[c] = (int16_t)q;
            carry = __shfl_sync(0xffffffffu, q, 0);
        }
    }
    __syncthreads();
    // a run crossing the tile's end: its members past the end move too
    const bool crossing = te == kRunTile && nw > te && !((smask[te >> 5] >> (te & 31)) & 1u);
    int32_t dst[kRunPer + 1];   // new position - s of the key at position x, or -1
    int32_t val[kRunPer + 1];
    bool desc = false;
#pragma unroll
    for (int i = 0; i <= kRunPer; ++i) {
        dst[i] = -1;
        const int x = i < kRunPer ? (int)threadIdx.x + i * kRunThreads : te + (int)threadIdx.x;
        if (i < kRunPer ? x >= te : (!crossing || x >= nw)) continue;
        const int c = x >> 5, l = x & 31;
        const uint32_t m = smask[c];
        const bool st_here = (m >> l) & 1u;
        const bool st_next = l < 31 ? ((m >> (l + 1)) & 1u) : (smask[c + 1] & 1u);
        if (st_here && st_next) continue;               // a run of one key
        const uint64_t kx = sk[x + 2];
        if (!st_here) desc |= (kx & lowm) < (sk[x + 1] & lowm);
        // the run [a, b) from the start masks
        int a;
        const uint32_t le = m & (0xffffffffu >> (31 - l));
        if (le) {
            a = c * 32 + 31 - __clz(le);
        } else {
            const int pc = c > 0 ? prv[c - 1] : -1;
            if (pc < 0) continue;                       // the run began before this tile
            a = pc * 32 + 31 - __clz(smask[pc]);
        }
        if (a >= te) continue;                          // the run begins after this tile
        const uint32_t gt = l < 31 ? (m & (0xffffffffu << (l + 1))) : 0u;
        int b;
        if (gt) {
            b = c * 32 + __ffs(gt) - 1;
        } else {
            const int nc = nxt[c + 1];
            b = nc * 32 + __ffs(smask[nc]) - 1;
        }
        if (b > nw) b = nw;
        // longer runs (including any that reach the end of the loaded span
        // before the end of the keys) go to the block sort
        if (b - a > kRunMax) {
            if (x == a) rb.queue[atomicAdd(&info->misc_ctr[5], 1u)] = (int32_t)(s + a);
            continue;
        }
        // rank by (low bits, position); the low bits fit 32 bits (shift0 <= 32)
        const uint32_t lp = (uint32_t)(kx & lowm);
        int r = 0;
#pragma unroll 4
        for (int j = a; j < b; ++j) {
            const uint32_t lj = (uint32_t)(sk[j + 2] & lowm);
            r += (lj < lp) || (lj == lp && j < x);
        }
        if (a + r == x) continue;
        dst[i] = a + r;
        val[i] = vals[s + x];
    }
    desc = __syncthreads_or(desc);   // also: every moved value is read before any is overwritten
    if (threadIdx.x == 0) rb.desc[blockIdx.x] = desc ? 1 : 0;
#pragma unroll
    for (int i = 0; i <= kRunPer; ++i) {
        if (dst[i] < 0) continue;
        const int x = i < kRunPer ? (int)threadIdx.x + i * kRunThreads : te + (int)threadIdx.x;
        keys[s + dst[i]] = sk[x + 2];
        vals[s + dst[i]] = val[i];
    }
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
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(long_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(CtaSortShared));
        attr = true;
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
