// tb_sort.cu -- stable LSD radix sort of (key, original index) pairs
// (Sec. 2.3 step 2).
//
// The paper sorts on the CPU with parallel sorting by regular sampling; on
// the GPU the keys are sorted by ceil(63 / b) stable least-significant-digit
// passes of b bits (bit 63 is always 1).  Each pass is one "onesweep" launch
// (Adinets & Merrill 2022):
//   - every block takes the next tile id from an atomic counter, so a block
//     only ever waits on tiles that blocks already running own;
//   - it ranks its tile's digits stably, warp by warp (ballot peer masks,
//     shared-memory counters), in tile order;
//   - it publishes its per-digit counts to a look-back array and walks back
//     over earlier tiles until it meets an inclusive prefix (decoupled
//     look-back); every wait is bounded and reports a timeout instead of
//     hanging;
//   - it orders the tile by digit in shared memory and writes keys and
//     indices out as runs of consecutive addresses.
// The passes order the keys by their upper ceil(40 / b) * b bits only; the runs
// of equal upper bits they leave (short in practice) are ordered by the low
// bits afterwards (tb_runs.cu).  Digit offsets of every pass come from the
// histograms taken while the keys were made.  Look-back words carry an epoch (build counter + pass) so that
// the array is never cleared between passes or builds.
#include "tb_device.cuh"

namespace tb {

namespace {

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr int kLookWindow = 4;
constexpr uint64_t kFlagIncl = 2ull << 62;

template <int RADIX_BITS, int THREADS, int ITEMS>
struct SortSmem {
    static constexpr int RADIX = 1 << RADIX_BITS;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int TILE = THREADS * ITEMS;
    uint64_t keys[TILE];
    int32_t vals[TILE];
    uint32_t warp_hist[WARPS][RADIX + 1];
    uint32_t tile_off[RADIX + 1];
    uint32_t glob_base[RADIX];
    uint32_t scan_tmp[WARPS];
    uint32_t tile;
};

template <int RADIX_BITS, int THREADS, int ITEMS, bool FIRST>
__global__ void __launch_bounds__(THREADS, (THREADS <= 256 ? (ITEMS <= 8 ? 4 : 2) : (ITEMS <= 8 ? 2 : 1)))
    onesweep_kernel(const uint64_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in,
                    uint64_t *__restrict__ keys_out, int32_t *__restrict__ vals_out, int64_t n,
                    int pass, int shift0, const uint32_t *__restrict__ digit_off, uint64_t *lookback,
                    DevInfo *info, int64_t spin_limit) {
    using S = SortSmem<RADIX_BITS, THREADS, ITEMS>;
    constexpr int RADIX = S::RADIX;
    constexpr int WARPS = S::WARPS;
    constexpr int TILE = S::TILE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int shift = shift0 + pass * RADIX_BITS;

    if (threadIdx.x == 0) sm.tile = atomicAdd(&info->sort_tile_ctr[pass], 1u);
    for (int i = threadIdx.x; i < WARPS * (RADIX + 1); i += THREADS)
        (&sm.warp_hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = sm.tile;
    const int64_t tile_base = (int64_t)tile * TILE;
    const int valid = (int)min64(TILE, n - tile_base);

    // load (warp-striped: warp w owns 32*ITEMS consecutive elements)
    uint64_t key[ITEMS];
    int32_t val[ITEMS];
    uint32_t rank[ITEMS];
    const int wbase = warp * 32 * ITEMS;
    const bool full = valid == TILE;
    if (full) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int e = wbase + i * 32 + lane;
            key[i] = keys_in[tile_base + e];
            val[i] = FIRST ? (int32_t)(tile_base + e) : vals_in[tile_base + e];
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int e = wbase + i * 32 + lane;
            if (e < valid) {
                key[i] = keys_in[tile_base + e];
                val[i] = FIRST ? (int32_t)(tile_base + e) : vals_in[tile_base + e];
            } else {
                key[i] = 0;
                val[i] = 0;
            }
        }
    }

    // stable rank within the warp, in element order.  The lanes holding the
    // same digit are found with one ballot per digit bit (plus one for the
    // tail sentinel); the lowest of them adds the group's size to the warp's
    // digit counter with a shared-memory atomic, whose returned old value is
    // collected only after every item has been issued, so no item waits on
    // the one before.  A warp's atomics on one counter are applied in issue
    // order, which keeps equal digits in element order.
    const unsigned lt = lanemask_lt();
    uint32_t old_cnt[ITEMS], lead_rank[ITEMS];
    // a full tile needs no sentinel bit: RADIX_BITS ballots per item
    const int nbits = full ? RADIX_BITS : RADIX_BITS + 1;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int e = wbase + i * 32 + lane;
        const uint32_t d = (full || e < valid) ? (uint32_t)((key[i] >> shift) & (RADIX - 1))
                                               : (uint32_t)RADIX;
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b <= RADIX_BITS; ++b) {
            if (b == RADIX_BITS && nbits == RADIX_BITS) break;
            const bool bit = (d >> b) & 1u;
            const unsigned v = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? v : ~v;
        }
        const int leader = __ffs(peers) - 1;
        old_cnt[i] = (lane == leader) ? atomicAdd(&sm.warp_hist[warp][d], (uint32_t)__popc(peers)) : 0u;
        lead_rank[i] = (uint32_t)leader | ((uint32_t)__popc(peers & lt) << 8);
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        rank[i] = __shfl_sync(0xffffffffu, old_cnt[i], lead_rank[i] & 31u) + (lead_rank[i] >> 8);
    __syncthreads();

    // per-digit: offsets of each warp within the digit, tile digit counts
    uint32_t my_count[(RADIX + THREADS - 1) / THREADS];
#pragma unroll
    for (int r = 0; r < (RADIX + THREADS - 1) / THREADS; ++r) {
        int d = r * THREADS + threadIdx.x;
        uint32_t acc = 0;
        if (d < RADIX) {
            for (int w = 0; w < WARPS; ++w) {
                uint32_t c = sm.warp_hist[w][d];
                sm.warp_hist[w][d] = acc;
                acc += c;
            }
        }
        my_count[r] = acc;
    }
    // exclusive scan of the counts over digits
    if constexpr (RADIX <= THREADS) {
        // one digit per thread: a warp scan and one across the warps
        const uint32_t c = (threadIdx.x < RADIX) ? my_count[0] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) sm.scan_tmp[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += sm.scan_tmp[w];
        if (threadIdx.x < RADIX) sm.tile_off[threadIdx.x] = wpre + x - c;
        if (threadIdx.x == 0) sm.tile_off[RADIX] = (uint32_t)valid;
    } else {
        // each thread holds a contiguous group of digits
        constexpr int PER = (RADIX + THREADS - 1) / THREADS;
        // regroup: thread t owns digits [t*PER, t*PER+PER) for the scan
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            int d = r * THREADS + threadIdx.x;
            if (d < RADIX) sm.tile_off[d] = my_count[r];
        }
        __syncthreads();
        uint32_t loc[PER];
        uint32_t sum = 0;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            int d = threadIdx.x * PER + r;
            loc[r] = (d < RADIX) ? sm.tile_off[d] : 0u;
            sum += loc[r];
        }
        uint32_t x = sum;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) sm.scan_tmp[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += sm.scan_tmp[w];
        uint32_t run = wpre + x - sum;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            int d = threadIdx.x * PER + r;
            if (d < RADIX) sm.tile_off[d] = run;
            run += loc[r];
        }
        if (threadIdx.x == 0) sm.tile_off[RADIX] = (uint32_t)valid;
    }
    __syncthreads();

    // publish this tile's digit counts (aggregate), then order the tile by
    // digit in shared memory while the predecessors finish theirs
    const uint64_t epoch = (uint64_t)((info->epoch + (uint32_t)pass) & 0x3fffffffu);
#pragma unroll
    for (int r = 0; r < (RADIX + THREADS - 1) / THREADS; ++r) {
        int d = r * THREADS + threadIdx.x;
        if (d >= RADIX) continue;
        uint64_t *slot = lookback + (int64_t)tile * RADIX + d;
        st_relaxed_u64(slot, (tile == 0 ? kFlagIncl : kFlagAgg) | (epoch << 32) | my_count[r]);
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int e = wbase + i * 32 + lane;
        if (e < valid) {
            uint32_t d = (uint32_t)((key[i] >> shift) & (RADIX - 1));
            uint32_t p = sm.tile_off[d] + sm.warp_hist[warp][d] + rank[i];
            sm.keys[p] = key[i];
            sm.vals[p] = val[i];
        }
    }

    // decoupled look-back, one digit per thread, kLookWindow predecessors
    // read per round so that one memory latency covers several tiles
#pragma unroll
    for (int r = 0; r < (RADIX + THREADS - 1) / THREADS; ++r) {
        int d = r * THREADS + threadIdx.x;
        if (d >= RADIX) continue;
        uint32_t excl = 0;
        if (tile > 0) {
            int64_t pred = (int64_t)tile - 1;
            int64_t iter = 0;
            for (;;) {
                uint64_t w[kLookWindow];
#pragma unroll
                for (int j = 0; j < kLookWindow; ++j)
                    w[j] = (pred - j >= 0) ? ld_relaxed_u64(lookback + (pred - j) * RADIX + d) : 0ull;
                int adv = 0;
                bool found = false, blocked = false;
#pragma unroll
                for (int j = 0; j < kLookWindow; ++j) {
                    if (found || blocked) continue;
                    if (pred - j < 0 || ((w[j] >> 32) & 0x3fffffffu) != epoch || (w[j] >> 62) == 0) {
                        blocked = true;
                        continue;
                    }
                    excl += (uint32_t)w[j];
                    adv = j + 1;
                    if ((w[j] >> 62) == 2) found = true;
                }
                if (found) break;
                pred -= adv;
                if (adv == 0 && !poll_backoff(iter, spin_limit)) {
                    flag_error(&info->status, kErrTimeout);
                    break;
                }
            }
            st_relaxed_u64(lookback + (int64_t)tile * RADIX + d,
                           kFlagIncl | (epoch << 32) | (excl + my_count[r]));
        }
        sm.glob_base[d] = digit_off[d] + excl - sm.tile_off[d];
    }
    __syncthreads();

    // write runs of equal digits to consecutive global addresses
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int j = i * THREADS + threadIdx.x;
        if (j < valid) {
            uint64_t k = sm.keys[j];
            uint32_t d = (uint32_t)((k >> shift) & (RADIX - 1));
            uint64_t dst = (uint64_t)sm.glob_base[d] + (uint32_t)j;
            dst &= 0xffffffffull;
            if ((int64_t)dst < n) {
                keys_out[dst] = k;
                vals_out[dst] = sm.vals[j];
            } else {
                flag_error(&info->status, kErrTimeout);
            }
        }
    }
}

template <int B, int T, int I>
cudaError_t run_passes(uint64_t *ka, uint64_t *kb, int32_t *pa, int32_t *pb, int64_t n,
                       Workspace &ws, const SortPlan &plan, uint64_t *&kout, int32_t *&pout,
                       cudaStream_t s) {
    using S = SortSmem<B, T, I>;
    const size_t smem = sizeof(S);
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        cudaFuncSetAttribute(onesweep_kernel<B, T, I, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(onesweep_kernel<B, T, I, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(onesweep_kernel<B, T, I, true>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(onesweep_kernel<B, T, I, false>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    const int64_t tiles = (n + S::TILE - 1) / S::TILE;
    // the unsorted keys are in `ka`; passes alternate ka -> kb -> ka ...
    uint64_t *src = ka, *dst = kb;
    int32_t *vsrc = pa, *vdst = pb;
    const int64_t spin = g_wait_limit;
    for (int p = 0; p < plan.passes; ++p) {
        if (p == 0)
            onesweep_kernel<B, T, I, true><<<(unsigned)tiles, T, smem, s>>>(
                src, nullptr, dst, vdst, n, p, plan.shift0, ws.hist + p * (1 << B), ws.lookback,
                ws.info, spin);
        else
            onesweep_kernel<B, T, I, false><<<(unsigned)tiles, T, smem, s>>>(
                src, vsrc, dst, vdst, n, p, plan.shift0, ws.hist + p * (1 << B), ws.lookback,
                ws.info, spin);
        ++g_launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        mark(ws, "sort_pass", s);
        uint64_t *t = src; src = dst; dst = t;
        int32_t *u = vsrc; vsrc = vdst; vdst = u;
    }
    kout = src;
    pout = vsrc;
    // finish the runs of equal upper bits; the other buffers are free scratch
    cudaError_t e = launch_runs(src, vsrc, dst, vdst, n, plan.shift0, ws.long_runs, ws, s);
    if (e != cudaSuccess) return e;
    if (plan.shift0 > 0) mark(ws, "sort_runs", s);
    return cudaSuccess;
}

}  // namespace

// Polls after which a look-back wait gives up (about 17 s with the back-off);
// tb_set_wait_limit lowers it to exercise the timeout path.
int64_t g_wait_limit = kDefaultWaitLimit;

// Compiled variants: digit bits, threads per tile, keys per thread.
static const SortCfg kVariants[] = {
    {8, 256, 16}, {8, 512, 16}, {8, 512, 12}, {8, 512, 8}, {8, 256, 8},
    {9, 256, 16}, {9, 512, 16}, {9, 512, 8}, {10, 256, 16}, {10, 512, 8}, {11, 256, 16},
};
static const int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

const SortCfg *sort_variant(int i) { return (i >= 0 && i < kNumVariants) ? &kVariants[i] : nullptr; }

SortCfg default_sort_cfg(int radix_bits) {
    for (int i = 0; i < kNumVariants; ++i)
        if (kVariants[i].radix_bits == radix_bits) return kVariants[i];
    return kVariants[0];
}

bool sort_cfg_valid(const SortCfg &c) {
    for (int i = 0; i < kNumVariants; ++i)
        if (kVariants[i].radix_bits == c.radix_bits && kVariants[i].threads == c.threads &&
            kVariants[i].items == c.items)
            return true;
    return false;
}

int64_t sort_tiles(const SortCfg &c, int64_t n) { return (n + c.tile() - 1) / c.tile(); }

SortPlan sort_plan(const SortCfg &c) {
    // global passes cover the upper ceil(40 / b) * b key bits; the runs of
    // equal upper bits are finished locally
    const int b = c.radix_bits;
    const int passes = (40 + b - 1) / b;
    return {passes, 63 - passes * b};
}

cudaError_t launch_sort(uint64_t *ka, uint64_t *kb, int32_t *pa, int32_t *pb, int64_t n,
                        Workspace &ws, const SortCfg &cfg, uint64_t *&kout, int32_t *&pout,
                        cudaStream_t s) {
    const SortPlan plan = sort_plan(cfg);
#define TB_SORT_CASE(B, T, I)                                             \
    if (cfg.radix_bits == B && cfg.threads == T && cfg.items == I)        \
        return run_passes<B, T, I>(ka, kb, pa, pb, n, ws, plan, kout, pout, s);
    TB_SORT_CASE(8, 256, 16)
    TB_SORT_CASE(8, 512, 16)
    TB_SORT_CASE(8, 512, 12)
    TB_SORT_CASE(8, 512, 8)
    TB_SORT_CASE(8, 256, 8)
    TB_SORT_CASE(9, 256, 16)
    TB_SORT_CASE(9, 512, 16)
    TB_SORT_CASE(9, 512, 8)
    TB_SORT_CASE(10, 256, 16)
    TB_SORT_CASE(10, 512, 8)
    TB_SORT_CASE(11, 256, 16)
#undef TB_SORT_CASE
    return cudaErrorInvalidValue;
}

}  // namespace tb
