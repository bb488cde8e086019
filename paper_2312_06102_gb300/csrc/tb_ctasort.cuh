// tb_ctasort.cuh -- a stable LSD radix sort of one contiguous range of
// (64-bit key, 32-bit value) pairs by a single block of T threads (T = 512 or
// 1024): every pass takes the range's tiles in order with running per-digit
// offsets, so it needs no coordination with other blocks.  Used for the sets
// of a batched build and for the rare long runs left by the single-tree sort.
#pragma once

#include "tb_device.cuh"

namespace tb {
namespace {

constexpr int kCtaThreads = 1024;                // block of the long-run sort
constexpr int kCtaRadixBits = 8;
constexpr int kCtaRadix = 1 << kCtaRadixBits;
constexpr int kCtaMaxPasses = 8;
constexpr int kCtaItems = 4;                     // keys per thread of a tile

template <int T>
struct CtaSortSharedT {
    static constexpr int WARPS = T / 32;
    static constexpr int TILE = T * kCtaItems;
    uint64_t keys[TILE];
    int32_t vals[TILE];
    uint32_t warp_hist[WARPS][kCtaRadix + 1];
    uint32_t hist[kCtaMaxPasses][kCtaRadix];
    uint32_t run[kCtaRadix];
    uint32_t tile_off[kCtaRadix + 1];
    uint32_t cnt[kCtaRadix];
    uint32_t carry[kCtaRadix / 32];
};
using CtaSortShared = CtaSortSharedT<kCtaThreads>;

// Exclusive prefix of the kCtaRadix counts in[] into out[] (out may alias
// in), with the total in out[kCtaRadix] when out_total is set: eight warps,
// 32 digits each, one shuffle scan per warp and a carry across warps.  All
// threads of the block call it; it ends with a barrier.
template <int T>
__device__ __forceinline__ void cta_digit_scan(const uint32_t *in, uint32_t *out, bool out_total,
                                               uint32_t *s_carry /* [kCtaRadix / 32] */) {
    static_assert(kCtaRadix == 256 && T >= kCtaRadix, "digit scan shape");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = 0, x = 0;
    if (threadIdx.x < kCtaRadix) {
        v = in[threadIdx.x];
        x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_carry[warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < kCtaRadix) {
        uint32_t c = 0;
        for (int w = 0; w < warp; ++w) c += s_carry[w];
        out[threadIdx.x] = c + x - v;
        if (out_total && threadIdx.x == kCtaRadix - 1) out[kCtaRadix] = c + x;
    }
    __syncthreads();
}

// Digit counts of every pass over [o, o + ns) into sm.hist.
template <int T>
__device__ void cta_histograms(const uint64_t *keys, int64_t o, int64_t ns, int shift0, int passes,
                               CtaSortSharedT<T> &sm) {
    for (int i = threadIdx.x; i < kCtaMaxPasses * kCtaRadix; i += T) (&sm.hist[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = o + threadIdx.x; i < o + ns; i += T) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p)
            atomicAdd(&sm.hist[p][(k >> (shift0 + p * kCtaRadixBits)) & (kCtaRadix - 1)], 1u);
    }
    __syncthreads();
}

// Stable LSD sort of [o, o + ns) by the digits at shift0 + 8 p, p < passes,
// with sm.hist holding each pass's digit counts.  Buffers alternate
// (keys, vals) -> (alt_k, alt_v) -> ...; with index_vals the first pass takes
// each element's own position as its value.  Returns the number of passes
// (the result is in alt_k / alt_v when it is odd).
template <int T>
__device__ int cta_lsd_sort(uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v,
                            int64_t o, int64_t ns, int shift0, int passes, bool index_vals,
                            CtaSortSharedT<T> &sm) {
    constexpr int kCtaWarps = CtaSortSharedT<T>::WARPS;
    constexpr int kCtaTile = CtaSortSharedT<T>::TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *src = keys, *dst = alt_k;
    int32_t *vsrc = vals, *vdst = alt_v;
    for (int p = 0; p < passes; ++p) {
        const int shift = shift0 + p * kCtaRadixBits;
        cta_digit_scan<T>(sm.hist[p], sm.run, false, sm.carry);
        for (int64_t tb = 0; tb < ns; tb += kCtaTile) {
            const int valid = (int)min64(kCtaTile, ns - tb);
            for (int i = threadIdx.x; i < kCtaWarps * (kCtaRadix + 1); i += T)
                (&sm.warp_hist[0][0])[i] = 0;
            __syncthreads();
            uint64_t key[kCtaItems];
            int32_t val[kCtaItems];
            uint32_t rank[kCtaItems];
            const int wbase = warp * 32 * kCtaItems;
#pragma unroll
            for (int i = 0; i < kCtaItems; ++i) {
                const int e = wbase + i * 32 + lane;
                if (e < valid) {
                    key[i] = src[o + tb + e];
                    val[i] = (p == 0 && index_vals) ? (int32_t)(o + tb + e) : vsrc[o + tb + e];
                } else {
                    key[i] = 0;
                    val[i] = 0;
                }
            }
            // stable warp ranking: ballot peer masks, leader-updated counters
            const unsigned lt = lanemask_lt();
            uint32_t oldc[kCtaItems], lr[kCtaItems];
#pragma unroll
            for (int i = 0; i < kCtaItems; ++i) {
                const int e = wbase + i * 32 + lane;
                const uint32_t d = (e < valid) ? (uint32_t)((key[i] >> shift) & (kCtaRadix - 1))
                                               : (uint32_t)kCtaRadix;
                unsigned peers = 0xffffffffu;
#pragma unroll
                for (int b = 0; b <= kCtaRadixBits; ++b) {
                    const bool bit = (d >> b) & 1u;
                    const unsigned v = __ballot_sync(0xffffffffu, bit);
                    peers &= bit ? v : ~v;
                }
                const int leader = __ffs(peers) - 1;
                oldc[i] = (lane == leader) ? atomicAdd(&sm.warp_hist[warp][d], (uint32_t)__popc(peers)) : 0u;
                lr[i] = (uint32_t)leader | ((uint32_t)__popc(peers & lt) << 8);
            }
#pragma unroll
            for (int i = 0; i < kCtaItems; ++i)
                rank[i] = __shfl_sync(0xffffffffu, oldc[i], lr[i] & 31u) + (lr[i] >> 8);
            __syncthreads();
            // warp offsets within each digit, tile digit counts
            for (int d = threadIdx.x; d < kCtaRadix; d += T) {
                uint32_t acc = 0;
                for (int w = 0; w < kCtaWarps; ++w) {
                    const uint32_t c = sm.warp_hist[w][d];
                    sm.warp_hist[w][d] = acc;
                    acc += c;
                }
                sm.cnt[d] = acc;
            }
            __syncthreads();
            cta_digit_scan<T>(sm.cnt, sm.tile_off, true, sm.carry);
#pragma unroll
            for (int i = 0; i < kCtaItems; ++i) {
                const int e = wbase + i * 32 + lane;
                if (e < valid) {
                    const uint32_t d = (uint32_t)((key[i] >> shift) & (kCtaRadix - 1));
                    const uint32_t ps = sm.tile_off[d] + sm.warp_hist[warp][d] + rank[i];
                    sm.keys[ps] = key[i];
                    sm.vals[ps] = val[i];
                }
            }
            __syncthreads();
            for (int j = threadIdx.x; j < valid; j += T) {
                const uint64_t k = sm.keys[j];
                const uint32_t d = (uint32_t)((k >> shift) & (kCtaRadix - 1));
                const int64_t to = o + sm.run[d] + (j - sm.tile_off[d]);
                dst[to] = k;
                vdst[to] = sm.vals[j];
            }
            __syncthreads();
            for (int d = threadIdx.x; d < kCtaRadix; d += T) sm.run[d] += sm.cnt[d];
            __syncthreads();
        }
        uint64_t *t = src; src = dst; dst = t;
        int32_t *u = vsrc; vsrc = vdst; vdst = u;
    }
    return passes;
}

}  // namespace
}  // namespace tb
