// tb_runs.cuh -- the in-place ordering of the runs of equal upper key bits
// left by radix passes over the upper bits only (see tb_runs.cu), one tile of
// 2048 positions at a time by one block; shared by the single-tree sort and
// the per-set sorts of the batched build.
#pragma once

#include "tb_ctasort.cuh"

namespace tb {
namespace {

constexpr int kRunTile = 2048;
constexpr int kRunMax = 128;                                 // longest run ordered in place
constexpr int kRunSpan = kRunTile + kRunMax;                 // positions a tile loads
constexpr int kRunChunks = kRunSpan / 32 + 1;                // 32-position start masks (+ one past)

struct RunSmem {
    // sk[x + 2] = keys[s + x] for x in [-1, nw); sk[nw + 2] is a sentinel
    // whose upper bits differ from every key's (keys leave bit 63 clear)
    __align__(16) uint64_t sk[kRunSpan + 4];
    uint32_t smask[kRunChunks];   // bit l of chunk c: position 32 c + l starts a run
};

// Orders in place, by (low shift0 bits, position), every run of equal
// key >> shift0 that starts in the tile [s, s + 2048) of the range [lo, hi)
// and holds at most kRunMax keys; calls queue_long(a) once for each longer run
// starting at a in the tile.  All THREADS threads of the block take part.
// Returns, the same in every thread, whether a key of the tile is smaller
// than its predecessor in the same run (a descent).
template <int THREADS, class QueueLong>
__device__ bool run_tile(uint64_t *__restrict__ keys, int32_t *__restrict__ vals, int64_t lo, int64_t s,
                         int64_t hi, int shift0, RunSmem &S, QueueLong queue_long) {
    constexpr int PER = kRunTile / THREADS;
    uint64_t *sk = S.sk;
    uint32_t *smask = S.smask;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int te = (int)min64(kRunTile, hi - s);
    const int nw = (int)min64(kRunSpan, hi - s);
    if ((reinterpret_cast<uintptr_t>(keys + s) & 15u) == 0) {
        const ulonglong2 *src2 = reinterpret_cast<const ulonglong2 *>(keys + s);
        ulonglong2 *dst2 = reinterpret_cast<ulonglong2 *>(sk + 2);
        for (int x = threadIdx.x; x < nw / 2; x += THREADS) dst2[x] = src2[x];
        if (threadIdx.x == 0 && (nw & 1)) sk[nw + 1] = keys[s + nw - 1];
    } else {
        for (int x = threadIdx.x; x < nw; x += THREADS) sk[x + 2] = keys[s + x];
    }
    if (threadIdx.x == 0) {
        sk[1] = s > lo ? keys[s - 1] : ~0ull;
        sk[nw + 2] = ~0ull;
    }
    __syncthreads();
    const uint64_t lim = uint64_t(1) << shift0;   // equal upper bits <=> xor below lim
    const uint64_t lowm = lim - 1;
    // start masks; positions past the loaded ones count as starts
    bool multi = false;
    for (int c = warp; c < kRunChunks; c += THREADS / 32) {
        const int x = c * 32 + lane;
        const bool st = x >= nw || ((sk[x + 2] ^ sk[x + 1]) >= lim);
        const uint32_t m = __ballot_sync(0xffffffffu, st);
        if (lane == 0) smask[c] = m;
        multi |= (m != 0xffffffffu) && c * 32 <= te;   // includes position te (a run from te - 1)
    }
    // a tile of single-key runs is done (the barrier also publishes the masks)
    if (!__syncthreads_or(multi)) return false;
    // a run crossing the tile's end: its members past the end move too
    const bool crossing = te == kRunTile && nw > te && !((smask[te >> 5] >> (te & 31)) & 1u);
    int32_t dst[PER + 1];   // new position - s of the key at position x, or -1
    int32_t val[PER + 1];
    bool desc = false;
#pragma unroll
    for (int i = 0; i <= PER; ++i) {
        dst[i] = -1;
        const int x = i < PER ? (int)threadIdx.x + i * THREADS : te + (int)threadIdx.x;
        if (i < PER ? x >= te : (!crossing || x >= nw)) continue;
        const int c = x >> 5, l = x & 31;
        const uint32_t m = smask[c];
        const bool st_here = (m >> l) & 1u;
        const bool st_next = l < 31 ? ((m >> (l + 1)) & 1u) : (smask[c + 1] & 1u);
        if (st_here && st_next) continue;               // a run of one key
        const uint64_t kx = sk[x + 2];
        if (!st_here) desc |= (kx & lowm) < (sk[x + 1] & lowm);
        // the run [a, b) from the start masks, looking at most kScan chunks
        // away: a run that reaches further is longer than kRunMax, and the
        // member at its start queues it
        constexpr int kScan = kRunMax / 32 + 2;
        int a = -1;
        const uint32_t le = m & (0xffffffffu >> (31 - l));
        if (le) {
            a = c * 32 + 31 - __clz(le);
        } else {
            for (int cc = c - 1; cc >= 0 && cc >= c - kScan; --cc) {
                const uint32_t mc = smask[cc];
                if (mc) {
                    a = cc * 32 + 31 - __clz(mc);
                    break;
                }
            }
            if (a < 0) continue;                        // began before this tile, or long
        }
        if (a >= te) continue;                          // the run begins after this tile
        const uint32_t gt = l < 31 ? (m & (0xffffffffu << (l + 1))) : 0u;
        int b = -1;                                     // stays -1 for a long run
        if (gt) {
            b = c * 32 + __ffs(gt) - 1;
        } else {
            // the chunk holding position nw starts runs from there on
            for (int cc = c + 1; cc < kRunChunks && cc <= c + kScan; ++cc) {
                const uint32_t mc = smask[cc];
                if (mc) {
                    b = cc * 32 + __ffs(mc) - 1;
                    break;
                }
            }
        }
        if (b > nw) b = nw;
        // longer runs (including any that reach the end of the loaded span
        // before the end of the keys) go to the block sort
        if (b < 0 || b - a > kRunMax) {
            if (x == a) queue_long(s + a);
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
#pragma unroll
    for (int i = 0; i <= PER; ++i) {
        if (dst[i] < 0) continue;
        const int x = i < PER ? (int)threadIdx.x + i * THREADS : te + (int)threadIdx.x;
        keys[s + dst[i]] = sk[x + 2];
        vals[s + dst[i]] = val[i];
    }
    __syncthreads();   // the shared tile may be reloaded next
    return desc;
}

}  // namespace
}  // namespace tb
