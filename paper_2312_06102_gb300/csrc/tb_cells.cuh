// tb_cells.cuh -- device code shared by the single-tree and the batched cell
// emission: the per-tile derivation of m_k and L_k and of the per-level start
// masks, and the cells one particle opens and closes.  See tb_cells.cu for
// the method.
#pragma once

#include "tb_device.cuh"

namespace tb {
namespace {

constexpr int kLvThreads = 1024;
constexpr int kLvWarps = kLvThreads / 32;
constexpr int kLvTile = kLvThreads;   // one particle per thread

__host__ __device__ inline int lv_pow2(int ncrit) {
    int p = 1;
    while (2 * p <= ncrit + 1) p *= 2;
    return p;
}

// Shared memory of tile_front for tiles of T particles.
template <int T = kLvTile>
__host__ __device__ inline size_t lv_smem_bytes(int ncrit) {
    size_t ext = (size_t)T + 2 * (size_t)ncrit + 1;   // keys of [s-n-1, e+n)
    size_t nc = (size_t)T + ncrit + 1;                // c over [s-n-1, e)
    return ((ext * 8 + 15) & ~size_t(15)) + 2 * ((nc + 15) & ~size_t(15)) + 64;
}

struct Front {
    int m, L, Lprev;      // this thread's particle k (m = 255 beyond the tile)
    int64_t k;
};

// Shared state of one tile of T particles (one per thread): masks and counts
// per warp and field (fields 0..21 = cell starts per level, 22 = leaf starts).
template <int T>
struct TileSharedT {
    static constexpr int WARPS = T / 32;
    uint32_t mask[WARPS][kLevelFields];
    uint32_t base[kLevelFields];
};
using TileShared = TileSharedT<kLvThreads>;

// Per-warp masks of the lanes starting a cell at each level (fields 0..21)
// and of the lanes starting a leaf (field 22).  Each lane holds the interval
// [m, L] as a row of bits; a 32 x 32 bit-matrix transpose across the warp
// (five exchange rounds) leaves in lane d the mask of field d.
template <int T>
__device__ __forceinline__ void store_level_masks(int m, int L, TileSharedT<T> &ts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = (m <= L) ? (((2u << L) - (1u << m)) | (1u << kLevels)) : 0u;
    uint32_t msk = 0x0000ffffu;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1, msk ^= msk << j) {
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        if (lane & j) x ^= ((y >> j) ^ x) & msk;
        else x ^= (((x >> j) ^ y) & msk) << j;
    }
    if (lane < kLevelFields) ts.mask[warp][lane] = x;
}

// m, L and L of the previous particle for particle s + threadIdx.x of the
// tile [s, e), and the ballot masks of the level starts of every warp.  The
// tile lies in the segment [seg_lo, seg_hi) of sorted keys that forms one
// tree (the whole array, or one set of a batch); keys outside it do not
// exist for this tree.
template <int T>
__device__ Front tile_front(const uint64_t *__restrict__ skeys, int64_t seg_lo, int64_t seg_hi,
                            int ncrit, int64_t s, int64_t e, unsigned char *raw, TileSharedT<T> &ts) {
    const int64_t lo = s - ncrit - 1;
    const int next = (int)(e + ncrit - lo);
    const int nc = (int)(e - lo);
    const size_t ext = (size_t)T + 2 * (size_t)ncrit + 1;
    const size_t ncp = ((size_t)T + ncrit + 1 + 15) & ~size_t(15);
    uint64_t *key = reinterpret_cast<uint64_t *>(raw);
    uint8_t *A = raw + ((ext * 8 + 15) & ~size_t(15));
    uint8_t *B = A + ncp;
    for (int x = threadIdx.x; x < next; x += T) {
        const int64_t i = lo + x;
        key[x] = (i >= seg_lo && i < seg_hi) ? skeys[i] : 0ull;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < nc; x += T) {
        const int64_t i = lo + x;
        int v = 0;
        if (i >= seg_lo && i + ncrit < seg_hi) v = min(kDepthMax, min_depth(key[x], key[x + ncrit]));
        A[x] = (uint8_t)v;
    }
    __syncthreads();
    const int p = lv_pow2(ncrit);
    for (int q = 1; q < p; q *= 2) {
        for (int x = threadIdx.x; x < nc; x += T)
            B[x] = (x + q < nc) ? max(A[x], A[x + q]) : A[x];
        __syncthreads();
        uint8_t *t = A; A = B; B = t;
    }
    // A[x] = max of c over [x, x + p) (truncated at the end)
    Front f;
    f.k = s + threadIdx.x;
    auto window = [&](int64_t k) {   // max c over [k - n, k], k in [s - 1, e)
        const int x0 = (int)(k - ncrit - lo), x1 = (int)(k - p + 1 - lo);
        return (int)max(A[x0], A[x1]);
    };
    if (f.k < e) {
        const int x = (int)(f.k - lo);
        f.m = (f.k == seg_lo) ? 0 : min_depth(key[x - 1], key[x]);
        f.L = window(f.k);
        f.Lprev = window(f.k - 1);
    } else {
        f.m = 255;
        f.L = 0;
        f.Lprev = 0;
    }
    store_level_masks(f.m, f.L, ts);
    __syncthreads();
    return f;
}

// The same Front from the m_k | L_k << 8 words a counting pass stored for
// every particle (no keys needed): particle s + threadIdx.x of the tile
// [s, e) of the tree [seg_lo, ...), and the level masks of every warp.
template <int T>
__device__ Front tile_front_ml(const uint16_t *__restrict__ ml, int64_t seg_lo, int64_t s,
                               int64_t e, TileSharedT<T> &ts) {
    Front f;
    f.k = s + threadIdx.x;
    if (f.k < e) {
        const uint32_t v = ml[f.k];
        f.m = (int)(v & 0xffu);
        f.L = (int)(v >> 8);
        f.Lprev = (f.k > seg_lo) ? (int)(ml[f.k - 1] >> 8) : 0;
    } else {
        f.m = 255;
        f.L = 0;
        f.Lprev = 0;
    }
    store_level_masks(f.m, f.L, ts);
    __syncthreads();
    return f;
}

// Per-field prefix over the warps of a tile, one warp per field (fields
// 0..22, taken in turns when the tile has fewer than 23 warps), one lane per
// warp of the tile: woff[w][f] = starts of field f in warps before w; tot[f] =
// the tile's total.  Needs a barrier before (masks written) and after
// (results read).
template <int T>
__device__ __forceinline__ void warp_field_prefix(const TileSharedT<T> &ts,
                                                  uint32_t (*woff)[kLevelFields], uint32_t *tot) {
    constexpr int W = TileSharedT<T>::WARPS;
    const int lane = threadIdx.x & 31;
    for (int f = threadIdx.x >> 5; f < kLevelFields; f += W) {
        const uint32_t v = lane < W ? __popc(ts.mask[lane][f]) : 0u;
        uint32_t x = v;
#pragma unroll
        for (int sh = 1; sh < 32; sh <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, sh);
            if (lane >= sh) x += y;
        }
        if (woff && lane < W) woff[lane][f] = x - v;
        if (lane == 31) tot[f] = x;
    }
}

struct EmitOut {
    uint64_t *ckey;
    uint8_t *level;
    int32_t *parent, *child_first, *child_end, *pfirst, *pend;
    int32_t *leaf_cell;
};

// Cells opened and closed by one particle.  P(d) is the global index of the
// next level-d cell before k's own starts (P(kLevels): next leaf slot);
// seg_hi is one past the tree's last particle; K is k's key.
template <class PF>
__device__ __forceinline__ void emit_particle(const Front &f, const PF &P, int64_t seg_lo,
                                              int64_t seg_hi, uint64_t K, const EmitOut &out) {
    const int64_t k = f.k;
    const int m = f.m, L = f.L;
    if (k > seg_lo) {
        // close the cells holding k-1 but not k
        for (int d = m; d <= f.Lprev; ++d) {
            const uint32_t idx = P(d) - 1;
            out.pend[idx] = (int32_t)k;
            out.child_end[idx] = (d < f.Lprev) ? (int32_t)P(d + 1) : -1;
        }
    }
    if (m <= L) {
        for (int d = m; d <= L; ++d) {
            const uint32_t idx = P(d);
            out.ckey[idx] = cell_key(K, d);
            out.level[idx] = (uint8_t)d;
            out.pfirst[idx] = (int32_t)k;
            out.parent[idx] = (d == 0) ? -1 : (int32_t)P(d - 1) - (d == m ? 1 : 0);
            out.child_first[idx] = (d < L) ? (int32_t)P(d + 1) : -1;
        }
        out.leaf_cell[P(kLevels)] = (int32_t)P(L);
    }
    if (k == seg_hi - 1) {
        // the tree's last particle closes every cell holding it
        for (int d = 0; d <= L; ++d) {
            const uint32_t own = (m <= d) ? 1u : 0u;
            const uint32_t idx = P(d) + own - 1;
            out.pend[idx] = (int32_t)seg_hi;
            out.child_end[idx] = (d < L) ? (int32_t)(P(d + 1) + ((m <= d + 1) ? 1u : 0u)) : -1;
        }
    }
}

}  // namespace
}  // namespace tb
