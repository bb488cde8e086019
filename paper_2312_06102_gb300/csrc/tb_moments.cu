// tb_moments.cu -- cell moments without traversing the tree (Sec. 2.3: cell
// properties are computed as cells are created; the centre of mass of a
// parent comes from those of its children, higher multipoles likewise).
//
//   leaf_tile_kernel     : every leaf, one block per tile of 2048 positions in
//                          key order: the tile's permutation bulk-copied (TMA)
//                          into shared memory, its (x, y, z, m) records
//                          gathered beside it (Sec. 2.3 step 3, the reorder),
//                          one thread per leaf summing from there;
//   long_leaf_kernel     : leaves the tile could not hold, members read
//                          through the permutation;
//   big_leaf_kernel      : depth-21 leaves of identical keys that are too long
//                          for one thread, summed block-wide;
//   level_moments_kernel : one launch per level, deepest first: the children
//                          of the level, in tiles bulk-copied (TMA) into
//                          shared memory, and every non-leaf cell of the
//                          level combined from its tile.
//
// Moments of a cell: M = sum m; centre of mass c = sum m x / M; central
// second moment Q = sum m (x - c)(x - c)^T (6 components xx xy xz yy yz zz);
// member bounding box.  Sums run relative to a reference point inside the
// cell (the first member particle for a leaf, the first child's centre for a
// parent), which keeps the FP32 differences small and exact or nearly so.
// Parent from children (parallel-axis theorem):
//   M = sum M_j, c = sum M_j c_j / M, Q = sum [Q_j + M_j (c_j - c)(c_j - c)^T].
//
// Modes:
//   FP32_COMP  -- two-sum / two-product compensated FP32; the centre of mass
//                 is kept as an unevaluated pair com + com_lo (an FP32 value
//                 cannot hold a deep cell's centre to 2e-6 of its side);
//   FP32_PLAIN -- uncompensated FP32, com_lo = 0;
//   FP64       -- FP64 accumulation; FP64 outputs beside the FP32 ones.
// A leaf of more than 2^20 particles is summed in FP64 in every mode, and so
// is a parent of that many in the FP32-plain mode; compensated parents stay
// in FP32 at every size (their error is relative to their own mass and side).
#include "tb_moments.cuh"

namespace tb {

namespace {

// ------------------------------------------------------------ kernels

// Shuffle every field of an accumulator down the warp by `off` lanes.
template <class Acc>
__device__ __forceinline__ Acc shfl_down_acc(const Acc &a, int off) {
    Acc b;
    constexpr int W = sizeof(Acc) / 4;
    static_assert(sizeof(Acc) % 4 == 0, "accumulators are made of 4-byte words");
    const uint32_t *u = reinterpret_cast<const uint32_t *>(&a);
    uint32_t *v = reinterpret_cast<uint32_t *>(&b);
#pragma unroll
    for (int i = 0; i < W; ++i) v[i] = __shfl_down_sync(0xffffffffu, u[i], off);
    return b;
}

// One leaf [pf, pe) summed by a whole warp (all 32 lanes call it): each lane
// sums a stride of the members about the leaf's first member, then the
// lanes' sums merge in a fixed tree (compensated merges in the compensated
// mode) and lane 0 writes the cell.  `src` is any source of key-ordered
// records (shared memory, or a PermSrc).
template <int MODE, class Src>
__device__ __forceinline__ void warp_leaf_sum(const MomOut &o, Src src, int64_t c, int64_t pf,
                                              int64_t pe) {
    using Acc = typename std::conditional<
        MODE == TB_MOM_FP64, AccD,
        typename std::conditional<MODE == TB_MOM_FP32_COMP, AccC, AccP>::type>::type;
    const int lane = threadIdx.x & 31;
    const float4 r0 = src[pf];
    const float ref[3] = {r0.x, r0.y, r0.z};
    float bb[6] = {r0.x, r0.y, r0.z, r0.x, r0.y, r0.z};
    Acc A;
    A.init();
    for (int64_t k = pf + lane; k < pe; k += 32) {
        const float4 v = src[k];
        const float x[3] = {v.x, v.y, v.z};
        for (int a = 0; a < 3; ++a) {
            bb[a] = fminf(bb[a], x[a]);
            bb[3 + a] = fmaxf(bb[3 + a], x[a]);
        }
        if constexpr (MODE == TB_MOM_FP64) {
            const double dx[3] = {(double)x[0] - (double)ref[0], (double)x[1] - (double)ref[1],
                                  (double)x[2] - (double)ref[2]};
            A.add((double)v.w, dx);
        } else {
            const float dx[3] = {__fsub_rn(x[0], ref[0]), __fsub_rn(x[1], ref[1]),
                                 __fsub_rn(x[2], ref[2])};
            A.add(v.w, dx);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Acc B = shfl_down_acc(A, off);
        A.merge(B);
        for (int a = 0; a < 3; ++a) {
            bb[a] = fminf(bb[a], __shfl_down_sync(0xffffffffu, bb[a], off));
            bb[3 + a] = fmaxf(bb[3 + a], __shfl_down_sync(0xffffffffu, bb[3 + a], off));
        }
    }
    if (lane == 0) {
        if constexpr (MODE == TB_MOM_FP64) finish_d(o, c, A, ref, bb, true);
        else if constexpr (MODE == TB_MOM_FP32_COMP) finish_c(o, c, A, ref, bb);
        else finish_p(o, c, A, ref, bb);
    }
}

// Leaves, one block per tile of kLtTile consecutive key-order positions.
//   1. The permutation of the tile and of a halo of kLtHalo positions past
//      it is bulk-copied (TMA) into shared memory, and m_k | L_k << 8 of the
//      same positions is read beside it.
//   2. The records (x, y, z, m) of those particles are gathered into shared
//      memory: xm[perm[k]] (Sec. 2.3 step 3).  When the permutation of the
//      span is one ascending run -- input already in key order, as after a
//      reorder -- the records are one contiguous stretch and come in with one
//      bulk copy instead.  With `xs` set (pos_sorted asked for), the tile's
//      records are bulk-stored to it.
//   3. k starts a leaf iff m_k <= L_k (Alg. 1 as a closed form); leaves tile
//      the key order, so a leaf ends where the next one starts.  The leaves
//      starting in the tile are listed in order; their index among all
//      leaves comes from the scanned per-tile leaf counts of the cell pass.
//   4. One thread per leaf sums its members from shared memory.  A leaf that
//      runs past the staged span (only a depth-21 leaf of identical keys, or
//      n_crit above the halo, can) and, in the compensated mode, a leaf of
//      more than kSplitLeaf members go to the queue of long_leaf_kernel.
constexpr int kLtThreads = 256;
constexpr int kLtTile = 2048;                  // two cell-pass tiles of 1024
constexpr int kLtHalo = 64;
constexpr int kLtSpan = kLtTile + kLtHalo;
constexpr int kLtPer = kLtTile / kLtThreads;   // positions per thread when listing starts
static_assert(kLtTile == 2 * 1024, "leaf tiles span two tiles of the cell pass");

struct LeafTileSmem {
    float4 rec[kLtSpan];
    int32_t perm[kLtSpan];
    uint16_t ml[kLtSpan];
    uint16_t start[kLtTile];                   // offsets of the leaf starts in the tile
    uint32_t wcount[kLtThreads / 32];
    int32_t next_start;                        // first start at or past the tile end, or -1
    // compensated mode: staged leaves of more than kSplitLeaf members, summed
    // by whole warps after the short ones (at most kLtTile / 17 of them)
    int32_t long_c[kLtTile / (kSplitLeaf + 1) + 1];
    uint32_t long_x[kLtTile / (kSplitLeaf + 1) + 1];   // start | end << 16 (tile offsets)
    uint32_t n_long;
    uint64_t bar;
};

size_t leaf_tile_smem() { return sizeof(LeafTileSmem); }

template <int MODE>
__global__ void __launch_bounds__(kLtThreads, 4)
    leaf_tile_kernel(MomOut o, const int32_t *__restrict__ leaf_cell,
                     const int32_t *__restrict__ perm, const float4 *__restrict__ xm,
                     const uint16_t *__restrict__ ml, const uint32_t *__restrict__ leaf_off,
                     int64_t n, float4 *__restrict__ xs, int32_t *long_queue, DevInfo *info,
                     int64_t wait_limit) {
    if (info->status & (kErrOverflow | kErrNonFinite | kErrTimeout)) return;
    extern __shared__ __align__(128) unsigned char lt_raw[];
    LeafTileSmem &S = *reinterpret_cast<LeafTileSmem *>(lt_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * kLtTile;
    const int span = (int)min64(kLtSpan, n - k0);
    const int te = (int)min64(kLtTile, n - k0);
    // 1. permutation of the span: its whole 16-byte groups by bulk copy
    //    (k0 is a multiple of 4), the rest by plain loads
    const int nbulk = span & ~3;
    if (threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        mbar_init_fence();
        if (nbulk > 0) {
            mbar_arrive_expect_tx(&S.bar, (uint32_t)nbulk * 4u);
            bulk_load(S.perm, perm + k0, (uint32_t)nbulk * 4u, &S.bar);
        }
    }
    for (int x = nbulk + (int)threadIdx.x; x < span; x += kLtThreads) S.perm[x] = perm[k0 + x];
    for (int x = threadIdx.x; x < span; x += kLtThreads) S.ml[x] = ml[k0 + x];
    __syncthreads();
    uint32_t phase = 0;
    bool ok = true;
    if (nbulk > 0) {
        ok = mbar_wait_bounded(&S.bar, phase, wait_limit);
        phase ^= 1u;
    }
    // a copy that did not complete: record it and leave once it has
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
            flag_error(&info->status, kErrTimeout);
            mbar_wait_bounded(&S.bar, 0, wait_limit);
        }
        return;
    }
    // 2. records of the span
    bool run = true, in_range = true;
    for (int x = threadIdx.x; x < span; x += kLtThreads) {
        const int32_t p = S.perm[x];
        in_range &= (uint32_t)p < (uint32_t)n;
        if (x + 1 < span) run &= S.perm[x + 1] == p + 1;
    }
    if (!__syncthreads_and(in_range)) {
        if (threadIdx.x == 0) flag_error(&info->status, kErrTimeout);
        return;
    }
    if (__syncthreads_and(run)) {
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&S.bar, (uint32_t)span * 16u);
            bulk_load(S.rec, xm + S.perm[0], (uint32_t)span * 16u, &S.bar);
        }
        ok = mbar_wait_bounded(&S.bar, phase, wait_limit);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                flag_error(&info->status, kErrTimeout);
                mbar_wait_bounded(&S.bar, phase, wait_limit);
            }
            return;
        }
    } else {
        // random gather: every record of the span in flight at once, by
        // asynchronous copies that hold no registers
        for (int x = threadIdx.x; x < span; x += kLtThreads) cp_async16(&S.rec[x], xm + S.perm[x]);
        cp_async_wait_all();
        __syncthreads();
    }
    // the reordered records, when asked for, go out by one bulk store (every
    // thread orders its shared-memory writes before the store reads them)
    if (xs) {
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) bulk_store(xs + k0, S.rec, (uint32_t)te * 16u);
    }
    // 3. leaf starts of the tile, in order
    uint32_t flags = 0;
#pragma unroll
    for (int j = 0; j < kLtPer; ++j) {
        const int x = threadIdx.x * kLtPer + j;
        if (x < te) {
            const uint32_t v = S.ml[x];
            if ((v & 0xffu) <= (v >> 8)) flags |= 1u << j;
        }
    }
    const uint32_t cnt = __popc(flags);
    uint32_t incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) S.wcount[warp] = incl;
    // the first start at or past the tile's end, from the halo: warp 0
    if (warp == 0) {
        int32_t nx = -1;
        for (int x0 = te; x0 < span && nx < 0; x0 += 32) {
            const int x = x0 + lane;
            bool st = false;
            if (x < span) {
                const uint32_t v = S.ml[x];
                st = (v & 0xffu) <= (v >> 8);
            }
            const unsigned b = __ballot_sync(0xffffffffu, st);
            if (b) nx = x0 + __ffs(b) - 1;
        }
        // the end of the array ends the last leaf
        if (nx < 0 && k0 + span == n) nx = span;
        if (lane == 0) {
            S.next_start = nx;
            S.n_long = 0;
        }
    }
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kLtThreads / 32; ++w) {
        const uint32_t c = S.wcount[w];
        if (w < warp) before += c;
        total += c;
    }
    uint32_t pos = before + incl - cnt;
#pragma unroll
    for (int j = 0; j < kLtPer; ++j)
        if (flags & (1u << j)) S.start[pos++] = (uint16_t)(threadIdx.x * kLtPer + j);
    __syncthreads();
    // 4. one thread per leaf
    const uint32_t jbase = leaf_off[2 * blockIdx.x];
    const int32_t nxt = S.next_start;
    for (uint32_t r = threadIdx.x; r < total; r += kLtThreads) {
        const int x = S.start[r];
        const int xe = (r + 1 < total) ? (int)S.start[r + 1] : nxt;
        const int64_t c = leaf_cell[jbase + r];
        const bool staged = xe >= 0;
        if (!staged) {
            long_queue[atomicAdd(&info->misc_ctr[5], 1u)] = (int32_t)c;
            continue;
        }
        if (MODE == TB_MOM_FP32_COMP && xe - x > kSplitLeaf) {
            const uint32_t q = atomicAdd(&S.n_long, 1u);
            S.long_c[q] = (int32_t)c;
            S.long_x[q] = (uint32_t)x | ((uint32_t)xe << 16);
            continue;
        }
        if constexpr (MODE == TB_MOM_FP32_COMP) leaf_sum_split(o, (const float4 *)S.rec, c, x, xe);
        else leaf_sum<MODE>(o, (const float4 *)S.rec, c, x, xe);
    }
    if constexpr (MODE == TB_MOM_FP32_COMP) {
        __syncthreads();
        const uint32_t nl = S.n_long;
        for (uint32_t q = warp; q < nl; q += kLtThreads / 32) {
            const uint32_t xx = S.long_x[q];
            warp_leaf_sum<TB_MOM_FP32_COMP>(o, (const float4 *)S.rec, S.long_c[q], xx & 0xffffu,
                                            xx >> 16);
        }
    }
    if (xs && threadIdx.x == 0) bulk_store_wait_read();
}

// The queued leaves, one warp per leaf, members read through the
// permutation (32 independent loads per round).  Leaves of more than
// kBigLeafThread members -- only depth-21 leaves of identical keys -- are
// queued again for big_leaf_kernel.
template <int MODE>
__global__ void __launch_bounds__(kMomThreads, 4)
    long_leaf_kernel(TreeIn T, MomOut o, PermSrc src, const int32_t *long_queue, DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite | kErrTimeout)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nq = *(volatile const uint32_t *)&info->misc_ctr[5];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; q < nq; q += nwarps) {
        const int64_t c = long_queue[q];
        const int64_t pf = T.pfirst[c], pe = T.pend[c];
        if (pe - pf > kBigLeafThread) {
            if (lane == 0) T.big_leaf[atomicAdd(&info->misc_ctr[2], 1u)] = (int32_t)c;
            continue;
        }
        warp_leaf_sum<MODE>(o, src, c, pf, pe);
    }
}

// Non-leaf cells of level d from their children at level d + 1, which the
// leaf launches or the launch for level d + 1 finished.  The children of
// consecutive cells are consecutive cells, so level d + 1 is cut into tiles
// of kLmTile children: a block bulk-copies (TMA) the FP32 moments and the
// parent links of its tile -- plus the few children past it that belong to
// its last parents -- into shared memory, lists the parents whose first
// child lies in the tile (a child is the first of its parent iff its parent
// differs from the previous cell's), and combines them there.  Each copy
// covers whole groups of four cells, so that every array's piece starts on a
// 16-byte boundary; the moment and parent arrays are allocated kMomentPad
// cells past the capacity, which the rounding never passes.  The up to three
// cells the rounding adds before a level's first tile belong to level d,
// which this launch writes: they are copied but never read.  Blocks loop
// over the tiles of the level (one persistent grid per launch).
constexpr int kLmThreads = 128;
constexpr int kLmTile = 512;
constexpr int kLmSpan = kLmTile + 16;   // 3 before the tile, 7 past it, rounding to 4

struct LevelSmem {
    float mass[kLmSpan];
    float com[3 * kLmSpan];
    float com_lo[3 * kLmSpan];
    float quad[6 * kLmSpan];
    float aabb[6 * kLmSpan];
    int32_t par[kLmSpan + 4];                 // parents of the staged cells and of 4 before
    int32_t own[kLmTile];                     // parents whose first child is in the tile
    uint32_t wcount[kLmThreads / 32];
    uint64_t bar;
};
static_assert(kLmSpan % 4 == 0, "each staged array spans whole 16-byte groups");
static_assert(kLmTile == 4 * kLmThreads, "the listing takes four children per thread");

// Children's FP32 moments staged in shared memory: cell c at slot c - base.
struct CellsStaged {
    const LevelSmem *S;
    int64_t base;
    __device__ __forceinline__ float m(int64_t c) const { return S->mass[c - base]; }
    __device__ __forceinline__ float x(int64_t c, int a) const { return S->com[3 * (c - base) + a]; }
    __device__ __forceinline__ float xl(int64_t c, int a) const { return S->com_lo[3 * (c - base) + a]; }
    __device__ __forceinline__ float2 q2(int64_t c, int i) const {
        return reinterpret_cast<const float2 *>(S->quad + 6 * (c - base))[i];
    }
    __device__ __forceinline__ float2 b2(int64_t c, int i) const {
        return reinterpret_cast<const float2 *>(S->aabb + 6 * (c - base))[i];
    }
};

template <int MODE>
__global__ void __launch_bounds__(kLmThreads, 5)
    level_moments_kernel(TreeIn T, MomOut o, DevInfo *info, int d, int64_t wait_limit) {
    if (info->status & (kErrOverflow | kErrNonFinite | kErrTimeout)) return;
    extern __shared__ __align__(128) unsigned char lm_raw[];
    LevelSmem &S = *reinterpret_cast<LevelSmem *>(lm_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t off1 = info->level_offset[d + 1], off2 = info->level_offset[d + 2];
    const int64_t tiles = (off2 - off1 + kLmTile - 1) / kLmTile;
    if ((int64_t)blockIdx.x >= tiles) return;
    if (threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t c_lo = off1 + t * kLmTile, c_hi = min64(c_lo + kLmTile, off2);
        const int64_t s_lo = c_lo & ~int64_t(3);
        const int64_t s_hi = (min64(c_hi + 7, off2) + 3) & ~int64_t(3);
        // parent links from one group of four before s_lo (the cell before
        // c_lo), or from the level's start
        const int64_t p_lo = s_lo >= off1 + 4 ? s_lo - 4 : (off1 & ~int64_t(3));
        if (threadIdx.x == 0) {
            const uint32_t len = (uint32_t)(s_hi - s_lo);
            const uint32_t plen = (uint32_t)(s_hi - p_lo);
            mbar_arrive_expect_tx(&S.bar, len * 76u + plen * 4u);
            bulk_load(S.mass, o.mass + s_lo, len * 4u, &S.bar);
            bulk_load(S.com, o.com + 3 * s_lo, len * 12u, &S.bar);
            bulk_load(S.com_lo, o.com_lo + 3 * s_lo, len * 12u, &S.bar);
            bulk_load(S.quad, o.quad + 6 * s_lo, len * 24u, &S.bar);
            bulk_load(S.aabb, o.aabb + 6 * s_lo, len * 24u, &S.bar);
            bulk_load(S.par, T.parent + p_lo, plen * 4u, &S.bar);
        }
        const bool ok = mbar_wait_bounded(&S.bar, phase, wait_limit);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                flag_error(&info->status, kErrTimeout);
                mbar_wait_bounded(&S.bar, phase ^ 1u, wait_limit);
            }
            return;
        }
        // the parents whose first child is in the tile, in order: four
        // children per thread, a warp prefix and one across the warps
        const int nt = (int)(c_hi - c_lo);
        uint32_t fl = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = 4 * (int)threadIdx.x + j;
            if (x < nt) {
                const int64_t c = c_lo + x;
                if (c == off1 || S.par[c - p_lo] != S.par[c - 1 - p_lo]) fl |= 1u << j;
            }
        }
        const uint32_t cnt = __popc(fl);
        uint32_t incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) S.wcount[warp] = incl;
        __syncthreads();
        uint32_t pos = incl - cnt, before = 0;
#pragma unroll
        for (int w = 0; w < kLmThreads / 32; ++w) {
            const uint32_t v = S.wcount[w];
            if (w < warp) pos += v;
            before += v;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (fl & (1u << j)) S.own[pos++] = S.par[c_lo + 4 * (int)threadIdx.x + j - p_lo];
        __syncthreads();
        const CellsStaged src{&S, s_lo};
        for (uint32_t i = threadIdx.x; i < before; i += kLmThreads)
            combine_children<MODE>(T, o, S.own[i], src);
        // the next tile's copies overwrite what this one read
        fence_proxy_async_smem();
        __syncthreads();
    }
}

// Block-wide sums of the long depth-21 leaves queued by the leaf launch.
template <int MODE>
__global__ void __launch_bounds__(kBigThreads)
    big_leaf_kernel(TreeIn T, MomOut o, PermSrc xs, DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite | kErrTimeout)) return;
    __shared__ uint32_t s_q;
    __shared__ float s_bb[kBigThreads][6];
    __shared__ double s_d[kBigThreads][10];
    __shared__ float s_f[kBigThreads][20];
    const uint32_t nq = *(volatile uint32_t *)&info->misc_ctr[2];
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(&info->misc_ctr[3], 1u);
        __syncthreads();
        const uint32_t q = s_q;
        __syncthreads();
        if (q >= nq) return;
        const int64_t c = T.big_leaf[q];
        const int64_t pf = T.pfirst[c], pe = T.pend[c];
        const int64_t cnt = pe - pf;
        const int64_t chunk = (cnt + kBigThreads - 1) / kBigThreads;
        const int64_t a0 = pf + threadIdx.x * chunk, a1 = min64(pe, a0 + chunk);
        const float4 r0 = xs[pf];
        const float ref[3] = {r0.x, r0.y, r0.z};
        float bb[6] = {r0.x, r0.y, r0.z, r0.x, r0.y, r0.z};
        const bool f64 = (MODE == TB_MOM_FP64) || cnt > kBigCell;
        AccD D;
        AccC Cc;
        AccP Pp;
        D.init(); Cc.init(); Pp.init();
        for (int64_t k = a0; k < a1; ++k) {
            const float4 v = xs[k];
            const float x[3] = {v.x, v.y, v.z};
            for (int a = 0; a < 3; ++a) { bb[a] = fminf(bb[a], x[a]); bb[3 + a] = fmaxf(bb[3 + a], x[a]); }
            if (f64) {
                double dx[3];
                for (int a = 0; a < 3; ++a) dx[a] = (double)x[a] - (double)ref[a];
                D.add((double)v.w, dx);
            } else {
                float dx[3];
                for (int a = 0; a < 3; ++a) dx[a] = __fsub_rn(x[a], ref[a]);
                if (MODE == TB_MOM_FP32_COMP) Cc.add(v.w, dx);
                else Pp.add(v.w, dx);
            }
        }
        // tree reduction in shared memory, fixed order
        for (int a = 0; a < 6; ++a) s_bb[threadIdx.x][a] = bb[a];
        if (f64) {
            s_d[threadIdx.x][0] = D.M;
            for (int a = 0; a < 3; ++a) s_d[threadIdx.x][1 + a] = D.S[a];
            for (int q2 = 0; q2 < 6; ++q2) s_d[threadIdx.x][4 + q2] = D.Q[q2];
        } else if (MODE == TB_MOM_FP32_COMP) {
            s_f[threadIdx.x][0] = Cc.M; s_f[threadIdx.x][1] = Cc.Mc;
            for (int a = 0; a < 3; ++a) { s_f[threadIdx.x][2 + a] = Cc.S[a]; s_f[threadIdx.x][5 + a] = Cc.Sc[a]; }
            for (int q2 = 0; q2 < 6; ++q2) { s_f[threadIdx.x][8 + q2] = Cc.Q[q2]; s_f[threadIdx.x][14 + q2] = Cc.Qc[q2]; }
        } else {
            s_f[threadIdx.x][0] = Pp.M;
            for (int a = 0; a < 3; ++a) s_f[threadIdx.x][2 + a] = Pp.S[a];
            for (int q2 = 0; q2 < 6; ++q2) s_f[threadIdx.x][8 + q2] = Pp.Q[q2];
        }
        __syncthreads();
        for (int half = kBigThreads / 2; half > 0; half >>= 1) {
            if (threadIdx.x < half) {
                const int u = threadIdx.x, v = threadIdx.x + half;
                for (int a = 0; a < 3; ++a) {
                    s_bb[u][a] = fminf(s_bb[u][a], s_bb[v][a]);
                    s_bb[u][3 + a] = fmaxf(s_bb[u][3 + a], s_bb[v][3 + a]);
                }
                if (f64) {
                    for (int z = 0; z < 10; ++z) s_d[u][z] += s_d[v][z];
                } else if (MODE == TB_MOM_FP32_COMP) {
                    AccC A, B;
                    A.M = s_f[u][0]; A.Mc = s_f[u][1]; B.M = s_f[v][0]; B.Mc = s_f[v][1];
                    for (int a = 0; a < 3; ++a) {
                        A.S[a] = s_f[u][2 + a]; A.Sc[a] = s_f[u][5 + a];
                        B.S[a] = s_f[v][2 + a]; B.Sc[a] = s_f[v][5 + a];
                    }
                    for (int q2 = 0; q2 < 6; ++q2) {
                        A.Q[q2] = s_f[u][8 + q2]; A.Qc[q2] = s_f[u][14 + q2];
                        B.Q[q2] = s_f[v][8 + q2]; B.Qc[q2] = s_f[v][14 + q2];
                    }
                    A.merge(B);
                    s_f[u][0] = A.M; s_f[u][1] = A.Mc;
                    for (int a = 0; a < 3; ++a) { s_f[u][2 + a] = A.S[a]; s_f[u][5 + a] = A.Sc[a]; }
                    for (int q2 = 0; q2 < 6; ++q2) { s_f[u][8 + q2] = A.Q[q2]; s_f[u][14 + q2] = A.Qc[q2]; }
                } else {
                    s_f[u][0] += s_f[v][0];
                    for (int a = 0; a < 3; ++a) s_f[u][2 + a] += s_f[v][2 + a];
                    for (int q2 = 0; q2 < 6; ++q2) s_f[u][8 + q2] += s_f[v][8 + q2];
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            float bbf[6];
            for (int a = 0; a < 6; ++a) bbf[a] = s_bb[0][a];
            if (f64) {
                AccD A;
                A.M = s_d[0][0];
                for (int a = 0; a < 3; ++a) A.S[a] = s_d[0][1 + a];
                for (int q2 = 0; q2 < 6; ++q2) A.Q[q2] = s_d[0][4 + q2];
                finish_d(o, c, A, ref, bbf, MODE == TB_MOM_FP64);
            } else if (MODE == TB_MOM_FP32_COMP) {
                AccC A;
                A.M = s_f[0][0]; A.Mc = s_f[0][1];
                for (int a = 0; a < 3; ++a) { A.S[a] = s_f[0][2 + a]; A.Sc[a] = s_f[0][5 + a]; }
                for (int q2 = 0; q2 < 6; ++q2) { A.Q[q2] = s_f[0][8 + q2]; A.Qc[q2] = s_f[0][14 + q2]; }
                finish_c(o, c, A, ref, bbf);
            } else {
                AccP A;
                A.M = s_f[0][0];
                for (int a = 0; a < 3; ++a) A.S[a] = s_f[0][2 + a];
                for (int q2 = 0; q2 < 6; ++q2) A.Q[q2] = s_f[0][8 + q2];
                finish_p(o, c, A, ref, bbf);
            }
        }
        __syncthreads();
    }
}

__global__ void wait_selftest_kernel(int64_t limit, uint32_t *status, const uint32_t *flag) {
    int64_t iter = 0;
    while (*(volatile const uint32_t *)flag == 0u) {
        if (!poll_backoff(iter, limit)) {
            flag_error(status, kErrTimeout);
            return;
        }
    }
}

template <int MODE>
cudaError_t moments_impl(tb_tree &t, Workspace &ws, cudaStream_t s) {
    TreeIn T{t.child_first, t.child_end, t.pfirst, t.pend, ws.big_leaf, t.parent};
    MomOut o{t.mass, t.com, t.com_lo, t.quad, t.aabb, t.mass64, t.com64, t.quad64};
    const int64_t n = t.n_particles;
    // misc_ctr[2..3]: big-leaf queue and tickets; [5]: long-leaf queue
    cudaError_t e = cudaMemsetAsync(&ws.info->misc_ctr[2], 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        cudaFuncSetAttribute(leaf_tile_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)leaf_tile_smem());
        cudaFuncSetAttribute(leaf_tile_kernel<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(level_moments_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(LevelSmem));
        cudaFuncSetAttribute(level_moments_kernel<MODE>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    // the long-leaf queue (at most n / 2 leaves of two or more members past
    // the first) sits in the upper half of the big-leaf buffer (at most
    // n / 2049 entries in the lower)
    int32_t *longq = ws.big_leaf + (n + 1) / 2;
    const int64_t tiles = (n + kLtTile - 1) / kLtTile;
    const int64_t level_tiles = (n + level_tile_size() - 1) / level_tile_size();
    const uint32_t *leaf_off = ws.level_cnt + (int64_t)kLevels * level_tiles;
    leaf_tile_kernel<MODE><<<(unsigned)tiles, kLtThreads, leaf_tile_smem(), s>>>(
        o, t.leaf_cell, t.perm, ws.xm, ws.ml, leaf_off, n,
        t.pos_sorted ? reinterpret_cast<float4 *>(t.pos_sorted) : nullptr, longq, ws.info,
        g_wait_limit);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const PermSrc src{ws.xm, t.perm};
    long_leaf_kernel<MODE><<<152 * 2, kMomThreads, 0, s>>>(T, o, src, longq, ws.info);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    big_leaf_kernel<MODE><<<152, kBigThreads, 0, s>>>(T, o, src, ws.info);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(ws, "leaves", s);
    // one persistent grid per launch: five blocks per SM, never more than
    // the tiles a level of at most n cells can have
    int64_t grid = (n + kLmTile - 1) / kLmTile;
    if (grid > 152 * 5) grid = 152 * 5;
    if (grid < 1) grid = 1;
    for (int d = kDepthMax - 1; d >= 0; --d) {
        level_moments_kernel<MODE><<<(unsigned)grid, kLmThreads, sizeof(LevelSmem), s>>>(
            T, o, ws.info, d, g_wait_limit);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(ws, "moments", s);
    return cudaSuccess;
}

// xs[k] = xm[perm[k]]: the particles in key order, for the tree walk when
// the moments did not write them; every thread keeps four gathers in flight.
__global__ void __launch_bounds__(256)
    gather_records_kernel(const int32_t *__restrict__ perm, const float4 *__restrict__ xm,
                          float4 *__restrict__ xs, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n / 4;
    const int4 *p4 = reinterpret_cast<const int4 *>(perm);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n4; g += stride) {
        const int4 id = __ldcs(p4 + g);
        const float4 a = __ldg(xm + id.x), b = __ldg(xm + id.y), c = __ldg(xm + id.z),
                     d = __ldg(xm + id.w);
        xs[4 * g] = a;
        xs[4 * g + 1] = b;
        xs[4 * g + 2] = c;
        xs[4 * g + 3] = d;
    }
    for (int64_t k = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride)
        xs[k] = __ldg(xm + perm[k]);
}

}  // namespace

cudaError_t launch_gather_records(const int32_t *perm, const float4 *xm, float4 *xs, int64_t n,
                                  cudaStream_t s) {
    int64_t g = (n / 4 + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    gather_records_kernel<<<(unsigned)g, 256, 0, s>>>(perm, xm, xs, n);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_moments(tb_tree &t, Workspace &ws, int mode, cudaStream_t s) {
    switch (mode) {
        case TB_MOM_FP32_COMP: return moments_impl<TB_MOM_FP32_COMP>(t, ws, s);
        case TB_MOM_FP32_PLAIN: return moments_impl<TB_MOM_FP32_PLAIN>(t, ws, s);
        case TB_MOM_FP64: return moments_impl<TB_MOM_FP64>(t, ws, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wait_selftest(int64_t limit, uint32_t *status, uint32_t *flag, cudaStream_t s) {
    wait_selftest_kernel<<<1, 1, 0, s>>>(limit, status, flag);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace tb
