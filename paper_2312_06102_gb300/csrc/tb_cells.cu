// tb_cells.cu -- leaves and the remaining cells from the sorted keys
// (Sec. 2.3.1 Alg. 1, Sec. 2.3.2 Alg. 2, App. A), data-parallel.
//
// For sorted keys K and n = n_crit:
//   m_k = minDepth(k-1, k)  (m_0 = 0)                  -- where k leaves its predecessor's cells
//   c_i = min(21, minDepth(i, i+n)) for i+n < N, else 0 -- window [i, i+n] lies in a cell of
//                                                          depth < c_i, which then holds > n
//   L_k = max{ c_i : k-n <= i <= k }                    -- depth of the leaf holding k
// A depth-D cell holding k has more than n particles iff some window
// [i, i+n] containing k lies inside it, so L_k is the first depth at which
// k's cell holds n or fewer (or 21), which at a leaf start equals the
// D_k = max(minDepth(k-1,k), minDepth(k,k+n)) of App. A.  Particle k starts a
// cell at every depth d with m_k <= d <= L_k, and k starts a leaf iff
// m_k <= L_k.  Every cell is therefore (d, K_k >> (63 - 3d), first particle
// k) for exactly one k, which replaces the serial scans of Alg. 1 and the
// per-depth merges of Alg. 2 by one pass over the particles.
//
// Canonical order is level-major, key (= first particle) ascending within a
// level, so the index of cell (d, k) is level_offset[d] + P_d(k), P_d(k) the
// number of level-d starts before k: a 22-way prefix count, done in three
// launches over tiles of 1024 particles:
//   level_count_kernel : per tile, the cells started at each level and the
//                        leaves started (one warp ballot per level);
//   level_scan_kernel  : per level, prefix over tiles; the last block forms the
//                        level offsets, the cell count and the depth;
//   emit_starts_kernel : reads m and L back, lists the leaf starts, and writes
//                        every cell.
// Links follow from the same counts (P_d(k) before k's own starts):
//   index of (d, k)        = P_d(k);
//   parent of (d, k)       = (d-1, k) = P_{d-1}(k) if d > m_k, else the level-(d-1)
//                            cell holding k, started earlier: P_{d-1}(k) - 1;
//   child_first of (d, k)  = (d+1, k) = P_{d+1}(k) when d < L_k;
//   pend, child_end        = written by the leaf start k' that closes the cell:
//                            k' closes levels m_k' .. L_{k'-1} (the cells holding
//                            k'-1 but not k'), cell P_d(k') - 1, child_end
//                            P_{d+1}(k'); the last particle closes all.
// No cell is written twice and no pass over the cells is needed afterwards.
// L_k, a maximum over a window of n + 1 values of c, comes from a doubling
// table: M_1 = c, M_2q[i] = max(M_q[i], M_q[i+q]); with p the largest power of
// two <= n + 1, L_k = max(M_p[k-n], M_p[k-p+1]).
#include "tb_cells.cuh"

namespace tb {

namespace {

__global__ void __launch_bounds__(kLvThreads, 2)
    level_count_kernel(const uint64_t *__restrict__ skeys, int64_t n, int ncrit,
                       uint32_t *__restrict__ tile_cnt, int64_t n_tiles, uint16_t *__restrict__ ml) {
    extern __shared__ __align__(16) unsigned char raw[];
    __shared__ TileShared ts;
    __shared__ uint32_t tot[kLevelFields];
    const int64_t t = blockIdx.x;
    const int64_t s = t * kLvTile, e = min64(n, s + kLvTile);
    const Front f = tile_front(skeys, 0, n, ncrit, s, e, raw, ts);
    // keep m and L of every particle for the emission
    if (f.k < e) ml[f.k] = (uint16_t)(f.m | (f.L << 8));
    warp_field_prefix(ts, nullptr, tot);
    __syncthreads();
    if (threadIdx.x < kLevelFields) tile_cnt[(int64_t)threadIdx.x * n_tiles + t] = tot[threadIdx.x];
}

// The same counts, four consecutive particles per thread, for n_crit in
// [kLcMinN, kLcMaxN].  A block of 256 threads takes one count tile.  c is kept one byte per
// position; the window maxima of four neighbours share all but their ends:
// L_{k0+j} = max(suffix max from byte j of c[k0-n .. k0-n+3],
//                max of c[k0-n+4 .. k0-1],
//                prefix max to byte j of c[k0 .. k0+3]),
// taken four bytes at a time (byte-wise SIMD maxima).  The per-level counts
// come from histograms of m and of L + 1 over the leaf starts:
// #cells started at level d = #{m <= d} - #{L + 1 <= d}.
constexpr int kLcThreads = 256;
constexpr int kLcPer = 4;
constexpr int kLcSub = 1;                               // count tiles per block
constexpr int kLcTile = kLvTile * kLcSub;
constexpr int kLcMinN = 3, kLcMaxN = 60;

__host__ __device__ inline int lc_halo_words(int ncrit) { return (ncrit + 3) / 4 + 1; }
__host__ __device__ inline size_t lc_smem_bytes(int ncrit) {
    const size_t nk = (size_t)kLcTile + 4 * lc_halo_words(ncrit) + ncrit + 4;   // keys
    const size_t nw = (size_t)kLcTile / 4 + lc_halo_words(ncrit) + 2;          // c words
    return nk * 8 + nw * 4;
}

__global__ void __launch_bounds__(kLcThreads, 6)
    level_count_fast_kernel(const uint64_t *__restrict__ skeys, int64_t n, int ncrit,
                            uint32_t *__restrict__ tile_cnt, int64_t n_tiles,
                            uint16_t *__restrict__ ml) {
    extern __shared__ __align__(16) unsigned char raw[];
    __shared__ uint32_t hist_m[kLcSub][kLevels + 1];    // leaf starts by m
    __shared__ uint32_t hist_l[kLcSub][kLevels + 1];    // leaf starts by L + 1
    const int H = lc_halo_words(ncrit);
    const int64_t s = (int64_t)blockIdx.x * kLcTile, e = min64(n, s + kLcTile);
    const int64_t base = s - 4 * H;                     // position of key[0] and of c byte 0
    const int nk = (int)(e + ncrit - base);
    const int nw = (int)((e - base + 3) / 4);
    uint64_t *key = reinterpret_cast<uint64_t *>(raw);
    uint32_t *cw = reinterpret_cast<uint32_t *>(raw + ((size_t)kLcTile + 4 * H + ncrit + 4) * 8);
    // a block away from both ends of the array needs no bounds checks: every
    // window [i, i + n] of its span exists and the keys load as 16-byte pairs
    // (base is even, so key + base is 16-byte aligned)
    const bool interior = base >= 0 && e == s + kLcTile && e + ncrit + 1 <= n;
    if (interior) {
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(skeys + base);
        ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(key);
        for (int x = threadIdx.x; 2 * x < nk; x += kLcThreads) dst[x] = src[x];
    } else {
        for (int x = threadIdx.x; x < nk; x += kLcThreads) {
            const int64_t i = base + x;
            key[x] = (i >= 0 && i < n) ? skeys[i] : 0ull;
        }
    }
    for (int x = threadIdx.x; x < kLcSub * (kLevels + 1); x += kLcThreads) {
        (&hist_m[0][0])[x] = 0;
        (&hist_l[0][0])[x] = 0;
    }
    __syncthreads();
    // c of four positions per word: min(21, minDepth(i, i+n)) where the
    // window exists, else 0
    for (int w = threadIdx.x; w < nw; w += kLcThreads) {
        uint32_t v = 0;
        if (interior) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = 4 * w + j;
                v |= (uint32_t)min(kDepthMax, min_depth(key[x], key[x + ncrit])) << (8 * j);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = 4 * w + j;
                const int64_t i = base + x;
                if (i >= 0 && i + ncrit < n && i < e)
                    v |= (uint32_t)min(kDepthMax, min_depth(key[x], key[x + ncrit])) << (8 * j);
            }
        }
        cw[w] = v;
    }
    __syncthreads();
    const int64_t k0 = s + kLcPer * threadIdx.x;
    uint32_t Lw = 0, mw = 0xffffffffu;                  // bytes: L and m of k0 .. k0 + 3
    if (k0 < e) {
        const int x0 = (int)(k0 - base);                // multiple of 4
        const uint32_t T = cw[x0 >> 2];
        auto bytes4 = [&](int b) {                      // c bytes b .. b + 3 (b >= 0)
            const int w = b >> 2, sh = (b & 3) * 8;
            return sh ? __funnelshift_r(cw[w], cw[w + 1], sh) : cw[w];
        };
        const uint32_t Hw = bytes4(x0 - ncrit);
        uint32_t I = 0;
        const int mlen = ncrit - 4;                     // middle bytes x0 - n + 4 .. x0 - 1
        if (mlen >= 4) {
            for (int b = x0 - ncrit + 4; b + 4 <= x0; b += 4) I = __vmaxu4(I, bytes4(b));
            I = __vmaxu4(I, bytes4(x0 - 4));
        } else if (mlen > 0) {
            I = bytes4(x0 - ncrit + 4) & ((1u << (8 * mlen)) - 1u);
        }
        I = __vmaxu4(I, I >> 16);
        I = __vmaxu4(I, I >> 8);
        I = (I & 0xffu) * 0x01010101u;
        uint32_t S = __vmaxu4(Hw, Hw >> 8);
        S = __vmaxu4(S, S >> 16);
        uint32_t P = __vmaxu4(T, T << 8);
        P = __vmaxu4(P, P << 16);
        Lw = __vmaxu4(__vmaxu4(S, P), I);
        mw = 0;
        if (interior) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                mw |= (uint32_t)min_depth(key[x0 + j - 1], key[x0 + j]) << (8 * j);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t k = k0 + j;
                uint32_t m = 255u;
                if (k < e) m = (k == 0) ? 0u : (uint32_t)min_depth(key[x0 + j - 1], key[x0 + j]);
                mw |= m << (8 * j);
            }
        }
        // m and L of the four particles, for the emission
        if (k0 + 4 <= e) {
            uint2 v;
            v.x = (mw & 0xffu) | ((Lw & 0xffu) << 8) | (((mw >> 8) & 0xffu) << 16) | (((Lw >> 8) & 0xffu) << 24);
            v.y = ((mw >> 16) & 0xffu) | (((Lw >> 16) & 0xffu) << 8) | ((mw >> 24) << 16) | ((Lw >> 24) << 24);
            *reinterpret_cast<uint2 *>(ml + k0) = v;
        } else {
            for (int j = 0; j < 4 && k0 + j < e; ++j)
                ml[k0 + j] = (uint16_t)(((mw >> (8 * j)) & 0xffu) | (((Lw >> (8 * j)) & 0xffu) << 8));
        }
    }
    // histograms of m and L + 1 over the leaf starts (m <= L): about one
    // particle in seven is a start, so plain shared atomics rarely collide
    const int sub = (int)(kLcPer * threadIdx.x / kLvTile);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = (mw >> (8 * j)) & 0xff, L = (Lw >> (8 * j)) & 0xff;
        if (m <= L) {
            atomicAdd(&hist_m[sub][m], 1u);
            atomicAdd(&hist_l[sub][L + 1], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < kLcSub * kLevelFields) {
        const int sb = threadIdx.x / kLevelFields, f = threadIdx.x % kLevelFields;
        const int64_t t = (int64_t)blockIdx.x * kLcSub + sb;
        if (t < n_tiles) {
            uint32_t v = 0;
            if (f == kLevels) {
                for (int d = 0; d < kLevels; ++d) v += hist_m[sb][d];
            } else {
                for (int d = 0; d <= f; ++d) v += hist_m[sb][d] - hist_l[sb][d];
            }
            tile_cnt[(int64_t)f * n_tiles + t] = v;
        }
    }
}

// One block per field: exclusive prefix over tiles (in place); the last block
// to finish turns the field totals into level offsets.  The row is taken in
// chunks staged in shared memory (coalesced loads and stores), each thread
// scanning a contiguous stretch of a chunk.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr int kScanChunk = kScanThreads * kScanPer;
static_assert(kScanPer == 8, "the scan moves each thread's eight counts as two uint4");

__global__ void __launch_bounds__(kScanThreads)
    level_scan_kernel(uint32_t *tile_cnt, int64_t n_tiles, DevInfo *info, int64_t cell_cap) {
    const int f = blockIdx.x;
    uint32_t *row = tile_cnt + (int64_t)f * n_tiles;
    __shared__ __align__(16) uint32_t s_v[kScanChunk];
    __shared__ uint32_t s_w[kScanThreads / 32];
    __shared__ uint64_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    for (int64_t c0 = 0; c0 < n_tiles; c0 += kScanChunk) {
        const int len = (int)min64(kScanChunk, n_tiles - c0);
        for (int i = threadIdx.x; i < kScanChunk; i += kScanThreads) s_v[i] = i < len ? row[c0 + i] : 0u;
        __syncthreads();
        uint32_t v[kScanPer], sum = 0;
        {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(s_v) + 2 * threadIdx.x;
            const uint4 a = s4[0], b = s4[1];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        }
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) sum += v[j];
        uint32_t x = sum;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_w[lane];
            uint32_t z = w;
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, off);
                if (lane >= off) z += y;
            }
            s_w[lane] = z - w;
        }
        __syncthreads();
        // the per-field counts fit 32 bits (at most 2^31 particles)
        uint32_t run = (uint32_t)s_carry + s_w[warp] + x - sum;
        uint32_t o[kScanPer];
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) { o[j] = run; run += v[j]; }
        {
            uint4 *s4 = reinterpret_cast<uint4 *>(s_v) + 2 * threadIdx.x;
            s4[0] = make_uint4(o[0], o[1], o[2], o[3]);
            s4[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += kScanThreads) row[c0 + i] = s_v[i];
        if (threadIdx.x == kScanThreads - 1) s_carry = run;
        __syncthreads();
    }
    const uint64_t s_total = s_carry;
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        // totals land in a small array right after the per-tile rows
        tile_cnt[(int64_t)kLevelFields * n_tiles + f] = (uint32_t)s_total;
        __threadfence();
        s_last = (atomicAdd(&info->misc_ctr[1], 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    const uint32_t *tot = tile_cnt + (int64_t)kLevelFields * n_tiles;
    int64_t off = 0;
    int dmax = 0;
    for (int d = 0; d < kLevels; ++d) {
        uint32_t c = __ldcg(&tot[d]);
        info->level_offset[d] = off;
        off += c;
        if (c) dmax = d;
    }
    info->level_offset[kLevels] = off;
    info->n_cells = off;
    info->n_leaves = __ldcg(&tot[kLevels]);
    info->max_depth = dmax;
    if (cell_cap > 0 && off > cell_cap) info->status |= kErrOverflow;
    info->misc_ctr[1] = 0;
}

// Emission over the leaf starts only, one count tile (1024 particles) per
// block of 256 threads, four blocks per SM.  Only a leaf start (m_k <= L_k)
// opens or closes cells, one particle in four to seven on the tree
// workloads, so the block first lists them in order in shared memory
// (four particles per thread, a block-wide prefix of the counts) and then
// runs the per-level prefix and the writes over that list, 32 starts per
// warp: every lane holds a start, and the level masks are built for the
// list, not for every particle.  The tree's last particle, which closes every
// cell that holds it, is handled by its own thread: those are the last cells
// of their levels.
constexpr int kEfThreads = 256;
constexpr int kEfWarps = kEfThreads / 32;
static_assert(kEfWarps <= 32, "one warp scans the warps' counts");
constexpr int kEfTile = 4 * kEfThreads;                // four particles per thread
static_assert(kEfTile % kLvTile == 0 && kEfTile <= 2048, "whole count tiles; offsets fit 11 bits");
constexpr int kEfChunks = kEfTile / 32;

__global__ void __launch_bounds__(kEfThreads, 4)
    emit_starts_kernel(const uint64_t *__restrict__ skeys, const uint16_t *__restrict__ ml, int64_t n,
                       const uint32_t *__restrict__ tile_off, int64_t n_tiles, DevInfo *info_w,
                       EmitOut out) {
    const DevInfo *info = info_w;
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    __shared__ uint32_t s_entry[kEfTile];               // k - s | m << 11 | L << 16 | Lprev << 21
    __shared__ uint32_t s_mask[kEfChunks][kLevels];     // level masks of each chunk of 32 starts
    __shared__ uint32_t s_cpre[kEfChunks][kLevels];     // starts of each level in earlier chunks
    __shared__ uint32_t s_base[kLevelFields];           // first level-d cell (leaf) of the block
    __shared__ uint32_t s_wcnt[kEfWarps];
    __shared__ uint8_t s_Llast[kEfThreads];
    __shared__ uint32_t s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * (kEfTile / kLvTile);   // first count tile of the block
    const int64_t s = (int64_t)blockIdx.x * kEfTile, e = min64(n, s + kEfTile);
    if (threadIdx.x < kLevelFields)
        s_base[threadIdx.x] = ((threadIdx.x < kLevels) ? (uint32_t)info->level_offset[threadIdx.x] : 0u) +
                              tile_off[(int64_t)threadIdx.x * n_tiles + t0];
    // m and L of four particles per thread
    const int64_t k0 = s + 4 * (int64_t)threadIdx.x;
    uint32_t m[4], L[4];
    if (k0 + 4 <= e) {
        const uint2 v = *reinterpret_cast<const uint2 *>(ml + k0);
        m[0] = v.x & 0xffu; L[0] = (v.x >> 8) & 0xffu; m[1] = (v.x >> 16) & 0xffu; L[1] = v.x >> 24;
        m[2] = v.y & 0xffu; L[2] = (v.y >> 8) & 0xffu; m[3] = (v.y >> 16) & 0xffu; L[3] = v.y >> 24;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t v = (k0 + j < e) ? (uint32_t)ml[k0 + j] : 255u;
            m[j] = v & 0xffu;
            L[j] = (k0 + j < e) ? (v >> 8) : 0u;
        }
    }
    s_Llast[threadIdx.x] = (uint8_t)L[3];
    uint32_t Lbefore = 0;
    if (threadIdx.x == 0 && s > 0) Lbefore = (uint32_t)(ml[s - 1] >> 8);
    // the tree's last particle closes the cells holding it: the last cell of
    // each level 0 .. L, whose children end where the next level ends
    if (k0 <= n - 1 && n - 1 < k0 + 4) {
        const uint32_t Ll = L[(int)(n - 1 - k0)];
        for (int d = 0; d <= (int)Ll; ++d) {
            const int64_t idx = info->level_offset[d + 1] - 1;
            out.pend[idx] = (int32_t)n;
            out.child_end[idx] = (d < (int)Ll) ? (int32_t)info->level_offset[d + 2] : -1;
        }
    }
    __syncthreads();
    const uint32_t Lp0 = threadIdx.x > 0 ? (uint32_t)s_Llast[threadIdx.x - 1] : Lbefore;
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) cnt += (m[j] <= L[j]) ? 1u : 0u;
    uint32_t x = cnt;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_wcnt[warp] = x;
    __syncthreads();
    if (warp == 0) {
        // exclusive prefix of the warps' counts, by shuffles
        const uint32_t c = lane < kEfWarps ? s_wcnt[lane] : 0u;
        uint32_t r = c;
#pragma unroll
        for (int off = 1; off < kEfWarps; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, r, off);
            if (lane >= off) r += y;
        }
        if (lane < kEfWarps) s_wcnt[lane] = r - c;
        if (lane == kEfWarps - 1) s_total = r;
    }
    __syncthreads();
    uint32_t pos = s_wcnt[warp] + x - cnt;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (m[j] <= L[j]) {
            const uint32_t lp = j ? L[j - 1] : Lp0;
            s_entry[pos++] = (uint32_t)(4 * threadIdx.x + j) | (m[j] << 11) | (L[j] << 16) | (lp << 21);
        }
    }
    __syncthreads();
    const int total = (int)s_total;
    const int nchunks = (total + 31) / 32;
    // the keys of the warp's first chunk of starts, loaded now so that the
    // mask and prefix phases below cover their latency
    uint64_t Kfirst = 0;
    if (warp * 32 + lane < total) Kfirst = skeys[s + (s_entry[warp * 32 + lane] & 2047u)];
    // level masks of every chunk of 32 starts (a 32 x 32 bit transpose)
    for (int c = warp; c < nchunks; c += kEfWarps) {
        const int i = c * 32 + lane;
        uint32_t v = 0;
        if (i < total) {
            const uint32_t en = s_entry[i];
            const uint32_t mm = (en >> 11) & 31u, LL = (en >> 16) & 31u;
            v = (2u << LL) - (1u << mm);
        }
        uint32_t msk = 0x0000ffffu;
#pragma unroll
        for (int j = 16; j > 0; j >>= 1, msk ^= msk << j) {
            const uint32_t y = __shfl_xor_sync(0xffffffffu, v, j);
            if (lane & j) v ^= ((y >> j) ^ v) & msk;
            else v ^= (((v >> j) ^ y) & msk) << j;
        }
        if (lane < kLevels) s_mask[c][lane] = v;
    }
    __syncthreads();
    // per level, the starts in earlier chunks: a warp per level, a lane per
    // chunk, 32 chunks at a time
    for (int d = warp; d < kLevels; d += kEfWarps) {
        uint32_t carry = 0;
        for (int g = 0; g < nchunks; g += 32) {
            const int c = g + lane;
            const uint32_t v = c < nchunks ? (uint32_t)__popc(s_mask[c][d]) : 0u;
            uint32_t r = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, r, off);
                if (lane >= off) r += y;
            }
            if (c < nchunks) s_cpre[c][d] = carry + r - v;
            carry += __shfl_sync(0xffffffffu, r, 31);
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
    for (int c = warp; c < nchunks; c += kEfWarps) {
        const int i = c * 32 + lane;
        if (i >= total) continue;
        const uint32_t en = s_entry[i];
        const int64_t k = s + (en & 2047u);
        const int mm = (int)((en >> 11) & 31u), LL = (int)((en >> 16) & 31u), Lp = (int)((en >> 21) & 31u);
        auto P = [&](int d) { return s_base[d] + s_cpre[c][d] + (uint32_t)__popc(s_mask[c][d] & lt); };
        const uint64_t K = c == warp ? Kfirst : skeys[k];
        // P(d) of consecutive levels: each loop computes one new level per step
        const uint32_t pm = P(mm);
        if (k > 0) {
            // close the cells holding k-1 but not k
            uint32_t pd = pm;
            for (int d = mm; d <= Lp; ++d) {
                const uint32_t pn = d < Lp ? P(d + 1) : 0u;
                out.pend[pd - 1] = (int32_t)k;
                out.child_end[pd - 1] = (d < Lp) ? (int32_t)pn : -1;
                pd = pn;
            }
        }
        uint32_t pprev = mm > 0 ? P(mm - 1) : 0u, pd = pm;
        for (int d = mm;; ++d) {
            const uint32_t pn = d < LL ? P(d + 1) : 0u;
            out.ckey[pd] = cell_key(K, d);
            out.level[pd] = (uint8_t)d;
            out.pfirst[pd] = (int32_t)k;
            out.parent[pd] = (d == 0) ? -1 : (int32_t)pprev - (d == mm ? 1 : 0);
            out.child_first[pd] = (d < LL) ? (int32_t)pn : -1;
            if (d == LL) break;
            pprev = pd;
            pd = pn;
        }
        out.leaf_cell[s_base[kLevels] + (uint32_t)i] = (int32_t)pd;
    }
}

}  // namespace

int level_tile_size() { return kLvTile; }

cudaError_t launch_levels(const uint64_t *skeys, int64_t n, int ncrit, Workspace &ws,
                          cudaStream_t s) {
    const int64_t tiles = (n + kLvTile - 1) / kLvTile;
    const size_t smem = lv_smem_bytes(ncrit);
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        cudaFuncSetAttribute(level_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lv_smem_bytes(kMaxNcrit));
        cudaFuncSetAttribute(level_count_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    if (ncrit >= kLcMinN && ncrit <= kLcMaxN) {
        static std::atomic<uint64_t> fast_attr_done{0};
        if (first_on_device(fast_attr_done)) {
            cudaFuncSetAttribute(level_count_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)lc_smem_bytes(kLcMaxN));
            cudaFuncSetAttribute(level_count_fast_kernel,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        }
        const int64_t blocks = (n + kLcTile - 1) / kLcTile;
        level_count_fast_kernel<<<(unsigned)blocks, kLcThreads, lc_smem_bytes(ncrit), s>>>(
            skeys, n, ncrit, ws.level_cnt, tiles, ws.ml);
    } else {
        level_count_kernel<<<(unsigned)tiles, kLvThreads, smem, s>>>(skeys, n, ncrit, ws.level_cnt,
                                                                     tiles, ws.ml);
    }
    ++g_launches;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    level_scan_kernel<<<kLevelFields, kScanThreads, 0, s>>>(ws.level_cnt, tiles, ws.info,
                                                            ws.cell_cap_request);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_emit(const uint64_t *skeys, int64_t n, int ncrit, Workspace &ws, tb_tree &t,
                        cudaStream_t s) {
    (void)ncrit;
    const int64_t tiles = (n + kLvTile - 1) / kLvTile;
    EmitOut o{t.ckey, t.level, t.parent, t.child_first, t.child_end, t.pfirst, t.pend,
              t.leaf_cell};
    const int64_t blocks = (n + kEfTile - 1) / kEfTile;
    emit_starts_kernel<<<(unsigned)blocks, kEfThreads, 0, s>>>(skeys, ws.ml, n, ws.level_cnt, tiles,
                                                               ws.info, o);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace tb
