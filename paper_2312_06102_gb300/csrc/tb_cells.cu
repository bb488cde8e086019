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
// level, so the index of cell (d, k) is level_offset[d] plus the number of
// level-d starts before k: a 22-way prefix count, done in three launches:
//   level_count_kernel : per tile of particles, the number of cells started at
//                        each level and the number of leaves started;
//   level_scan_kernel  : per level, prefix over tiles; the last block forms the
//                        level offsets, the cell count and the depth;
//   emit_kernel        : re-derives m and L, and writes every cell.
// Links follow from the same counts:
//   parent of (d, k)       = the level-(d-1) cell holding k: index P[d-1] - 1
//                            once k's own shallower cells are counted;
//   child_first of (d, k)  = (d+1, k) when d < L_k: index P[d+1];
//   pend, child_end        = written by the leaf start k' that closes the cell:
//                            k' closes levels m_k' .. L_{k'-1} (the cells holding
//                            k'-1 but not k'); the last particle closes all.
// No cell is written twice and no pass over the cells is needed afterwards.
#include "tb_device.cuh"

namespace tb {

namespace {

constexpr int kLvThreads = 256;
constexpr int kLvItems = 16;
constexpr int kLvTile = kLvThreads * kLvItems;

// Shared-memory layout of one level tile.
struct LvSmem {
    uint64_t *key;   // keys of [s - n - 1, e + n)
    uint8_t *c;      // c_i over [s - n - 1, e)
    uint8_t *pm;     // prefix max within blocks of n + 1
    uint8_t *sm;     // suffix max within blocks of n + 1
    uint8_t *L;      // L_k over [s - 1, e)        (index k - s + 1)
    uint8_t *m;      // m_k over [s, e)            (index k - s), padded to kLvTile
};

__host__ __device__ inline size_t lv_smem_bytes(int ncrit) {
    size_t ext = (size_t)kLvTile + 2 * (size_t)ncrit + 1;
    size_t b = (ext * 8 + 15) & ~size_t(15);   // keys, padded to 16 bytes
    b += 3 * ((ext + 15) & ~size_t(15));       // c, pm, sm
    b += (kLvTile + 16) + kLvTile;       // L, m
    return b + 64;
}

__device__ inline LvSmem lv_carve(unsigned char *raw, int ncrit) {
    size_t ext = (size_t)kLvTile + 2 * (size_t)ncrit + 1;
    size_t extp = (ext + 15) & ~size_t(15);
    LvSmem s;
    s.key = reinterpret_cast<uint64_t *>(raw);
    unsigned char *p = raw + ((ext * 8 + 15) & ~size_t(15));   // every region 16-byte aligned
    s.c = p; p += extp;
    s.pm = p; p += extp;
    s.sm = p; p += extp;
    s.L = p; p += kLvTile + 16;
    s.m = p;
    return s;
}

// m and L for every particle of the tile [s, e) (plus L of s - 1), into
// shared memory.  Out-of-range neighbours contribute nothing.
__device__ void tile_levels(const uint64_t *__restrict__ skeys, int64_t n, int ncrit, int64_t s,
                            int64_t e, const LvSmem &sm) {
    const int64_t ext_lo = s - ncrit - 1;
    const int next = (int)(e + ncrit - ext_lo);     // keys held
    const int nc = (int)(e - ext_lo);               // c values held
    for (int x = threadIdx.x; x < next; x += blockDim.x) {
        int64_t i = ext_lo + x;
        sm.key[x] = (i >= 0 && i < n) ? skeys[i] : 0ull;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < nc; x += blockDim.x) {
        int64_t i = ext_lo + x;
        int v = 0;
        if (i >= 0 && i + ncrit < n) v = min(kDepthMax, min_depth(sm.key[x], sm.key[x + ncrit]));
        sm.c[x] = (uint8_t)v;
    }
    __syncthreads();
    // running max inside consecutive blocks of w = n + 1 c-values
    const int w = ncrit + 1;
    const int nblk = (nc + w - 1) / w;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        int lo = b * w, hi = min(nc, lo + w);
        uint8_t run = 0;
        for (int x = lo; x < hi; ++x) { run = max(run, sm.c[x]); sm.pm[x] = run; }
        run = 0;
        for (int x = hi - 1; x >= lo; --x) { run = max(run, sm.c[x]); sm.sm[x] = run; }
    }
    __syncthreads();
    // L_i = max(c over [i-n, i]) = max(suffix max at i-n, prefix max at i)
    const int nL = (int)(e - s + 1);
    for (int y = threadIdx.x; y < kLvTile + 16; y += blockDim.x) {
        if (y < nL) {
            int x1 = y + ncrit;          // i - ext_lo for i = s - 1 + y
            int x0 = y;                  // (i - n) - ext_lo
            sm.L[y] = max(sm.sm[x0], sm.pm[x1]);
        } else {
            sm.L[y] = 0;                 // beyond the tile: with m = 255 starts nothing
        }
    }
    const int nm = (int)(e - s);
    for (int y = threadIdx.x; y < kLvTile; y += blockDim.x) {
        uint8_t v = 0;
        if (y < nm) {
            int64_t k = s + y;
            int x = (int)(k - ext_lo);
            v = (k == 0) ? 0 : (uint8_t)min_depth(sm.key[x - 1], sm.key[x]);
        } else {
            v = 255;   // beyond the tile: starts nothing
        }
        sm.m[y] = v;
    }
    __syncthreads();
}

// Per-thread counts of cell starts per level (fields 0..21) and leaf starts
// (field 22), 5 bits per field (a thread owns 16 particles), packed in two
// 64-bit words.
struct Packed {
    uint64_t a, b;
    __device__ void add(int f) {
        if (f < 12) a += 1ull << (5 * f);
        else b += 1ull << (5 * (f - 12));
    }
    __device__ uint32_t get(int f) const {
        return f < 12 ? (uint32_t)((a >> (5 * f)) & 31u) : (uint32_t)((b >> (5 * (f - 12))) & 31u);
    }
};

__device__ inline void load_items(const LvSmem &sm, uint8_t (&mm)[kLvItems], uint8_t (&LL)[kLvItems],
                                  uint8_t &Lprev) {
    const int y0 = threadIdx.x * kLvItems;
    uint4 mv = *reinterpret_cast<const uint4 *>(sm.m + y0);
    // L is stored from s - 1: L[y0 + 1 + j] is the item j, L[y0] the one before
    uint8_t lraw[kLvItems + 1];
#pragma unroll
    for (int j = 0; j <= kLvItems; ++j) lraw[j] = sm.L[y0 + j];
    const uint8_t *mb = reinterpret_cast<const uint8_t *>(&mv);
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) { mm[j] = mb[j]; LL[j] = lraw[j + 1]; }
    Lprev = lraw[0];
}

__global__ void __launch_bounds__(kLvThreads)
    level_count_kernel(const uint64_t *__restrict__ skeys, int64_t n, int ncrit,
                       uint32_t *__restrict__ tile_cnt, int64_t n_tiles) {
    extern __shared__ __align__(16) unsigned char raw[];
    LvSmem sm = lv_carve(raw, ncrit);
    const int64_t t = blockIdx.x;
    const int64_t s = t * kLvTile, e = min64(n, s + kLvTile);
    tile_levels(skeys, n, ncrit, s, e, sm);
    uint8_t mm[kLvItems], LL[kLvItems], Lp;
    load_items(sm, mm, LL, Lp);
    Packed pc{0, 0};
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
        int m = mm[j], L = LL[j];
        for (int d = m; d <= L; ++d) pc.add(d);
        if (m <= L) pc.add(kLevels);
    }
    // block sums of the 23 fields
    __shared__ uint32_t s_tot[kLevelFields];
    if (threadIdx.x < kLevelFields) s_tot[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int f = 0; f < kLevelFields; ++f) {
        uint32_t v = pc.get(f);
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_tot[f], v);
    }
    __syncthreads();
    if (threadIdx.x < kLevelFields) tile_cnt[(int64_t)threadIdx.x * n_tiles + t] = s_tot[threadIdx.x];
}

// One block per field: exclusive prefix over tiles (in place); the last block
// to finish turns the field totals into level offsets.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
    level_scan_kernel(uint32_t *tile_cnt, int64_t n_tiles, DevInfo *info, int64_t cell_cap) {
    const int f = blockIdx.x;
    uint32_t *row = tile_cnt + (int64_t)f * n_tiles;
    const int64_t per = (n_tiles + kScanThreads - 1) / kScanThreads;
    const int64_t lo = threadIdx.x * per, hi = min64(n_tiles, lo + per);
    uint64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += row[i];
    // block exclusive scan of `sum`
    __shared__ uint64_t s_w[kScanThreads / 32];
    __shared__ uint64_t s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = sum;
    for (int off = 1; off < 32; off <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t r = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) { uint64_t v = s_w[w]; s_w[w] = r; r += v; }
        s_total = r;
    }
    __syncthreads();
    uint64_t run = s_w[warp] + x - sum;
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t v = row[i];
        row[i] = (uint32_t)run;
        run += v;
    }
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

struct EmitOut {
    uint64_t *ckey;
    uint8_t *level;
    int32_t *parent, *child_first, *child_end, *pfirst, *pend;
    int32_t *leaf_cell;
};

__global__ void __launch_bounds__(kLvThreads)
    emit_kernel(const uint64_t *__restrict__ skeys, int64_t n, int ncrit,
                const uint32_t *__restrict__ tile_off, int64_t n_tiles, const DevInfo *info,
                EmitOut out) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    extern __shared__ __align__(16) unsigned char raw[];
    LvSmem sm = lv_carve(raw, ncrit);
    // P[f][thread]: running start counts, laid out field-major (no bank conflicts)
    __shared__ uint32_t s_P[kLevelFields][kLvThreads];
    __shared__ uint32_t s_wsum[kLvThreads / 32][kLevelFields];
    const int64_t t = blockIdx.x;
    const int64_t s = t * kLvTile, e = min64(n, s + kLvTile);
    tile_levels(skeys, n, ncrit, s, e, sm);
    uint8_t mm[kLvItems], LL[kLvItems], Lp;
    load_items(sm, mm, LL, Lp);
    Packed pc{0, 0};
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
        int m = mm[j], L = LL[j];
        for (int d = m; d <= L; ++d) pc.add(d);
        if (m <= L) pc.add(kLevels);
    }
    // exclusive scan over threads of every field
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl[kLevelFields];
#pragma unroll
    for (int f = 0; f < kLevelFields; ++f) {
        uint32_t v = pc.get(f), x = v;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        incl[f] = x - v;   // exclusive within the warp
        if (lane == 31) s_wsum[warp][f] = x;
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < kLevelFields; ++f) {
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w][f];
        uint32_t base = (f < kLevels) ? (uint32_t)info->level_offset[f] : 0u;
        s_P[f][threadIdx.x] = base + tile_off[(int64_t)f * n_tiles + t] + wpre + incl[f];
    }
    __syncthreads();

    const int64_t k0 = s + (int64_t)threadIdx.x * kLvItems;
    const uint64_t *keyp = sm.key + (k0 - (s - ncrit - 1));
#pragma unroll 1
    for (int j = 0; j < kLvItems; ++j) {
        const int64_t k = k0 + j;
        if (k >= e) break;
        const int m = mm[j], L = LL[j];
        const int Lprev = (j == 0) ? Lp : LL[j - 1];
        // close the cells holding k-1 but not k
        if (k > 0) {
            for (int d = m; d <= Lprev; ++d) {
                int32_t idx = (int32_t)s_P[d][threadIdx.x] - 1;
                out.pend[idx] = (int32_t)k;
                out.child_end[idx] = (d < Lprev) ? (int32_t)s_P[d + 1][threadIdx.x] : -1;
            }
        }
        // open k's cells, shallowest first
        if (m <= L) {
            const uint64_t K = keyp[j];
            for (int d = m; d <= L; ++d) {
                int32_t idx = (int32_t)s_P[d][threadIdx.x];
                out.ckey[idx] = cell_key(K, d);
                out.level[idx] = (uint8_t)d;
                out.pfirst[idx] = (int32_t)k;
                out.parent[idx] = (d == 0) ? -1 : (int32_t)s_P[d - 1][threadIdx.x] - 1;
                out.child_first[idx] = (d < L) ? (int32_t)s_P[d + 1][threadIdx.x] : -1;
                s_P[d][threadIdx.x] = (uint32_t)idx + 1;
            }
            uint32_t leaf = s_P[kLevels][threadIdx.x];
            out.leaf_cell[leaf] = (int32_t)s_P[L][threadIdx.x] - 1;
            s_P[kLevels][threadIdx.x] = leaf + 1;
        }
        if (k == n - 1) {
            for (int d = 0; d <= L; ++d) {
                int32_t idx = (int32_t)s_P[d][threadIdx.x] - 1;
                out.pend[idx] = (int32_t)n;
                out.child_end[idx] = (d < L) ? (int32_t)s_P[d + 1][threadIdx.x] : -1;
            }
        }
    }
}

}  // namespace

int level_tile_size() { return kLvTile; }

cudaError_t launch_levels(const uint64_t *skeys, int64_t n, int ncrit, Workspace &ws,
                          cudaStream_t s) {
    const int64_t tiles = (n + kLvTile - 1) / kLvTile;
    const size_t smem = lv_smem_bytes(ncrit);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(level_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lv_smem_bytes(kMaxNcrit));
        cudaFuncSetAttribute(emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lv_smem_bytes(kMaxNcrit));
        attr = true;
    }
    level_count_kernel<<<(unsigned)tiles, kLvThreads, smem, s>>>(skeys, n, ncrit, ws.level_cnt,
                                                                 tiles);
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
    const int64_t tiles = (n + kLvTile - 1) / kLvTile;
    const size_t smem = lv_smem_bytes(ncrit);
    EmitOut o{t.ckey, t.level, t.parent, t.child_first, t.child_end, t.pfirst, t.pend,
              t.leaf_cell};
    emit_kernel<<<(unsigned)tiles, kLvThreads, smem, s>>>(skeys, n, ncrit, ws.level_cnt, tiles,
                                                          ws.info, o);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace tb
