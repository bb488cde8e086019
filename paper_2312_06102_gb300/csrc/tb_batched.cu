// tb_batched.cu -- many independent trees in one call (tb_build_batched).
//
// Thousands of particle sets of uneven size each get their own tree (own
// root cube, keys, sort, cells and moments, exactly as tb_build + tb_moments
// would give for the set alone), with a fixed number of launches whatever the
// number of sets:
//   set_order_kernel    : sets ordered largest first (work-queue order);
//   batch_front_kernel  : persistent, one 1024-thread block per set taken from
//                         an atomic work queue: root cube, keys, (x, y, z, m)
//                         records and the digit histograms of every pass, then a
//                         stable LSD radix sort of the set inside the block (its
//                         tiles in order, so no look-back is needed), then the
//                         set's cell and leaf counts per level;
//   batch_scan_kernel   : cell and leaf offsets of every set (set order);
//   batch_emit_kernel   : persistent, one block per set: every cell with its
//                         links (the single-tree emission from the m_k and L_k
//                         the count stored, tile after tile with running
//                         counts), then the set's particles in key order;
//   batch_moments_kernel: persistent, one block per set: every leaf in key order,
//                         then the other cells level by level, deepest first,
//                         with a block barrier between levels.
// The paper builds disjoint subtrees on dynamically scheduled threads
// (Sec. 2.3.3); here the unit of dynamic scheduling is a whole set.
#include <cfloat>

#include "tb_cells.cuh"
#include "tb_ctasort.cuh"
#include "tb_runs.cuh"
#include "tb_moments.cuh"

namespace tb {

namespace {

// front / emit blocks: T threads, one particle per thread per cell tile;
// T = 512 (two sets per SM at a time) or 1024
constexpr int kBDefaultThreads = 512;
constexpr int kBRadixBits = kCtaRadixBits;
constexpr int kBRadix = kCtaRadix;
// the block sort orders the upper 40 key bits in five passes; the runs of
// equal upper bits are then ordered in place (tb_runs.cuh)
constexpr int kBPasses = 5;
constexpr int kBShift0 = 63 - kBPasses * kBRadixBits;
constexpr int kBMomThreads = 256;
constexpr int kBigLeafSerial = 1 << 20;       // leaves above this are summed in FP64


struct BatchArgs {
    const float *pos;
    const float *mass;
    const int64_t *off;       // [S+1]
    const int32_t *order;     // [S]
    int32_t n_sets;
    int32_t ncrit;
    uint64_t *pkey;
    int32_t *perm;
    uint64_t *kalt;
    int32_t *palt;
    float4 *xm;
    float4 *xs;
    uint16_t *ml;             // [n] m_k | L_k << 8 of each sorted particle (count -> emit)
    uint32_t *set_cnt;        // [S][kLevelFields]
    int64_t *set_cell_off;    // [S+1]
    int64_t *set_leaf_off;    // [S+1]
    double *set_root;         // [S][4]
    uint32_t *queue;          // [8] work-queue tickets [0..2], grid barrier [4..5]
    DevInfo *info;
    int32_t root_pow2;        // each set's root side forced to a power of two
};

template <int T>
__host__ __device__ inline size_t batch_front_smem(int ncrit) {
    size_t a = sizeof(CtaSortSharedT<T>), b = lv_smem_bytes<T>(ncrit);
    return (a > b ? a : b);
}

// Sets in descending size classes (floor(log2 size)), ascending index within
// a class: the largest sets are taken from the queues first.
// One block of up to 1024 threads (a multiple of 32).
__device__ void set_order_block(const int64_t *off, int32_t S, int32_t *order) {
    __shared__ uint32_t cls[34];
    if (threadIdx.x < 34) cls[threadIdx.x] = 0;
    __syncthreads();
    auto klass = [&](int s) {
        int64_t n = off[s + 1] - off[s];
        return n <= 0 ? 0 : 1 + (63 - __clzll((unsigned long long)n));   // 0 .. 32
    };
    for (int s = threadIdx.x; s < S; s += blockDim.x) atomicAdd(&cls[klass(s)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int c = 33; c >= 0; --c) { uint32_t v = cls[c]; cls[c] = run; run += v; }
    }
    __syncthreads();
    // stable within a class: chunks of 1024 sets in order; inside a chunk a
    // set's place is its class's running base, plus the sets of its class in
    // earlier warps, plus those in earlier lanes of its warp
    __shared__ uint32_t wc[32][34];
    __shared__ uint32_t tot[34];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        for (int i = threadIdx.x; i < 32 * 34; i += blockDim.x) (&wc[0][0])[i] = 0;
        __syncthreads();
        const int s = c0 + (int)threadIdx.x;
        const int c = s < S ? klass(s) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && lane == __ffs(peers) - 1) wc[warp][c] = (uint32_t)__popc(peers);
        __syncthreads();
        if (threadIdx.x < 34) {
            uint32_t r = 0;
            for (int w = 0; w < nw; ++w) { const uint32_t v = wc[w][threadIdx.x]; wc[w][threadIdx.x] = r; r += v; }
            tot[threadIdx.x] = r;
        }
        __syncthreads();
        if (c >= 0) order[cls[c] + wc[warp][c] + (uint32_t)__popc(peers & lt)] = s;
        __syncthreads();
        if (threadIdx.x < 34) cls[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) set_order_kernel(const int64_t *off, int32_t S,
                                                         int32_t *order, const DevInfo *info) {
    if (info->status & kErrInvalid) return;
    set_order_block(off, S, order);
}

__device__ __forceinline__ int take_set(uint32_t *ticket, int32_t S, int *s_q) {
    if (threadIdx.x == 0) *s_q = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int q = *s_q;
    __syncthreads();
    return q < S ? q : -1;
}

// Block-wide min / max / non-finite reduction of one set's positions.
__device__ void set_root_cube(const float *__restrict__ pos, int64_t o, int64_t ns, float *s_red,
                              uint32_t *s_bad) {
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    uint32_t bad = 0;
    for (int64_t i = o + threadIdx.x; i < o + ns; i += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const float x = pos[3 * i + a];
            bad |= !(fabsf(x) <= FLT_MAX);
            mn[a] = fminf(mn[a], x);
            mx[a] = fmaxf(mx[a], x);
        }
    for (int sh = 16; sh > 0; sh >>= 1) {
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], sh));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], sh));
        }
        bad |= __shfl_xor_sync(0xffffffffu, bad, sh);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) { s_red[warp * 6 + a] = mn[a]; s_red[warp * 6 + 3 + a] = mx[a]; }
        if (bad) atomicOr(s_bad, 1u);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = s_red[threadIdx.x];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            v = (threadIdx.x < 3) ? fminf(v, s_red[w * 6 + threadIdx.x])
                                  : fmaxf(v, s_red[w * 6 + threadIdx.x]);
        s_red[threadIdx.x] = v;   // warp 0's slots hold the result
    }
    __syncthreads();
}

// Every set from work queue 0: root cube, keys, sort, counts.  `raw` is the
// block's dynamic shared memory (batch_front_smem<T> bytes).
template <int T>
__device__ void front_sets(const BatchArgs &A, unsigned char *raw) {
    CtaSortSharedT<T> &sm = *reinterpret_cast<CtaSortSharedT<T> *>(raw);
    __shared__ TileSharedT<T> ts;
    __shared__ float s_red[(T / 32) * 6];
    __shared__ uint32_t s_bad, s_tot[kLevelFields], s_tile[kLevelFields];
    __shared__ float s_lo[3], s_shi, s_slo;
    __shared__ double s_scale;
    __shared__ bool s_exact, s_f32;
    __shared__ int s_q;
    __shared__ int s_nlong;
    __shared__ int64_t s_long[32];
    __shared__ unsigned long long s_end;
    for (;;) {
        const int q = take_set(&A.queue[0], A.n_sets, &s_q);
        if (q < 0) return;
        const int set = A.order[q];
        const int64_t o = A.off[set], ns = A.off[set + 1] - o;
        if (ns <= 0) {
            if (threadIdx.x < kLevelFields) A.set_cnt[(int64_t)set * kLevelFields + threadIdx.x] = 0;
            if (threadIdx.x < 4) A.set_root[4 * (int64_t)set + threadIdx.x] = threadIdx.x == 3 ? 1.0 : 0.0;
            continue;
        }
        // ---- root cube (Sec. 2.2), as in root_kernel
        if (threadIdx.x == 0) s_bad = 0;
        __syncthreads();
        set_root_cube(A.pos, o, ns, s_red, &s_bad);
        if (threadIdx.x == 0) {
            double L = 0.0;
            float amax = 0.f;
            for (int a = 0; a < 3; ++a) {
                s_lo[a] = s_red[a];
                const double e = __dsub_rn((double)s_red[3 + a], (double)s_red[a]);
                if (e > L) L = e;
                amax = fmaxf(amax, fmaxf(fabsf(s_red[a]), fabsf(s_red[3 + a])));
            }
            if (!(L > 0.0)) L = 1.0;
            if (A.root_pow2) L = pow2_ceil(L);
            const double scale = __ddiv_rn(2097152.0, L);
            s_scale = scale;
            s_shi = (float)scale;
            s_slo = (float)__dsub_rn(scale, (double)s_shi);
            s_exact = !(scale < 1e30 && scale > 1e-30 && amax < 1e30f);
            s_f32 = (double)s_shi == scale;
            for (int a = 0; a < 3; ++a) A.set_root[4 * (int64_t)set + a] = (double)s_lo[a];
            A.set_root[4 * (int64_t)set + 3] = L;
            if (s_bad) atomicOr(&A.info->status, kErrNonFinite);
        }
        for (int i = threadIdx.x; i < kBPasses * kBRadix; i += blockDim.x) (&sm.hist[0][0])[i] = 0;
        __syncthreads();
        // ---- keys, records and every pass's digit histogram
        {
            const float lx = s_lo[0], ly = s_lo[1], lz = s_lo[2], shi = s_shi, slo = s_slo;
            const double sc = s_scale;
            const bool ex = s_exact, f32 = s_f32;
            const float m_eq = (float)(1.0 / (double)ns);
            // unsorted keys go where pass 0 reads them: kBPasses is odd, so the
            // passes run kalt -> pkey -> ... -> pkey
            for (int64_t i = o + threadIdx.x; i < o + ns; i += blockDim.x) {
                const float x = A.pos[3 * i], y = A.pos[3 * i + 1], z = A.pos[3 * i + 2];
                const uint64_t k = morton_key(quantise(x, lx, shi, slo, sc, ex, f32),
                                              quantise(y, ly, shi, slo, sc, ex, f32),
                                              quantise(z, lz, shi, slo, sc, ex, f32));
                A.kalt[i] = k;
                A.xm[i] = make_float4(x, y, z, A.mass ? A.mass[i] : m_eq);
                for (int p = 0; p < kBPasses; ++p)
                    atomicAdd(&sm.hist[p][(k >> (kBShift0 + p * kBRadixBits)) & (kBRadix - 1)], 1u);
            }
        }
        __syncthreads();
        // ---- stable LSD sort of the set by its upper key bits (digit counts
        // taken above), then the runs of equal upper bits by the low bits
        cta_lsd_sort(A.kalt, A.palt, A.pkey, A.perm, o, ns, kBShift0, kBPasses, true, sm);
        __syncthreads();
        for (int64_t t0 = o; t0 < o + ns; t0 += kRunTile) {
            if (threadIdx.x == 0) s_nlong = 0;
            __syncthreads();
            run_tile<T>(A.pkey, A.perm, o, t0, o + ns, kBShift0, *reinterpret_cast<RunSmem *>(raw),
                                [&](int64_t a) { s_long[atomicAdd(&s_nlong, 1)] = a; });
            const int nl = s_nlong;
            for (int j = 0; j < nl; ++j) {
                // a run of more than kRunMax keys (at most 16 start in a tile):
                // its end, then the block sort of its low bits
                const int64_t a = s_long[j];
                const uint64_t tp = A.pkey[a] >> kBShift0;
                if (threadIdx.x == 0) s_end = (unsigned long long)(o + ns);
                __syncthreads();
                for (int64_t base = a + 1; base < o + ns; base += blockDim.x) {
                    const int64_t p = base + threadIdx.x;
                    if (p < o + ns && (A.pkey[p] >> kBShift0) != tp) atomicMin(&s_end, (unsigned long long)p);
                    __syncthreads();
                    const bool done = s_end < (unsigned long long)(o + ns);
                    __syncthreads();
                    if (done) break;
                }
                const int64_t len = (int64_t)s_end - a;
                constexpr int low_passes = (kBShift0 + kBRadixBits - 1) / kBRadixBits;
                cta_histograms(A.pkey, a, len, 0, low_passes, sm);
                const int np = cta_lsd_sort(A.pkey, A.perm, A.kalt, A.palt, a, len, 0, low_passes, false, sm);
                if (np & 1)
                    for (int64_t p = a + threadIdx.x; p < a + len; p += blockDim.x) {
                        A.pkey[p] = A.kalt[p];
                        A.perm[p] = A.palt[p];
                    }
                __syncthreads();
            }
        }
        // ---- cells and leaves started per level (the set is its own tree)
        if (threadIdx.x < kLevelFields) s_tot[threadIdx.x] = 0;
        __syncthreads();
        for (int64_t s = o; s < o + ns; s += T) {
            const int64_t e = min64(o + ns, s + T);
            const Front f = tile_front<T>(A.pkey, o, o + ns, A.ncrit, s, e, raw, ts);
            if (f.k < e) A.ml[f.k] = (uint16_t)(f.m | (f.L << 8));
            warp_field_prefix(ts, nullptr, s_tile);
            __syncthreads();
            if (threadIdx.x < kLevelFields) s_tot[threadIdx.x] += s_tile[threadIdx.x];
            __syncthreads();
        }
        if (threadIdx.x < kLevelFields)
            A.set_cnt[(int64_t)set * kLevelFields + threadIdx.x] = s_tot[threadIdx.x];
        __syncthreads();
    }
}

template <int T>
__global__ void __launch_bounds__(T, 1024 / T) batch_front_kernel(BatchArgs A) {
    if (A.info->status & kErrInvalid) return;
    extern __shared__ __align__(16) unsigned char raw[];
    front_sets<T>(A, raw);
}

// Cell and leaf offsets of the sets (in set order), totals and depth.
// One block of up to 1024 threads.
__device__ void batch_scan_block(const BatchArgs &A, int64_t cell_cap) {
    __shared__ int64_t s_c[1024], s_l[1024];
    __shared__ int s_dmax;
    const int S = A.n_sets;
    const int nt = blockDim.x;
    const int per = (S + nt - 1) / nt;
    const int lo = threadIdx.x * per, hi = min(S, lo + per);
    int64_t c = 0, l = 0;
    int dmax = 0;
    for (int s = lo; s < hi; ++s) {
        const uint32_t *r = A.set_cnt + (int64_t)s * kLevelFields;
        for (int d = 0; d < kLevels; ++d) {
            c += r[d];
            if (r[d]) dmax = max(dmax, d);
        }
        l += r[kLevels];
    }
    if (threadIdx.x == 0) s_dmax = 0;
    s_c[threadIdx.x] = c;
    s_l[threadIdx.x] = l;
    __syncthreads();
    atomicMax(&s_dmax, dmax);
    if (threadIdx.x == 0) {
        int64_t rc = 0, rl = 0;
        for (int t = 0; t < nt; ++t) {
            const int64_t vc = s_c[t], vl = s_l[t];
            s_c[t] = rc;
            s_l[t] = rl;
            rc += vc;
            rl += vl;
        }
        A.set_cell_off[S] = rc;
        A.set_leaf_off[S] = rl;
        A.info->n_cells = rc;
        A.info->n_leaves = (uint32_t)rl;
        for (int d = 0; d < kLevels; ++d) A.info->level_offset[d] = 0;
        A.info->level_offset[kLevels] = rc;
        if (cell_cap > 0 && rc > cell_cap) A.info->status |= kErrOverflow;
    }
    __syncthreads();
    int64_t rc = s_c[threadIdx.x], rl = s_l[threadIdx.x];
    for (int s = lo; s < hi; ++s) {
        A.set_cell_off[s] = rc;
        A.set_leaf_off[s] = rl;
        const uint32_t *r = A.set_cnt + (int64_t)s * kLevelFields;
        for (int d = 0; d < kLevels; ++d) rc += r[d];
        rl += r[kLevels];
    }
    if (threadIdx.x == 0) A.info->max_depth = s_dmax;
}

__global__ void __launch_bounds__(1024) batch_scan_kernel(BatchArgs A, int64_t cell_cap) {
    if (A.info->status & kErrInvalid) return;
    batch_scan_block(A, cell_cap);
}

// Every cell of one set with its links, then the set's particles in key
// order (tiles of T particles; all T threads of the block).
template <int T>
__device__ void emit_set(const BatchArgs &A, const EmitOut &out, int set) {
    __shared__ TileSharedT<T> ts;
    __shared__ uint32_t woff[T / 32][kLevelFields];
    __shared__ uint32_t s_run[kLevelFields], s_lvl[kLevelFields], s_tile[kLevelFields];
    {
        const int64_t o = A.off[set], ns = A.off[set + 1] - o;
        if (ns <= 0) return;
        const int64_t cell_base = A.set_cell_off[set], leaf_base = A.set_leaf_off[set];
        if (threadIdx.x == 0) {
            uint32_t r = 0;
            for (int d = 0; d < kLevels; ++d) {
                s_lvl[d] = r;
                r += A.set_cnt[(int64_t)set * kLevelFields + d];
            }
            s_lvl[kLevels] = 0;
        }
        if (threadIdx.x < kLevelFields) s_run[threadIdx.x] = 0;
        __syncthreads();
        for (int64_t s = o; s < o + ns; s += T) {
            const int64_t e = min64(o + ns, s + T);
            const Front f = tile_front_ml<T>(A.ml, o, s, e, ts);
            warp_field_prefix(ts, woff, s_tile);
            if (threadIdx.x < kLevelFields) {
                const int fld = threadIdx.x;
                ts.base[fld] = (uint32_t)(((fld < kLevels) ? cell_base : leaf_base) + s_lvl[fld] +
                                          s_run[fld]);
            }
            __syncthreads();
            if (f.k < e) {
                const int warp = threadIdx.x >> 5;
                const unsigned lt = lanemask_lt();
                auto P = [&](int d) {
                    return ts.base[d] + woff[warp][d] + (uint32_t)__popc(ts.mask[warp][d] & lt);
                };
                emit_particle(f, P, o, o + ns, A.pkey[f.k], out);
            }
            __syncthreads();
            if (threadIdx.x < kLevelFields) s_run[threadIdx.x] += s_tile[threadIdx.x];
            __syncthreads();
        }
        // the set's particles in key order, for its moments
        for (int64_t k = o + threadIdx.x; k < o + ns; k += blockDim.x) A.xs[k] = A.xm[A.perm[k]];
        __syncthreads();
    }
}

template <int T>
__global__ void __launch_bounds__(T, 2048 / T) batch_emit_kernel(BatchArgs A, EmitOut out) {
    if (A.info->status & (kErrOverflow | kErrNonFinite | kErrInvalid)) return;
    __shared__ int s_q;
    for (;;) {
        const int q = take_set(&A.queue[1], A.n_sets, &s_q);
        if (q < 0) return;
        emit_set<T>(A, out, A.order[q]);
    }
}

// FP64 sum of a leaf too long for the FP32 routes (more than 2^20 members).
__device__ __noinline__ void leaf_sum_f64_serial(const MomOut &o, const float4 *xs, int64_t c,
                                                 int64_t pf, int64_t pe, bool has64) {
    const float4 r0 = xs[pf];
    const float ref[3] = {r0.x, r0.y, r0.z};
    float bb[6] = {r0.x, r0.y, r0.z, r0.x, r0.y, r0.z};
    AccD D;
    D.init();
    for (int64_t k = pf; k < pe; ++k) {
        const float4 v = xs[k];
        const float x[3] = {v.x, v.y, v.z};
        double dx[3];
        for (int a = 0; a < 3; ++a) {
            bb[a] = fminf(bb[a], x[a]);
            bb[3 + a] = fmaxf(bb[3 + a], x[a]);
            dx[a] = (double)x[a] - (double)ref[a];
        }
        D.add((double)v.w, dx);
    }
    finish_d(o, c, D, ref, bb, has64);
}

// Moments of one set: every leaf in key order, then the other cells level by
// level, deepest first (all threads of the block).
template <int MODE>
__device__ void moments_set(const BatchArgs &A, const TreeIn &T, const MomOut &o,
                            const int32_t *__restrict__ leaf_cell, int set) {
    __shared__ int64_t s_lvl[kLevels + 1];
    {
        const int64_t ns = A.off[set + 1] - A.off[set];
        if (ns <= 0) return;
        if (threadIdx.x == 0) {
            int64_t r = A.set_cell_off[set];
            for (int d = 0; d < kLevels; ++d) {
                s_lvl[d] = r;
                r += A.set_cnt[(int64_t)set * kLevelFields + d];
            }
            s_lvl[kLevels] = r;
        }
        // every leaf of the set first, in key order (neighbouring lanes read
        // neighbouring records), then the other cells level by level
        const int64_t l0 = A.set_leaf_off[set], l1 = A.set_leaf_off[set + 1];
        for (int64_t j = l0 + threadIdx.x; j < l1; j += blockDim.x) {
            const int64_t c = leaf_cell[j];
            const int64_t pf = T.pfirst[c], pe = T.pend[c];
            if (pe - pf > kBigLeafSerial) leaf_sum_f64_serial(o, A.xs, c, pf, pe, MODE == TB_MOM_FP64);
            else leaf_sum<MODE>(o, A.xs, c, pf, pe);
        }
        __syncthreads();
        for (int d = kDepthMax - 1; d >= 0; --d) {
            for (int64_t c = s_lvl[d] + threadIdx.x; c < s_lvl[d + 1]; c += blockDim.x)
                if (T.child_first[c] >= 0) combine_children<MODE>(T, o, c, cells_of(o));
            __syncthreads();
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kBMomThreads, 3)
    batch_moments_kernel(BatchArgs A, TreeIn T, MomOut o, const int32_t *__restrict__ leaf_cell) {
    if (A.info->status & (kErrOverflow | kErrNonFinite | kErrInvalid)) return;
    __shared__ int s_q;
    for (;;) {
        const int q = take_set(&A.queue[2], A.n_sets, &s_q);
        if (q < 0) return;
        moments_set<MODE>(A, T, o, leaf_cell, A.order[q]);
    }
}

// The set offsets must partition [0, n_total): off[0] = 0, off[S] = n_total,
// non-decreasing.  Otherwise every batched kernel skips its work.
__device__ void set_check_grid(const int64_t *off, int32_t S, int64_t n_total, DevInfo *info) {
    bool bad = false;
    if (blockIdx.x == 0 && threadIdx.x == 0) bad = (off[0] != 0 || off[S] != n_total);
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x)
        bad |= off[s + 1] < off[s] || off[s + 1] - off[s] > 2147483647LL;
    if (bad) atomicOr(&info->status, kErrInvalid);
}

__global__ void set_check_kernel(const int64_t *off, int32_t S, int64_t n_total, DevInfo *info) {
    set_check_grid(off, S, n_total, info);
}

// A barrier across every block of a cooperative launch (all blocks are
// resident at once, so every block arrives).  bar[0] counts arrivals, bar[1]
// is the generation; the last block to arrive resets the count and opens the
// next generation.  The wait is bounded: one that runs out records a timeout
// and lets the block go on.
__device__ void grid_barrier(uint32_t *bar, int64_t limit, DevInfo *info) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *gen = bar + 1;
        const uint32_t g = *gen;
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            int64_t it = 0;
            while (*gen == g) {
                if (!poll_backoff(it, limit)) {
                    flag_error(&info->status, kErrTimeout);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// The whole batched build in one cooperative launch (fixed cell capacity):
// offsets checked, sets ordered, every set's front (keys, sort, counts), the
// offsets of all sets, then each set's cells and moments by the block that
// takes it -- phases separated by grid barriers.
template <int T, int MODE>
__global__ void __launch_bounds__(T, 1024 / T)
    batch_all_kernel(BatchArgs A, int32_t *order, EmitOut out, TreeIn Tr, MomOut o,
                     const int32_t *__restrict__ leaf_cell, int64_t n_total, int64_t cell_cap,
                     int64_t wait_limit) {
    extern __shared__ __align__(16) unsigned char raw[];
    uint32_t *bar = A.queue + 4;
    __shared__ int s_q;
    set_check_grid(A.off, A.n_sets, n_total, A.info);
    grid_barrier(bar, wait_limit, A.info);
    // the status words below were all written before a barrier: every block
    // reads the same values and takes the same branch
    if (*(volatile uint32_t *)&A.info->status & kErrInvalid) return;
    if (blockIdx.x == 0) set_order_block(A.off, A.n_sets, order);
    grid_barrier(bar, wait_limit, A.info);
    front_sets<T>(A, raw);
    grid_barrier(bar, wait_limit, A.info);
    if (blockIdx.x == 0) batch_scan_block(A, cell_cap);
    grid_barrier(bar, wait_limit, A.info);
    if (*(volatile uint32_t *)&A.info->status & (kErrOverflow | kErrNonFinite)) return;
    for (;;) {
        const int q = take_set(&A.queue[1], A.n_sets, &s_q);
        if (q < 0) return;
        const int set = order[q];
        emit_set<T>(A, out, set);
        moments_set<MODE>(A, Tr, o, leaf_cell, set);
    }
}

}  // namespace

cudaError_t launch_set_check(const int64_t *off, int32_t S, int64_t n_total, Workspace &ws,
                             cudaStream_t s) {
    int grid = (S + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > 1024) grid = 1024;
    set_check_kernel<<<grid, 256, 0, s>>>(off, S, n_total, ws.info);
    ++g_launches;
    return cudaGetLastError();
}

namespace {

template <int T>
cudaError_t launch_batched_t(const BatchArgs &A, int32_t S, int ncrit, tb_tree &t, Workspace &ws,
                             int64_t cell_cap, int phase, int mode, cudaStream_t s) {
    cudaError_t e;
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        const int sm_front = (int)batch_front_smem<T>(kMaxNcrit);
        cudaFuncSetAttribute(batch_front_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sm_front);
        cudaFuncSetAttribute(batch_front_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // persistent grids: as many blocks as fit at once (1024 / T front blocks
    // per SM, two emission blocks), at most one per set
    auto fit = [&](int per_sm) { return S < per_sm * nsm ? (S > 0 ? S : 1) : per_sm * nsm; };
    if (phase == 0) {
        set_order_kernel<<<1, 1024, 0, s>>>(A.off, S, ws.set_order, ws.info);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        batch_front_kernel<T><<<fit(1024 / T), T, batch_front_smem<T>(ncrit), s>>>(A);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        mark(ws, "batch_front", s);
        batch_scan_kernel<<<1, 1024, 0, s>>>(A, cell_cap);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        mark(ws, "batch_scan", s);
        return cudaSuccess;
    }
    EmitOut out{t.ckey, t.level, t.parent, t.child_first, t.child_end, t.pfirst, t.pend,
                t.leaf_cell};
    // the emission keeps 1024-thread tiles whatever the front's block size
    // (two blocks per SM at 32 registers): measured faster than 512 (0.96
    // against 1.10 ms on the 4,096-set workload)
    batch_emit_kernel<1024><<<fit(2), 1024, 0, s>>>(A, out);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(ws, "batch_emit", s);
    TreeIn Tr{t.child_first, t.child_end, t.pfirst, t.pend, ws.big_leaf, t.parent};
    MomOut o{t.mass, t.com, t.com_lo, t.quad, t.aabb, t.mass64, t.com64, t.quad64};
    const int grid_mom = fit(3);
    switch (mode) {
        case TB_MOM_FP32_COMP:
            batch_moments_kernel<TB_MOM_FP32_COMP><<<grid_mom, kBMomThreads, 0, s>>>(A, Tr, o, t.leaf_cell);
            break;
        case TB_MOM_FP32_PLAIN:
            batch_moments_kernel<TB_MOM_FP32_PLAIN><<<grid_mom, kBMomThreads, 0, s>>>(A, Tr, o, t.leaf_cell);
            break;
        default:
            batch_moments_kernel<TB_MOM_FP64><<<grid_mom, kBMomThreads, 0, s>>>(A, Tr, o, t.leaf_cell);
            break;
    }
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(ws, "batch_moments", s);
    return cudaSuccess;
}

}  // namespace

template <int T, int MODE>
cudaError_t launch_batched_one_t(const BatchArgs &A, int32_t S, int ncrit, int64_t n_total,
                                 tb_tree &t, Workspace &ws, int64_t cell_cap, cudaStream_t s) {
    auto kern = batch_all_kernel<T, MODE>;
    const size_t smem = batch_front_smem<T>(ncrit);
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_front_smem<T>(kMaxNcrit));
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    int dev = 0, nsm = 152, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // every block resident at once (the grid barriers need it), at most one
    // block per set
    const int grid = S < per_sm * nsm ? (S > 0 ? S : 1) : per_sm * nsm;
    BatchArgs a = A;
    int32_t *order = ws.set_order;
    EmitOut out{t.ckey, t.level, t.parent, t.child_first, t.child_end, t.pfirst, t.pend,
                t.leaf_cell};
    TreeIn Tr{t.child_first, t.child_end, t.pfirst, t.pend, ws.big_leaf, t.parent};
    MomOut o{t.mass, t.com, t.com_lo, t.quad, t.aabb, t.mass64, t.com64, t.quad64};
    const int32_t *leaf_cell = t.leaf_cell;
    int64_t nt = n_total, cap = cell_cap, lim = g_wait_limit;
    void *args[] = {&a, &order, &out, &Tr, &o, &leaf_cell, &nt, &cap, &lim};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(T), args,
                                    smem, s);
    if (e != cudaSuccess) return e;
    ++g_launches;
    mark(ws, "batch_all", s);
    return cudaSuccess;
}

bool batch_threads_valid(int threads) { return threads == 0 || threads == 512 || threads == 1024; }

cudaError_t launch_batched_one(const float *pos, const float *mass, const int64_t *off, int32_t S,
                               int64_t n_total, int ncrit, int threads, tb_tree &t, Workspace &ws,
                               int64_t cell_cap, int mode, cudaStream_t s) {
    BatchArgs A{pos, mass, off, ws.set_order, S, ncrit, t.pkey, t.perm, ws.keys_alt,
                ws.perm_alt, ws.xm, ws.xs, ws.ml, ws.set_cnt, t.set_cell_offset, ws.set_leaf_off,
                t.set_root, ws.set_ctr, ws.info, ws.root_pow2 ? 1 : 0};
    const int T = threads ? threads : kBDefaultThreads;
#define TB_ONE(TT, MM) \
    if (T == TT && mode == MM) return launch_batched_one_t<TT, MM>(A, S, ncrit, n_total, t, ws, cell_cap, s);
    TB_ONE(512, TB_MOM_FP32_COMP)
    TB_ONE(512, TB_MOM_FP32_PLAIN)
    TB_ONE(512, TB_MOM_FP64)
    TB_ONE(1024, TB_MOM_FP32_COMP)
    TB_ONE(1024, TB_MOM_FP32_PLAIN)
    TB_ONE(1024, TB_MOM_FP64)
#undef TB_ONE
    return cudaErrorInvalidValue;
}

cudaError_t launch_batched(const float *pos, const float *mass, const int64_t *off, int32_t S,
                           int ncrit, int threads, tb_tree &t, Workspace &ws, int64_t cell_cap,
                           int phase, int mode, cudaStream_t s) {
    BatchArgs A{pos, mass, off, ws.set_order, S, ncrit, t.pkey, t.perm, ws.keys_alt,
                ws.perm_alt, ws.xm, ws.xs, ws.ml, ws.set_cnt, t.set_cell_offset, ws.set_leaf_off,
                t.set_root, ws.set_ctr, ws.info, ws.root_pow2 ? 1 : 0};
    switch (threads ? threads : kBDefaultThreads) {
        case 512: return launch_batched_t<512>(A, S, ncrit, t, ws, cell_cap, phase, mode, s);
        case 1024: return launch_batched_t<1024>(A, S, ncrit, t, ws, cell_cap, phase, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tb
