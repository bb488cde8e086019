// tb_moments.cu -- cell moments without traversing the tree (Sec. 2.3: cell
// properties are computed as cells are created; the centre of mass of a
// parent comes from those of its children, higher multipoles likewise).
//
//   gather_kernel        : particles in key order, (x, y, z, m) records
//                          (Sec. 2.3 step 3, the reorder); every thread keeps
//                          four independent gathers in flight;
//   leaf_moments_kernel  : every leaf sums its contiguous members (leaves in
//                          key order, one launch for all levels);
//   big_leaf_kernel      : depth-21 leaves of identical keys that are too long
//                          for one thread, summed block-wide;
//   level_moments_kernel : one launch per level, deepest first: every other
//                          cell combines its children, which earlier launches
//                          finished.
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
// A cell of more than 2^20 particles is summed / combined in FP64 in every
// mode.
#include "tb_moments.cuh"

namespace tb {

namespace {

// ------------------------------------------------------------ kernels

// xs[k] = xm[perm[k]]: the particles in key order.
__global__ void __launch_bounds__(256)
    gather_kernel(const int32_t *__restrict__ perm, const float4 *__restrict__ xm,
                  float4 *__restrict__ xs, int64_t n, const DevInfo *info) {
    if (info->status & kErrNonFinite) return;
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

// Every leaf, in key order (so a warp reads one stretch of the records).
// Leaves longer than kBigLeafThread -- only depth-21 leaves of identical keys
// can be -- are queued for big_leaf_kernel.
template <int MODE>
__global__ void __launch_bounds__(kMomThreads, 3)
    leaf_moments_kernel(TreeIn T, MomOut o, const int32_t *__restrict__ leaf_cell,
                        const float4 *__restrict__ xs, DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    const int64_t nl = info->n_leaves;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nl; j += stride) {
        const int64_t c = leaf_cell[j];
        const int64_t pf = T.pfirst[c], pe = T.pend[c];
        if (pe - pf > kBigLeafThread) {
            const uint32_t q = atomicAdd(&info->misc_ctr[2], 1u);
            T.big_leaf[q] = (int32_t)c;
            continue;
        }
        leaf_sum<MODE>(o, xs, c, pf, pe);
    }
}

// Compensated mode: every leaf of at most kSplitLeaf members, in key order,
// with the split sums only (few registers, many warps in flight); longer
// leaves are queued for mid_leaf_kernel (compensated sums) or, beyond
// kBigLeafThread, for big_leaf_kernel.
__global__ void __launch_bounds__(kMomThreads, 4)
    leaf_split_kernel(TreeIn T, MomOut o, const int32_t *__restrict__ leaf_cell,
                      const float4 *__restrict__ xs, int32_t *mid_queue, DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    const int64_t nl = info->n_leaves;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nl; j += stride) {
        const int64_t c = leaf_cell[j];
        const int64_t pf = T.pfirst[c], pe = T.pend[c];
        if (pe - pf > kBigLeafThread) T.big_leaf[atomicAdd(&info->misc_ctr[2], 1u)] = (int32_t)c;
        else if (pe - pf > kSplitLeaf) mid_queue[atomicAdd(&info->misc_ctr[5], 1u)] = (int32_t)c;
        else leaf_sum_split(o, xs, c, pf, pe);
    }
}

// Compensated mode: the queued leaves of kSplitLeaf + 1 .. kBigLeafThread members.
__global__ void __launch_bounds__(kMomThreads, 3)
    mid_leaf_kernel(TreeIn T, MomOut o, const float4 *__restrict__ xs, const int32_t *mid_queue,
                    DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    const int64_t nq = *(volatile const uint32_t *)&info->misc_ctr[5];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += stride) {
        const int64_t c = mid_queue[q];
        leaf_sum<TB_MOM_FP32_COMP>(o, xs, c, T.pfirst[c], T.pend[c]);
    }
}

// The non-leaf cells of level d, from their children (finished by the
// launch for level d + 1, or by the leaf launches).  Each warp takes 64
// consecutive cells and packs their non-leaf ones, in order, onto its lanes.
template <int MODE>
__global__ void __launch_bounds__(kMomThreads, 4)
    level_moments_kernel(TreeIn T, MomOut o, DevInfo *info, int d) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    __shared__ int32_t s_list[kMomThreads / 32][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t lo = info->level_offset[d], hi = info->level_offset[d + 1];
    const int64_t nwarps = (int64_t)gridDim.x * (kMomThreads / 32);
    const unsigned lt = lanemask_lt();
    for (int64_t base = lo + ((int64_t)blockIdx.x * (kMomThreads / 32) + warp) * 64; base < hi;
         base += nwarps * 64) {
        const int64_t c0 = base + lane, c1 = base + 32 + lane;
        const bool p0 = c0 < hi && T.child_first[c0] >= 0;
        const bool p1 = c1 < hi && T.child_first[c1] >= 0;
        const unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
        if (p0) s_list[warp][__popc(b0 & lt)] = (int32_t)c0;
        if (p1) s_list[warp][__popc(b0) + __popc(b1 & lt)] = (int32_t)c1;
        __syncwarp();
        const int cnt = __popc(b0) + __popc(b1);
        for (int k = lane; k < cnt; k += 32) combine_children<MODE>(T, o, s_list[warp][k]);
        __syncwarp();
    }
}

// Block-wide sums of the long depth-21 leaves queued by the leaf launch.
template <int MODE>
__global__ void __launch_bounds__(kBigThreads)
    big_leaf_kernel(TreeIn T, MomOut o, const float4 *__restrict__ xs, DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
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
    TreeIn T{t.child_first, t.child_end, t.pfirst, t.pend, ws.big_leaf};
    MomOut o{t.mass, t.com, t.com_lo, t.quad, t.aabb, t.mass64, t.com64, t.quad64};
    const int64_t n = t.n_particles;
    // misc_ctr[2..3]: big-leaf queue and tickets; [5]: mid-leaf queue
    cudaError_t e = cudaMemsetAsync(&ws.info->misc_ctr[2], 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int64_t g = (n / 4 + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    gather_kernel<<<(unsigned)g, 256, 0, s>>>(t.perm, ws.xm, ws.xs, n, ws.info);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(ws, "gather", s);
    // one persistent grid per launch; a level holds at most n cells
    int64_t grid = (n + kMomThreads - 1) / kMomThreads;
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    if constexpr (MODE == TB_MOM_FP32_COMP) {
        // the mid-leaf queue (at most n / 17 leaves) sits in the upper half
        // of the big-leaf buffer (at most n / 2049 entries in the lower)
        int32_t *mid = ws.big_leaf + (n + 1) / 2;
        leaf_split_kernel<<<(unsigned)(152 * 8), kMomThreads, 0, s>>>(T, o, t.leaf_cell, ws.xs, mid,
                                                                     ws.info);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        mid_leaf_kernel<<<(unsigned)grid, kMomThreads, 0, s>>>(T, o, ws.xs, mid, ws.info);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        leaf_moments_kernel<MODE><<<(unsigned)grid, kMomThreads, 0, s>>>(T, o, t.leaf_cell, ws.xs,
                                                                         ws.info);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    big_leaf_kernel<MODE><<<152, kBigThreads, 0, s>>>(T, o, ws.xs, ws.info);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(ws, "leaves", s);
    for (int d = kDepthMax - 1; d >= 0; --d) {
        level_moments_kernel<MODE><<<(unsigned)grid, kMomThreads, 0, s>>>(T, o, ws.info, d);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    mark(ws, "moments", s);
    return cudaSuccess;
}

}  // namespace

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
