// tb_walk.cu -- gravity from the built tree (Sec. 2.1): the Barnes-Hut walk
// with the opening test l / d < theta of Eq. 1, monopole plus quadrupole, and
// Barnes' modified algorithm, in which the particles of one small cell share
// one interaction list.
//
//   walk_groups_kernel : the groups -- every cell holding at most n_group
//                        particles whose parent holds more (the root if it
//                        holds at most n_group), and every leaf holding more
//                        (only depth-21 leaves of one key can);
//   walk_kernel        : one warp per group (taken from an atomic ticket),
//                        32 particles at a time (one per lane; a larger group
//                        is walked in chunks of 32, each with its own box).
//                        The warp walks the tree from the root, up to 32 cells
//                        at a time: a cell whose particle range meets the chunk's is
//                        always opened; any other cell is accepted when
//                        l < theta * d_min, d_min the distance from its centre
//                        of mass to the group's bounding box (so l / d < theta
//                        holds for every particle of the group); an opened leaf
//                        contributes its particles one by one.  Accepted cells
//                        and opened leaves go to lists in shared memory; when a
//                        list is full, and at the end, every lane evaluates the
//                        lists for its particles of the group.
// Forces (G = 1): a softened point mass m (r^2 + eps^2)^(-3/2) r for every
// particle and cell; for a cell also the quadrupole term
//   T r / |r|^5 - (5/2) (r.T r) r / |r|^7,  T = 3 Q - tr(Q) I,
// with Q the cell's central second moment and r = x - COM (unsoftened).
// Offsets are taken as (x - com) - com_lo, exact to one rounding when the
// target and the centre are close.  The result is written in the caller's
// particle order.  A walk on a tree with profiling enabled also counts the
// interactions it evaluated (target-cell and target-particle pairs), read
// back by tb_walk_counts.
#include "tb_device.cuh"

namespace tb {

namespace {

constexpr int kWalkWarps = 4;
constexpr int kWalkBlocks = 152 * 6;   // as many as fit (shared memory)
constexpr int kWalkThreads = 32 * kWalkWarps;
// cells waiting to be tested, per warp in global memory: a round takes at most
// 32 cells and adds at most 7 per cell, and only cells above depth 21 have
// children, so the stack stays below 21 * 256 + 1 entries
constexpr int kStackCap = 6144;
constexpr int kCellCap = 128;       // accepted cells
constexpr int kRangeCap = 128;      // particle ranges of opened leaves

struct WalkTree {
    const int32_t *child_first, *child_end, *pfirst, *pend;
    const uint8_t *level;
    const float *mass, *com, *com_lo, *quad, *aabb;
    const float4 *xs;               // particles in key order: x, y, z, m
    const int32_t *perm;
    double side;
    const float4 *rec;              // [C][4] per cell: com + m, com_lo, T xx xy xz yy, T yz zz
};

struct WarpLists {
    float4 cell[kCellCap][4];       // the accepted cells' records, copied when accepted
    int2 range[kRangeCap];
};

__device__ __forceinline__ float3 point_acc(float3 a, float rx, float ry, float rz, float m, float eps2) {
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2)));
    const float inv = rsqrtf(r2);
    const float f = m * inv * inv * inv;
    a.x = fmaf(-f, rx, a.x);
    a.y = fmaf(-f, ry, a.y);
    a.z = fmaf(-f, rz, a.z);
    return a;
}

// the lists of one warp against its lane's particle k (when k < ke)
__device__ float3 evaluate(const WalkTree &T, const WarpLists &W, int ncell, int nrange, int64_t k,
                           int64_t ke, float eps2, bool use_quad, float3 a) {
    const float4 x = k < ke ? T.xs[k] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
    for (int j = 0; j < ncell; ++j) {
        const float4 c0 = W.cell[j][0], c1 = W.cell[j][1];
        const float m = c0.w;
        const float rx = (x.x - c0.x) - c1.x;
        const float ry = (x.y - c0.y) - c1.y;
        const float rz = (x.z - c0.z) - c1.z;
        a = point_acc(a, rx, ry, rz, m, eps2);
        if (use_quad) {
            const float4 t0 = W.cell[j][2], t1 = W.cell[j][3];
            const float txx = t0.x, txy = t0.y, txz = t0.z, tyy = t0.w, tyz = t1.x, tzz = t1.y;
            const float trx = txx * rx + txy * ry + txz * rz;
            const float try_ = txy * rx + tyy * ry + tyz * rz;
            const float trz = txz * rx + tyz * ry + tzz * rz;
            const float rtr = rx * trx + ry * try_ + rz * trz;
            const float ir = rsqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
            const float ir2 = ir * ir;
            const float ir5 = ir2 * ir2 * ir;
            const float s = 2.5f * rtr * ir5 * ir2;
            a.x += trx * ir5 - s * rx;
            a.y += try_ * ir5 - s * ry;
            a.z += trz * ir5 - s * rz;
        }
    }
    for (int j = 0; j < nrange; ++j) {
        const int2 r = W.range[j];
        for (int q = r.x; q < r.y; ++q) {
            if (q == k) continue;                       // no self-force
            const float4 y = T.xs[q];
            a = point_acc(a, x.x - y.x, x.y - y.y, x.z - y.z, y.w, eps2);
        }
    }
    return a;
}

// Per cell, kRec float4: the four the list evaluation reads (centre and
// mass; the centre's low part, with the cell's level in the last word; the
// traceless tensor T = 3 Q - tr(Q) I) and the links the traversal reads
// (pfirst, pend, child_first, child_end), so that a cell tested costs three
// 16-byte loads.
constexpr int kRec = 5;

__global__ void walk_pack_kernel(const float *__restrict__ mass, const float *__restrict__ com,
                                 const float *__restrict__ com_lo, const float *__restrict__ quad,
                                 const uint8_t *__restrict__ level, const int32_t *__restrict__ pfirst,
                                 const int32_t *__restrict__ pend, const int32_t *__restrict__ child_first,
                                 const int32_t *__restrict__ child_end, int64_t n_cells,
                                 float4 *__restrict__ rec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cells; c += stride) {
        const float *q = quad + 6 * c;
        const float tr = q[0] + q[3] + q[5];
        float4 *r = rec + kRec * c;
        r[0] = make_float4(com[3 * c], com[3 * c + 1], com[3 * c + 2], mass[c]);
        r[1] = make_float4(com_lo[3 * c], com_lo[3 * c + 1], com_lo[3 * c + 2],
                           __int_as_float((int)level[c]));
        r[2] = make_float4(3.f * q[0] - tr, 3.f * q[1], 3.f * q[2], 3.f * q[3] - tr);
        r[3] = make_float4(3.f * q[4], 3.f * q[5] - tr, 0.f, 0.f);
        reinterpret_cast<int4 *>(r)[4] = make_int4(pfirst[c], pend[c], child_first[c], child_end[c]);
    }
}

__global__ void walk_groups_kernel(const int32_t *__restrict__ parent, const int32_t *__restrict__ child_first,
                                   const int32_t *__restrict__ pfirst, const int32_t *__restrict__ pend,
                                   int64_t n_cells, int n_group, int32_t *groups, uint32_t *ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cells; c += stride) {
        const int64_t cnt = (int64_t)pend[c] - pfirst[c];
        const int32_t p = parent[c];
        const bool small = cnt <= n_group && (p < 0 || (int64_t)pend[p] - pfirst[p] > n_group);
        const bool big_leaf = child_first[c] < 0 && cnt > n_group;
        if (small || big_leaf) groups[atomicAdd(&ctr[0], 1u)] = (int32_t)c;
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(kWalkThreads)
    walk_kernel(WalkTree T, const int32_t *__restrict__ groups, uint32_t *ctr, int32_t *stacks,
                float theta, float eps2, int use_quad, float *__restrict__ acc_out, DevInfo *info) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    __shared__ WarpLists lists[kWalkWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpLists &W = lists[warp];
    int32_t *stack = stacks + ((int64_t)blockIdx.x * kWalkWarps + warp) * kStackCap;
    const uint32_t ngroups = *(volatile const uint32_t *)&ctr[0];
    const unsigned lt = lanemask_lt();
    const float side = (float)T.side;
    // interactions evaluated by this warp (lane 0 counts): target x accepted
    // cell, and target x source particle (self excluded); added to the
    // walk's totals when the warp is done
    unsigned long long n_cell_int = 0, n_pp_int = 0;
    unsigned long long *totals = reinterpret_cast<unsigned long long *>(ctr + 2);
    auto count = [&](int ncell, int nrange, int64_t nt) {
        if (!COUNT) return;
        long long srcs = 0;
        for (int j = lane; j < nrange; j += 32) srcs += W.range[j].y - W.range[j].x;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) srcs += __shfl_xor_sync(0xffffffffu, srcs, off);
        if (lane == 0) {
            n_cell_int += (unsigned long long)(ncell * nt);
            n_pp_int += (unsigned long long)(srcs * nt);
        }
    };
    for (;;) {
        uint32_t gi = 0;
        if (lane == 0) gi = atomicAdd(&ctr[1], 1u);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= ngroups) {
            if (COUNT && lane == 0) {
                atomicAdd(&totals[0], n_cell_int);
                atomicAdd(&totals[1], n_pp_int);
            }
            return;
        }
        const int32_t g = groups[gi];
        const int64_t gpf = T.pfirst[g], gpe = T.pend[g];
        for (int64_t kb = gpf; kb < gpe; kb += 32) {
            const int64_t ke = min64(gpe, kb + 32);
            const int64_t k = kb + lane;
            // bounding box of the chunk
            float bmin[3], bmax[3];
            {
                const float4 x = T.xs[k < ke ? k : kb];
                bmin[0] = bmax[0] = x.x;
                bmin[1] = bmax[1] = x.y;
                bmin[2] = bmax[2] = x.z;
                for (int off = 16; off > 0; off >>= 1)
                    for (int a = 0; a < 3; ++a) {
                        bmin[a] = fminf(bmin[a], __shfl_xor_sync(0xffffffffu, bmin[a], off));
                        bmax[a] = fmaxf(bmax[a], __shfl_xor_sync(0xffffffffu, bmax[a], off));
                    }
            }
            float3 acc = make_float3(0.f, 0.f, 0.f);
            int sp = 1, ncell = 0, nrange = 0;
            if (lane == 0) stack[0] = 0;
            __syncwarp();
            bool overflow = false;
            while (sp > 0) {
                // room for this round: 32 accepted cells or leaf ranges, and
                // 7 more stack entries per cell taken
                if (ncell + 32 > kCellCap || nrange + 32 > kRangeCap) {
                    count(ncell, nrange, ke - kb);
                    acc = evaluate(T, W, ncell, nrange, k, ke, eps2, use_quad != 0, acc);
                    ncell = nrange = 0;
                    __syncwarp();
                }
                const int take = min(min(sp, 32), (kStackCap - sp) / 7);
                if (take == 0) {
                    overflow = true;
                    break;
                }
                int c = -1;
                if (lane < take) c = stack[sp - 1 - lane];
                sp -= take;
                __syncwarp();
                int kind = 0;                           // 1 accept, 2 leaf, 3 open
                int nch = 0, c0 = 0;
                float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
                int4 lk = make_int4(0, 0, 0, 0);        // pfirst, pend, child_first, child_end
                if (c >= 0) {
                    lk = reinterpret_cast<const int4 *>(T.rec + kRec * (int64_t)c)[4];
                    const bool meets = lk.x < ke && kb < lk.y;
                    c0 = lk.z;
                    bool accept = false;
                    if (!meets) {
                        r0 = T.rec[kRec * (int64_t)c];
                        r1 = T.rec[kRec * (int64_t)c + 1];
                        const float l = scalbnf(side, -__float_as_int(r1.w));
                        const float cx[3] = {r0.x + r1.x, r0.y + r1.y, r0.z + r1.z};
                        float d2 = 0.f;
                        for (int a = 0; a < 3; ++a) {
                            const float u = fmaxf(fmaxf(bmin[a] - cx[a], cx[a] - bmax[a]), 0.f);
                            d2 = fmaf(u, u, d2);
                        }
                        accept = l * l < theta * theta * d2;
                    }
                    if (accept) kind = 1;
                    else if (c0 < 0) kind = 2;
                    else { kind = 3; nch = lk.w - c0; }
                }
                const unsigned ba = __ballot_sync(0xffffffffu, kind == 1);
                const unsigned bl = __ballot_sync(0xffffffffu, kind == 2);
                if (kind == 1) {
                    float4 *dst = W.cell[ncell + __popc(ba & lt)];
                    dst[0] = r0;
                    dst[1] = r1;
                    dst[2] = T.rec[kRec * (int64_t)c + 2];
                    dst[3] = T.rec[kRec * (int64_t)c + 3];
                }
                if (kind == 2) W.range[nrange + __popc(bl & lt)] = make_int2(lk.x, lk.y);
                ncell += __popc(ba);
                nrange += __popc(bl);
                // children onto the stack (exclusive scan of the counts)
                int pos = nch;
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, pos, off);
                    if (lane >= off) pos += y;
                }
                const int total = __shfl_sync(0xffffffffu, pos, 31);
                pos -= nch;
                for (int j = 0; j < nch; ++j) stack[sp + pos + j] = c0 + nch - 1 - j;
                sp += total;
                __syncwarp();
            }
            if (overflow) {
                if (lane == 0) atomicOr(&info->status, kErrWalk);
                return;
            }
            count(ncell, nrange, ke - kb);
            if (COUNT && lane == 0) n_pp_int -= (unsigned long long)(ke - kb);   // own pairs
            acc = evaluate(T, W, ncell, nrange, k, ke, eps2, use_quad != 0, acc);
            __syncwarp();
            if (k < ke) {
                const int64_t i = T.perm[k];
                acc_out[3 * i] = acc.x;
                acc_out[3 * i + 1] = acc.y;
                acc_out[3 * i + 2] = acc.z;
            }
        }
    }
}

}  // namespace

int64_t walk_buffer_words(int64_t n_cells) {
    return 4 * kRec * n_cells + 8 + n_cells + (int64_t)kWalkBlocks * kWalkWarps * kStackCap;
}

cudaError_t launch_walk(const tb_tree &t, Workspace &ws, float theta, float eps, int n_group,
                        int use_quad, float *acc, int32_t *buf, cudaStream_t s) {
    float4 *rec = reinterpret_cast<float4 *>(buf);   // first: 16-byte aligned
    uint32_t *ctr = reinterpret_cast<uint32_t *>(buf + 4 * kRec * t.n_cells);
    ws.walk_ctr = ctr;
    int32_t *groups = buf + 4 * kRec * t.n_cells + 8;
    int32_t *stacks = groups + t.n_cells;
    cudaError_t e = cudaMemsetAsync(ctr, 0, 8 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int64_t grid = (t.n_cells + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    walk_groups_kernel<<<(unsigned)grid, 256, 0, s>>>(t.parent, t.child_first, t.pfirst, t.pend,
                                                      t.n_cells, n_group, groups, ctr);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    walk_pack_kernel<<<(unsigned)grid, 256, 0, s>>>(t.mass, t.com, t.com_lo, t.quad, t.level, t.pfirst,
                                                    t.pend, t.child_first, t.child_end, t.n_cells,
                                                    rec);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    WalkTree T{t.child_first, t.child_end, t.pfirst, t.pend, t.level, t.mass, t.com, t.com_lo,
               t.quad, t.aabb, ws.xs, t.perm, t.side, rec};
    // the interaction counts cost about 15% of the walk: only profiled walks
    // take them
    if (ws.profile)
        walk_kernel<true><<<kWalkBlocks, kWalkThreads, 0, s>>>(T, groups, ctr, stacks, theta,
                                                               eps * eps, use_quad, acc, ws.info);
    else
        walk_kernel<false><<<kWalkBlocks, kWalkThreads, 0, s>>>(T, groups, ctr, stacks, theta,
                                                                eps * eps, use_quad, acc, ws.info);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace tb
