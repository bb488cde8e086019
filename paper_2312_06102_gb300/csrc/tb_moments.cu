// tb_moments.cu -- cell moments without traversing the tree (Sec. 2.3: cell
// properties are computed as cells are created; the centre of mass of a
// parent comes from those of its children, higher multipoles likewise).
//
//   gather_kernel        : particles in key order, (x, y, z, m) records
//                          (Sec. 2.3 step 3, the reorder); every thread keeps
//                          four independent gathers in flight;
//   level_moments_kernel : one launch per level, deepest first: a leaf sums its
//                          contiguous members, any other cell combines its
//                          children, which the previous launch finished;
//   big_leaf_kernel      : depth-21 leaves of identical keys that are too long
//                          for one thread, summed block-wide.
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
#include <type_traits>

#include "tb_device.cuh"

namespace tb {

namespace {

constexpr int kMomThreads = 256;
constexpr int kBigLeafThread = 2048;   // longer leaves are summed by a block
constexpr int kBigThreads = 256;

struct MomOut {
    float *mass, *com, *com_lo, *quad, *aabb;
    double *mass64, *com64, *quad64;
};

struct TreeIn {
    const int32_t *child_first, *child_end, *pfirst, *pend;
    int32_t *big_leaf;
};

__device__ __forceinline__ int qidx(int a, int b) {
    // xx xy xz yy yz zz
    return (a == 0) ? b : (a == 1 ? 2 + b : 5);
}

// --------------------------------------------------------- accumulators

// compensated FP32 raw sums relative to a reference point
struct AccC {
    float M, Mc, S[3], Sc[3], Q[6], Qc[6];
    __device__ void init() {
        M = Mc = 0.f;
        for (int a = 0; a < 3; ++a) S[a] = Sc[a] = 0.f;
        for (int j = 0; j < 6; ++j) Q[j] = Qc[j] = 0.f;
    }
    __device__ void add(float m, const float dx[3]) {
        float e;
        two_sum(M, m, M, e);
        Mc += e;
        float p[3], pe[3];
        for (int a = 0; a < 3; ++a) {
            two_prod(m, dx[a], p[a], pe[a]);
            two_sum(S[a], p[a], S[a], e);
            Sc[a] += e + pe[a];
        }
        int j = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b, ++j) {
                float q, qe;
                two_prod(p[a], dx[b], q, qe);
                qe = __fmaf_rn(pe[a], dx[b], qe);
                two_sum(Q[j], q, Q[j], e);
                Qc[j] += e + qe;
            }
    }
    // merge another accumulator of the same reference point
    __device__ void merge(const AccC &o) {
        float e;
        two_sum(M, o.M, M, e); Mc += e + o.Mc;
        for (int a = 0; a < 3; ++a) { two_sum(S[a], o.S[a], S[a], e); Sc[a] += e + o.Sc[a]; }
        for (int j = 0; j < 6; ++j) { two_sum(Q[j], o.Q[j], Q[j], e); Qc[j] += e + o.Qc[j]; }
    }
};

struct AccP {
    float M, S[3], Q[6];
    __device__ void init() {
        M = 0.f;
        for (int a = 0; a < 3; ++a) S[a] = 0.f;
        for (int j = 0; j < 6; ++j) Q[j] = 0.f;
    }
    __device__ void add(float m, const float dx[3]) {
        M += m;
        int j = 0;
        for (int a = 0; a < 3; ++a) {
            float w = m * dx[a];
            S[a] += w;
            for (int b = a; b < 3; ++b, ++j) Q[j] += w * dx[b];
        }
    }
    __device__ void merge(const AccP &o) {
        M += o.M;
        for (int a = 0; a < 3; ++a) S[a] += o.S[a];
        for (int j = 0; j < 6; ++j) Q[j] += o.Q[j];
    }
};

struct AccD {
    double M, S[3], Q[6];
    __device__ void init() {
        M = 0.0;
        for (int a = 0; a < 3; ++a) S[a] = 0.0;
        for (int j = 0; j < 6; ++j) Q[j] = 0.0;
    }
    __device__ void add(double m, const double dx[3]) {
        M += m;
        int j = 0;
        for (int a = 0; a < 3; ++a) {
            double w = m * dx[a];
            S[a] += w;
            for (int b = a; b < 3; ++b, ++j) Q[j] += w * dx[b];
        }
    }
    __device__ void merge(const AccD &o) {
        M += o.M;
        for (int a = 0; a < 3; ++a) S[a] += o.S[a];
        for (int j = 0; j < 6; ++j) Q[j] += o.Q[j];
    }
};

// double-float quotient (nh + nl) / (dh + dl)
__device__ __forceinline__ void df_div(float nh, float nl, float dh, float dl, float &qh, float &ql) {
    float q1 = __fdiv_rn(nh, dh);
    float r = __fmaf_rn(-q1, dh, nh);
    r = __fadd_rn(r, nl);
    r = __fmaf_rn(-q1, dl, r);
    float q2 = __fdiv_rn(r, dh);
    fast_two_sum(q1, q2, qh, ql);
}

// ------------------------------------------------------------ writers

__device__ void write_cell_f32(const MomOut &o, int64_t c, float M, const float ch[3],
                               const float cl[3], const float Q[6], const float bb[6]) {
    o.mass[c] = M;
    for (int a = 0; a < 3; ++a) { o.com[3 * c + a] = ch[a]; o.com_lo[3 * c + a] = cl[a]; }
    for (int j = 0; j < 6; ++j) { o.quad[6 * c + j] = Q[j]; o.aabb[6 * c + j] = bb[j]; }
}

__device__ void write_cell_f64(const MomOut &o, int64_t c, double M, const double com[3],
                               const double Q[6], const float bb[6], bool has64) {
    float ch[3], cl[3], q[6];
    for (int a = 0; a < 3; ++a) {
        ch[a] = __double2float_rn(com[a]);
        cl[a] = __double2float_rn(__dsub_rn(com[a], (double)ch[a]));
    }
    for (int j = 0; j < 6; ++j) q[j] = __double2float_rn(Q[j]);
    write_cell_f32(o, c, __double2float_rn(M), ch, cl, q, bb);
    if (has64) {
        o.mass64[c] = M;
        for (int a = 0; a < 3; ++a) o.com64[3 * c + a] = com[a];
        for (int j = 0; j < 6; ++j) o.quad64[6 * c + j] = Q[j];
    }
}

// Leaf / chunk finalisation from raw sums about a reference point.
__device__ void finish_c(const MomOut &o, int64_t c, const AccC &A, const float ref[3],
                         const float bb[6]) {
    float Mh, Ml;
    fast_two_sum(A.M, A.Mc, Mh, Ml);
    float rh[3], rl[3];
    for (int a = 0; a < 3; ++a) {
        float sh, sl;
        fast_two_sum(A.S[a], A.Sc[a], sh, sl);
        if (Mh != 0.f) df_div(sh, sl, Mh, Ml, rh[a], rl[a]);
        else rh[a] = rl[a] = 0.f;
    }
    float Q[6];
    int j = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++j) {
            // Q = S2 - M c c^T about the reference point
            float t = __fmul_rn(Mh, rh[a]);
            float p, pe;
            two_prod(t, rh[b], p, pe);
            float te = __fmaf_rn(Mh, rh[a], -t);
            pe = __fmaf_rn(te, rh[b], pe);
            pe = __fmaf_rn(Mh, __fmaf_rn(rh[a], rl[b], rl[a] * rh[b]), pe);
            float qh, ql;
            two_sum(A.Q[j], -p, qh, ql);
            Q[j] = __fadd_rn(qh, __fadd_rn(ql, __fsub_rn(A.Qc[j], pe)));
        }
    float ch[3], cl[3];
    for (int a = 0; a < 3; ++a) {
        float h, l;
        two_sum(ref[a], rh[a], h, l);
        l = __fadd_rn(l, rl[a]);
        fast_two_sum(h, l, ch[a], cl[a]);
    }
    write_cell_f32(o, c, Mh + Ml, ch, cl, Q, bb);
}

__device__ void finish_p(const MomOut &o, int64_t c, const AccP &A, const float ref[3],
                         const float bb[6]) {
    float r[3], ch[3], cl[3], Q[6];
    for (int a = 0; a < 3; ++a) r[a] = (A.M != 0.f) ? A.S[a] / A.M : 0.f;
    int j = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++j) Q[j] = A.Q[j] - A.M * r[a] * r[b];
    for (int a = 0; a < 3; ++a) { ch[a] = ref[a] + r[a]; cl[a] = 0.f; }
    write_cell_f32(o, c, A.M, ch, cl, Q, bb);
}

__device__ void finish_d(const MomOut &o, int64_t c, const AccD &A, const float ref[3],
                         const float bb[6], bool has64) {
    double r[3], com[3], Q[6];
    for (int a = 0; a < 3; ++a) r[a] = (A.M != 0.0) ? A.S[a] / A.M : 0.0;
    int j = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++j) Q[j] = A.Q[j] - A.M * r[a] * r[b];
    for (int a = 0; a < 3; ++a) com[a] = (double)ref[a] + r[a];
    write_cell_f64(o, c, A.M, com, Q, bb, has64);
}

// ------------------------------------------------------------- leaves

// Sum the members [pf, pe) of one leaf from the key-ordered records; loads
// are issued four at a time before any is used.  Leaves reaching this path
// hold at most 2048 particles (longer ones, only possible at depth 21, go to
// big_leaf_kernel), so the FP32 modes never need the FP64 route here.
template <int MODE>
__device__ void leaf_sum(const MomOut &o, const float4 *__restrict__ xs, int64_t c, int64_t pf,
                         int64_t pe) {
    constexpr int G = 4;
    const float4 r0 = xs[pf];
    const float ref[3] = {r0.x, r0.y, r0.z};
    float bb[6] = {r0.x, r0.y, r0.z, r0.x, r0.y, r0.z};
    typename std::conditional<MODE == TB_MOM_FP64, AccD,
                              typename std::conditional<MODE == TB_MOM_FP32_COMP, AccC,
                                                        AccP>::type>::type A;
    A.init();
    for (int64_t k0 = pf; k0 < pe; k0 += G) {
        const int cnt = (int)min64(G, pe - k0);
        float4 v[G];
#pragma unroll
        for (int j = 0; j < G; ++j)
            if (j < cnt) v[j] = xs[k0 + j];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (j >= cnt) break;
            const float x[3] = {v[j].x, v[j].y, v[j].z};
            for (int a = 0; a < 3; ++a) {
                bb[a] = fminf(bb[a], x[a]);
                bb[3 + a] = fmaxf(bb[3 + a], x[a]);
            }
            if constexpr (MODE == TB_MOM_FP64) {
                const double dx[3] = {(double)x[0] - (double)ref[0], (double)x[1] - (double)ref[1],
                                      (double)x[2] - (double)ref[2]};
                A.add((double)v[j].w, dx);
            } else if constexpr (MODE == TB_MOM_FP32_COMP) {
                const float dx[3] = {__fsub_rn(x[0], ref[0]), __fsub_rn(x[1], ref[1]),
                                     __fsub_rn(x[2], ref[2])};
                A.add(v[j].w, dx);
            } else {
                const float dx[3] = {x[0] - ref[0], x[1] - ref[1], x[2] - ref[2]};
                A.add(v[j].w, dx);
            }
        }
    }
    if constexpr (MODE == TB_MOM_FP64) finish_d(o, c, A, ref, bb, true);
    else if constexpr (MODE == TB_MOM_FP32_COMP) finish_c(o, c, A, ref, bb);
    else finish_p(o, c, A, ref, bb);
}

// ----------------------------------------------------------- parents

// Offset of child c's centre from the reference point ref, as a
// double-float (h, l): (com_c - ref) + com_lo_c.
__device__ __forceinline__ void child_offset(const MomOut &o, int64_t c, int a, float ref, float &h,
                                             float &l) {
    float u, v;
    two_sum(o.com[3 * c + a], -ref, u, v);
    v = __fadd_rn(v, o.com_lo[3 * c + a]);
    fast_two_sum(u, v, h, l);
}

// Children [c0, c1) of p combined in FP64 (FP64 mode, or a cell of more
// than 2^20 particles in the FP32 modes).  Kept out of line so that its
// registers do not weigh on the FP32 path.
template <int MODE>
__device__ __noinline__ void combine_f64(const MomOut &o, int64_t p, int32_t c0, int32_t c1,
                                         const float bb[6]) {
        // FP64: relative to the first child's centre
        double ref[3];
        for (int a = 0; a < 3; ++a)
            ref[a] = (MODE == TB_MOM_FP64) ? o.com64[3 * (int64_t)c0 + a]
                                           : (double)o.com[3 * (int64_t)c0 + a] +
                                                 (double)o.com_lo[3 * (int64_t)c0 + a];
        auto cm = [&](int64_t c, int a) {
            return (MODE == TB_MOM_FP64) ? o.com64[3 * c + a]
                                         : (double)o.com[3 * c + a] + (double)o.com_lo[3 * c + a];
        };
        auto ms = [&](int64_t c) {
            return (MODE == TB_MOM_FP64) ? o.mass64[c] : (double)o.mass[c];
        };
        double M = 0.0, S[3] = {0, 0, 0};
        for (int32_t c = c0; c < c1; ++c) {
            double mc = ms(c);
            M += mc;
            for (int a = 0; a < 3; ++a) S[a] += mc * (cm(c, a) - ref[a]);
        }
        double r[3], com[3], Q[6] = {0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 3; ++a) {
            r[a] = (M != 0.0) ? S[a] / M : 0.0;
            com[a] = ref[a] + r[a];
        }
        for (int32_t c = c0; c < c1; ++c) {
            double mc = ms(c), e[3];
            for (int a = 0; a < 3; ++a) e[a] = (cm(c, a) - ref[a]) - r[a];
            int q = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = a; b < 3; ++b, ++q) {
                    double qc = (MODE == TB_MOM_FP64) ? o.quad64[6 * (int64_t)c + q]
                                                      : (double)o.quad[6 * (int64_t)c + q];
                    Q[q] += qc + mc * e[a] * e[b];
                }
        }
        write_cell_f64(o, p, M, com, Q, bb, MODE == TB_MOM_FP64);
}

template <int MODE>
__device__ void combine_children(const TreeIn &T, const MomOut &o, int64_t p) {
    const int32_t c0 = T.child_first[p], c1 = T.child_end[p];
    float bb[6];
    for (int a = 0; a < 6; ++a) bb[a] = o.aabb[6 * (int64_t)c0 + a];
    for (int32_t c = c0 + 1; c < c1; ++c)
        for (int a = 0; a < 3; ++a) {
            bb[a] = fminf(bb[a], o.aabb[6 * (int64_t)c + a]);
            bb[3 + a] = fmaxf(bb[3 + a], o.aabb[6 * (int64_t)c + 3 + a]);
        }
    const bool big = (int64_t)(T.pend[p] - T.pfirst[p]) > kBigCell;
    if (MODE == TB_MOM_FP64 || big) {
        combine_f64<MODE>(o, p, c0, c1, bb);
    } else if constexpr (MODE == TB_MOM_FP32_COMP) {
        float ref[3];
        for (int a = 0; a < 3; ++a) ref[a] = o.com[3 * (int64_t)c0 + a];
        // pass 1: mass and first moment about ref
        float Mh = 0.f, Mc = 0.f, Sh[3] = {0, 0, 0}, Sc[3] = {0, 0, 0};
        for (int32_t c = c0; c < c1; ++c) {
            float m = o.mass[c], e;
            two_sum(Mh, m, Mh, e);
            Mc += e;
            for (int a = 0; a < 3; ++a) {
                float h, l, pp, pe;
                child_offset(o, c, a, ref[a], h, l);
                two_prod(m, h, pp, pe);
                pe = __fmaf_rn(m, l, pe);
                two_sum(Sh[a], pp, Sh[a], e);
                Sc[a] += e + pe;
            }
        }
        float MH, ML;
        fast_two_sum(Mh, Mc, MH, ML);
        float rh[3], rl[3];
        for (int a = 0; a < 3; ++a) {
            float sh, sl;
            fast_two_sum(Sh[a], Sc[a], sh, sl);
            if (MH != 0.f) df_div(sh, sl, MH, ML, rh[a], rl[a]);
            else rh[a] = rl[a] = 0.f;
        }
        // pass 2: second moment with the parallel-axis shift
        float Q[6], Qc[6];
        for (int q = 0; q < 6; ++q) Q[q] = Qc[q] = 0.f;
        for (int32_t c = c0; c < c1; ++c) {
            const float m = o.mass[c];
            float e[3];
            for (int a = 0; a < 3; ++a) {
                float h, l;
                child_offset(o, c, a, ref[a], h, l);
                e[a] = __fadd_rn(__fsub_rn(h, rh[a]), __fsub_rn(l, rl[a]));
            }
            int q = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = a; b < 3; ++b, ++q) {
                    float sum, er;
                    two_sum(Q[q], o.quad[6 * (int64_t)c + q], sum, er);
                    Q[q] = sum;
                    Qc[q] += er;
                    float t, te, pp, pe;
                    two_prod(m, e[a], t, te);
                    two_prod(t, e[b], pp, pe);
                    pe = __fmaf_rn(te, e[b], pe);
                    two_sum(Q[q], pp, sum, er);
                    Q[q] = sum;
                    Qc[q] += er + pe;
                }
        }
        float Qf[6], ch[3], cl[3];
        for (int q = 0; q < 6; ++q) Qf[q] = __fadd_rn(Q[q], Qc[q]);
        for (int a = 0; a < 3; ++a) {
            float h, l;
            two_sum(ref[a], rh[a], h, l);
            l = __fadd_rn(l, rl[a]);
            fast_two_sum(h, l, ch[a], cl[a]);
        }
        write_cell_f32(o, p, MH + ML, ch, cl, Qf, bb);
    } else {
        float ref[3];
        for (int a = 0; a < 3; ++a) ref[a] = o.com[3 * (int64_t)c0 + a];
        float M = 0.f, S[3] = {0, 0, 0};
        for (int32_t c = c0; c < c1; ++c) {
            float m = o.mass[c];
            M += m;
            for (int a = 0; a < 3; ++a) S[a] += m * (o.com[3 * (int64_t)c + a] - ref[a]);
        }
        float r[3];
        for (int a = 0; a < 3; ++a) r[a] = (M != 0.f) ? S[a] / M : 0.f;
        float Q[6] = {0, 0, 0, 0, 0, 0};
        for (int32_t c = c0; c < c1; ++c) {
            float m = o.mass[c], e[3];
            for (int a = 0; a < 3; ++a) e[a] = (o.com[3 * (int64_t)c + a] - ref[a]) - r[a];
            int q = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = a; b < 3; ++b, ++q) Q[q] += o.quad[6 * (int64_t)c + q] + m * e[a] * e[b];
        }
        float ch[3], cl[3];
        for (int a = 0; a < 3; ++a) { ch[a] = ref[a] + r[a]; cl[a] = 0.f; }
        write_cell_f32(o, p, M, ch, cl, Q, bb);
    }
}

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

// Every cell of level d: leaves from their members, the others from their
// children (finished by the launch for level d + 1).
template <int MODE>
__global__ void __launch_bounds__(kMomThreads, 3)
    level_moments_kernel(TreeIn T, MomOut o, const float4 *__restrict__ xs, DevInfo *info, int d) {
    if (info->status & (kErrOverflow | kErrNonFinite)) return;
    const int64_t lo = info->level_offset[d], hi = info->level_offset[d + 1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < hi; c += stride) {
        if (T.child_first[c] >= 0) {
            combine_children<MODE>(T, o, c);
        } else {
            const int64_t pf = T.pfirst[c], pe = T.pend[c];
            if (d == kDepthMax && pe - pf > kBigLeafThread) {
                uint32_t q = atomicAdd(&info->misc_ctr[2], 1u);
                T.big_leaf[q] = (int32_t)c;
                continue;
            }
            leaf_sum<MODE>(o, xs, c, pf, pe);
        }
    }
}

// Block-wide sums of the long depth-21 leaves queued by the level-21 launch.
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
    cudaError_t e = cudaMemsetAsync(&ws.info->misc_ctr[2], 0, 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int64_t g = (n / 4 + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    gather_kernel<<<(unsigned)g, 256, 0, s>>>(t.perm, ws.xm, ws.xs, n, ws.info);
    ++g_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark(ws, "gather", s);
    // one persistent grid per level; a level holds at most n cells
    int64_t grid = (n + kMomThreads - 1) / kMomThreads;
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    for (int d = kDepthMax; d >= 0; --d) {
        level_moments_kernel<MODE><<<(unsigned)grid, kMomThreads, 0, s>>>(T, o, ws.xs, ws.info, d);
        ++g_launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (d == kDepthMax) {
            big_leaf_kernel<MODE><<<152, kBigThreads, 0, s>>>(T, o, ws.xs, ws.info);
            ++g_launches;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
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
