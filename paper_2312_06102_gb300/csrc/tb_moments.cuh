// tb_moments.cuh -- moment arithmetic shared by the single-tree and the
// batched builds: compensated / plain / FP64 accumulators, the finishing of
// a leaf's sums, and the combination of a parent from its children.  See
// tb_moments.cu for the method.
#pragma once

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


}  // namespace
}  // namespace tb
