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
    const int32_t *parent;   // each cell's parent, -1 for the root
};

// The FP32 moments of cells (mass, centre of mass and its low part, second
// moment, bounding box) as a parent's combination reads its children's:
// straight from the tree's arrays ...
struct CellsGlobal {
    const float *mass, *com, *com_lo, *quad, *aabb;
    __device__ __forceinline__ float m(int64_t c) const { return mass[c]; }
    __device__ __forceinline__ float x(int64_t c, int a) const { return com[3 * c + a]; }
    __device__ __forceinline__ float xl(int64_t c, int a) const { return com_lo[3 * c + a]; }
    // rows of six (xx xy xz yy yz zz; lo xyz hi xyz) as three float2
    __device__ __forceinline__ float2 q2(int64_t c, int i) const {
        return reinterpret_cast<const float2 *>(quad + 6 * c)[i];
    }
    __device__ __forceinline__ float2 b2(int64_t c, int i) const {
        return reinterpret_cast<const float2 *>(aabb + 6 * c)[i];
    }
};
__device__ __forceinline__ CellsGlobal cells_of(const MomOut &o) {
    return {o.mass, o.com, o.com_lo, o.quad, o.aabb};
}

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
    // a child cell of mass m, centre ref + (h + l), central second moment q:
    // its mass, first moment and second moment about the reference point
    __device__ void add_cell(float m, const float h[3], const float l[3], const float q[6]) {
        float e;
        two_sum(M, m, M, e);
        Mc += e;
        float p[3], pe[3];
        for (int a = 0; a < 3; ++a) {
            two_prod(m, h[a], p[a], pe[a]);
            pe[a] = __fmaf_rn(m, l[a], pe[a]);
            two_sum(S[a], p[a], S[a], e);
            Sc[a] += e + pe[a];
        }
        int j = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b, ++j) {
                float e1, t, te;
                two_sum(Q[j], q[j], Q[j], e1);
                two_prod(p[a], h[b], t, te);
                te = __fmaf_rn(pe[a], h[b], te);
                te = __fmaf_rn(p[a], l[b], te);
                two_sum(Q[j], t, Q[j], e);
                Qc[j] += (e1 + e) + te;
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

// Parents in the compensated mode: mass and first moment compensated (their
// errors would otherwise add up over 21 levels), second moment plain -- a
// parent's second-moment error relative to M s^2 is at most about 54 u from
// its own sum and a quarter of each child's (whose side is half), so it stays
// below 72 u (4.3e-6), under the 1e-5 tolerance, at every level.
struct AccS {
    float M, Mc, S[3], Sc[3], Q[6];
    __device__ void init() {
        M = Mc = 0.f;
        for (int a = 0; a < 3; ++a) S[a] = Sc[a] = 0.f;
        for (int j = 0; j < 6; ++j) Q[j] = 0.f;
    }
    // a child of mass m, centre ref + (h + l), central second moment q
    __device__ void add_cell(float m, const float h[3], const float l[3], const float q[6]) {
        float e;
        two_sum(M, m, M, e);
        Mc += e;
        float p[3];
        for (int a = 0; a < 3; ++a) {
            float pe;
            two_prod(m, h[a], p[a], pe);
            pe = __fmaf_rn(m, l[a], pe);
            two_sum(S[a], p[a], S[a], e);
            Sc[a] += e + pe;
        }
        int j = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b, ++j) Q[j] = __fmaf_rn(p[a], h[b], __fadd_rn(Q[j], q[j]));
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
    // quad and aabb rows are 24 bytes, 8-byte aligned
    float2 *q2 = reinterpret_cast<float2 *>(o.quad + 6 * c);
    float2 *b2 = reinterpret_cast<float2 *>(o.aabb + 6 * c);
    for (int j = 0; j < 3; ++j) {
        q2[j] = make_float2(Q[2 * j], Q[2 * j + 1]);
        b2[j] = make_float2(bb[2 * j], bb[2 * j + 1]);
    }
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

__device__ void finish_s(const MomOut &o, int64_t c, const AccS &A, const float ref[3],
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
        for (int b = a; b < 3; ++b, ++j) Q[j] = __fmaf_rn(-__fmul_rn(Mh, rh[a]), rh[b], A.Q[j]);
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

// Compensated-mode leaves of at most this many members are summed with two
// interleaved plain FP32 accumulators (even and odd members) instead.  With
// u = 2^-24 and every member within one cell side s of the reference point on
// each axis, each half-sum of at most 8 terms plus its products and the final
// merge err by at most 9 u sum|terms|: 9 u M on the mass, 10 u s on the
// centre of mass, 12 u M s^2 on the second moment (1e-6 s and 1e-6 M s^2 or
// less), inside the tolerances the compensated parents carry upward.
constexpr int kSplitLeaf = 16;

__device__ void finish_split(const MomOut &o, int64_t c, const AccP &A, const AccP &B,
                             const float ref[3], const float bb[6]) {
    const float M = __fadd_rn(A.M, B.M);
    float r[3], Q[6], ch[3], cl[3];
    for (int a = 0; a < 3; ++a) r[a] = (M != 0.f) ? __fdiv_rn(__fadd_rn(A.S[a], B.S[a]), M) : 0.f;
    int j = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++j)
            Q[j] = __fmaf_rn(-__fmul_rn(M, r[a]), r[b], __fadd_rn(A.Q[j], B.Q[j]));
    for (int a = 0; a < 3; ++a) {
        float h, l;
        two_sum(ref[a], r[a], h, l);
        fast_two_sum(h, l, ch[a], cl[a]);
    }
    write_cell_f32(o, c, M, ch, cl, Q, bb);
}

// Records of the particles in key order read through the permutation:
// src[k] = xm[perm[k]], the (x, y, z, m) of the k-th particle in key order
// (Sec. 2.3 step 3) without writing the reordered array.
struct PermSrc {
    const float4 *__restrict__ xm;
    const int32_t *__restrict__ perm;
    __device__ __forceinline__ float4 operator[](int64_t k) const { return __ldg(xm + perm[k]); }
};

// A leaf of at most kSplitLeaf members in the compensated mode: two
// interleaved plain FP32 accumulators (see kSplitLeaf).  `xs` is any source
// of key-ordered records indexed by position: a pointer (global or shared
// memory) or a PermSrc.
template <class Src>
__device__ __forceinline__ void leaf_sum_split(const MomOut &o, Src xs, int64_t c, int64_t pf,
                                               int64_t pe) {
    constexpr int G = 4;
    const float4 r0 = xs[pf];
    const float ref[3] = {r0.x, r0.y, r0.z};
    float bb[6] = {r0.x, r0.y, r0.z, r0.x, r0.y, r0.z};
    AccP A, B;
    A.init();
    B.init();
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
            const float dx[3] = {__fsub_rn(x[0], ref[0]), __fsub_rn(x[1], ref[1]),
                                 __fsub_rn(x[2], ref[2])};
            if (j & 1) B.add(v[j].w, dx);
            else A.add(v[j].w, dx);
        }
    }
    finish_split(o, c, A, B, ref, bb);
}

// Sum the members [pf, pe) of one leaf from the key-ordered records; loads
// are issued four at a time before any is used.  Leaves reaching this path
// hold at most 2048 particles (longer ones, only possible at depth 21, go to
// big_leaf_kernel), so the FP32 modes never need the FP64 route here.
template <int MODE, class Src>
__device__ void leaf_sum(const MomOut &o, Src xs, int64_t c, int64_t pf, int64_t pe) {
    constexpr int G = 4;
    const float4 r0 = xs[pf];
    const float ref[3] = {r0.x, r0.y, r0.z};
    float bb[6] = {r0.x, r0.y, r0.z, r0.x, r0.y, r0.z};
    if constexpr (MODE == TB_MOM_FP32_COMP) {
        if (pe - pf <= kSplitLeaf) {
            leaf_sum_split(o, xs, c, pf, pe);
            return;
        }
    }
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
template <class Src>
__device__ __forceinline__ void child_offset(const Src &o, int64_t c, int a, float ref, float &h,
                                             float &l) {
    float u, v;
    two_sum(o.x(c, a), -ref, u, v);
    v = __fadd_rn(v, o.xl(c, a));
    fast_two_sum(u, v, h, l);
}

// Children [c0, c1) of p combined in FP64 (FP64 mode, or a cell of more
// than 2^20 particles in the FP32-plain mode).  Kept out of line so that its
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

// Parent p from its children, whose FP32 moments come from `src` (the tree's
// arrays, or a copy staged in shared memory); the FP64 route reads the tree's
// arrays.
template <int MODE, class Src>
__device__ void combine_children(const TreeIn &T, const MomOut &o, int64_t p, const Src &src) {
    const int32_t c0 = T.child_first[p], c1 = T.child_end[p];
    auto qrow = [&](int64_t c, float v[6]) {
        const float2 x = src.q2(c, 0), y = src.q2(c, 1), z = src.q2(c, 2);
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y; v[4] = z.x; v[5] = z.y;
    };
    auto brow = [&](int64_t c, float v[6]) {
        const float2 x = src.b2(c, 0), y = src.b2(c, 1), z = src.b2(c, 2);
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y; v[4] = z.x; v[5] = z.y;
    };
    auto grow = [](float bb[6], const float cb[6]) {
        for (int a = 0; a < 3; ++a) {
            bb[a] = fminf(bb[a], cb[a]);
            bb[3 + a] = fmaxf(bb[3 + a], cb[3 + a]);
        }
    };
    float bb[6];
    brow(c0, bb);
    if constexpr (MODE == TB_MOM_FP32_COMP) {
        {
            // one pass: mass, first and second moments about the first
            // child's centre, then the shift to the centre of mass (as for a
            // leaf).  The sums are compensated, and a parent's error is
            // relative to its own mass and size whatever its particle count,
            // so cells of any size take this route.
            float ref[3];
            for (int a = 0; a < 3; ++a) ref[a] = src.x(c0, a);
            AccS A;
            A.init();
            for (int32_t c = c0; c < c1; ++c) {
                float h[3], l[3], q[6], cb[6];
                for (int a = 0; a < 3; ++a) child_offset(src, c, a, ref[a], h[a], l[a]);
                qrow(c, q);
                if (c > c0) {
                    brow(c, cb);
                    grow(bb, cb);
                }
                A.add_cell(src.m(c), h, l, q);
            }
            finish_s(o, p, A, ref, bb);
            return;
        }
    }
    for (int32_t c = c0 + 1; c < c1; ++c) {
        float cb[6];
        brow(c, cb);
        grow(bb, cb);
    }
    const bool big = (int64_t)(T.pend[p] - T.pfirst[p]) > kBigCell;
    if (MODE == TB_MOM_FP64 || big) {
        combine_f64<MODE>(o, p, c0, c1, bb);
    } else {
        float ref[3];
        for (int a = 0; a < 3; ++a) ref[a] = src.x(c0, a);
        float M = 0.f, S[3] = {0, 0, 0};
        for (int32_t c = c0; c < c1; ++c) {
            float m = src.m(c);
            M += m;
            for (int a = 0; a < 3; ++a) S[a] += m * (src.x(c, a) - ref[a]);
        }
        float r[3];
        for (int a = 0; a < 3; ++a) r[a] = (M != 0.f) ? S[a] / M : 0.f;
        float Q[6] = {0, 0, 0, 0, 0, 0};
        for (int32_t c = c0; c < c1; ++c) {
            float m = src.m(c), e[3], qc[6];
            for (int a = 0; a < 3; ++a) e[a] = (src.x(c, a) - ref[a]) - r[a];
            qrow(c, qc);
            int q = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = a; b < 3; ++b, ++q) Q[q] += qc[q] + m * e[a] * e[b];
        }
        float ch[3], cl[3];
        for (int a = 0; a < 3; ++a) { ch[a] = ref[a] + r[a]; cl[a] = 0.f; }
        write_cell_f32(o, p, M, ch, cl, Q, bb);
    }
}


}  // namespace
}  // namespace tb
