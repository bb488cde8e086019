// tb_keys.cu -- root cell and particle keys (Sec. 2.2; Sec. 2.3 step 1).
//
// root_kernel : per-axis FP32 min / max of the positions and a non-finite
//               flag; the last block to finish derives the root cube
//               (corner lo, side L = largest extent, scale 2^21 / L) and
//               resets the per-build counters.
// keys_kernel : 21-bit quantisation per axis, bit interleave below a leading
//               1, and the digit histograms of every radix-sort pass (the
//               histogram of a digit does not depend on the order of the
//               keys, so all passes are counted in this one read).  The last
//               block turns the histograms into exclusive digit offsets.
//
// Both read the [n][3] FP32 positions four particles (three float4) per
// thread step when the array is 16-byte aligned.
#include <cfloat>
#include <cmath>

#include "tb_device.cuh"

namespace tb {

namespace {

constexpr int kRootThreads = 256;
constexpr int kKeysThreads = 256;

__device__ __forceinline__ bool finite_f(float x) { return fabsf(x) <= FLT_MAX; }

struct Box {
    float mn[3], mx[3];
    uint32_t bad;
    __device__ void init() {
        for (int a = 0; a < 3; ++a) { mn[a] = FLT_MAX; mx[a] = -FLT_MAX; }
        bad = 0;
    }
    __device__ void add(float x, int a) {
        bad |= !finite_f(x);
        mn[a] = fminf(mn[a], x);
        mx[a] = fmaxf(mx[a], x);
    }
};

__global__ void __launch_bounds__(kRootThreads) root_kernel(const float *__restrict__ pos, int64_t n,
                                                            bool vec, float *__restrict__ part,
                                                            DevInfo *info, uint32_t *hist,
                                                            int hist_len, bool pow2) {
    Box b;
    b.init();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const float4 *p4 = reinterpret_cast<const float4 *>(pos);
        const int64_t groups = n / 4;
#pragma unroll 2
        for (int64_t g = tid; g < groups; g += stride) {
            float4 a = __ldcs(p4 + 3 * g), c = __ldcs(p4 + 3 * g + 1), d = __ldcs(p4 + 3 * g + 2);
            b.add(a.x, 0); b.add(a.y, 1); b.add(a.z, 2); b.add(a.w, 0);
            b.add(c.x, 1); b.add(c.y, 2); b.add(c.z, 0); b.add(c.w, 1);
            b.add(d.x, 2); b.add(d.y, 0); b.add(d.z, 1); b.add(d.w, 2);
        }
        done = groups * 4;
    }
    for (int64_t i = done + tid; i < n; i += stride)
        for (int a = 0; a < 3; ++a) b.add(pos[3 * i + a], a);

    // block reduction
    for (int off = 16; off > 0; off >>= 1) {
        for (int a = 0; a < 3; ++a) {
            b.mn[a] = fminf(b.mn[a], __shfl_xor_sync(0xffffffffu, b.mn[a], off));
            b.mx[a] = fmaxf(b.mx[a], __shfl_xor_sync(0xffffffffu, b.mx[a], off));
        }
        b.bad |= __shfl_xor_sync(0xffffffffu, b.bad, off);
    }
    __shared__ float s_red[kRootThreads / 32][8];
    __shared__ bool s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) { s_red[warp][a] = b.mn[a]; s_red[warp][3 + a] = b.mx[a]; }
        s_red[warp][6] = __uint_as_float(b.bad);
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        float v = s_red[0][threadIdx.x];
        for (int w = 1; w < kRootThreads / 32; ++w) {
            float u = s_red[w][threadIdx.x];
            if (threadIdx.x < 3) v = fminf(v, u);
            else if (threadIdx.x < 6) v = fmaxf(v, u);
            else v = __uint_as_float(__float_as_uint(v) | __float_as_uint(u));
        }
        part[blockIdx.x * 8 + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&info->misc_ctr[0], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: combine the per-block partials and derive the root cube
    // every thread folds a stride of the partials, then the block reduces
    {
        Box c;
        c.init();
        for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
            const float4 lo = __ldcg(reinterpret_cast<const float4 *>(part + 8 * k));
            const float4 hi = __ldcg(reinterpret_cast<const float4 *>(part + 8 * k + 4));
            c.mn[0] = fminf(c.mn[0], lo.x); c.mn[1] = fminf(c.mn[1], lo.y); c.mn[2] = fminf(c.mn[2], lo.z);
            c.mx[0] = fmaxf(c.mx[0], lo.w); c.mx[1] = fmaxf(c.mx[1], hi.x); c.mx[2] = fmaxf(c.mx[2], hi.y);
            c.bad |= __float_as_uint(hi.z);
        }
        for (int off = 16; off > 0; off >>= 1) {
            for (int a = 0; a < 3; ++a) {
                c.mn[a] = fminf(c.mn[a], __shfl_xor_sync(0xffffffffu, c.mn[a], off));
                c.mx[a] = fmaxf(c.mx[a], __shfl_xor_sync(0xffffffffu, c.mx[a], off));
            }
            c.bad |= __shfl_xor_sync(0xffffffffu, c.bad, off);
        }
        __syncthreads();   // s_red's block partials were read above
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) { s_red[warp][a] = c.mn[a]; s_red[warp][3 + a] = c.mx[a]; }
            s_red[warp][6] = __uint_as_float(c.bad);
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            float v = s_red[0][threadIdx.x];
            for (int w = 1; w < kRootThreads / 32; ++w) {
                const float u = s_red[w][threadIdx.x];
                if (threadIdx.x < 3) v = fminf(v, u);
                else if (threadIdx.x < 6) v = fmaxf(v, u);
                else v = __uint_as_float(__float_as_uint(v) | __float_as_uint(u));
            }
            s_red[0][threadIdx.x] = v;
        }
    }
    for (int i = threadIdx.x; i < hist_len; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t bad = __float_as_uint(s_red[0][6]);
        double L = 0.0;
        float amax = 0.f;
        for (int a = 0; a < 3; ++a) {
            info->lo[a] = s_red[0][a];
            info->hi[a] = s_red[0][3 + a];
            double e = __dsub_rn((double)s_red[0][3 + a], (double)s_red[0][a]);
            if (e > L) L = e;
            amax = fmaxf(amax, fmaxf(fabsf(s_red[0][a]), fabsf(s_red[0][3 + a])));
        }
        if (!(L > 0.0)) L = 1.0;
        if (pow2) L = pow2_ceil(L);
        double scale = __ddiv_rn(2097152.0, L);
        float s_hi = (float)scale;
        float s_lo = (float)__dsub_rn(scale, (double)s_hi);
        info->side = L;
        info->scale = scale;
        info->s_hi = s_hi;
        info->s_lo = s_lo;
        // the FP32 route needs x - lo and its products to stay far from overflow
        // and underflow; otherwise every coordinate takes the FP64 route
        info->exact_only = !(scale < 1e30 && scale > 1e-30 && amax < 1e30f) ? 1u : 0u;
        info->s_fp32 = (double)s_hi == scale ? 1u : 0u;
        info->status = bad ? kErrNonFinite : 0u;
        info->epoch = (info->epoch + 16u) & 0x3fffffffu;
        for (int p = 0; p < 16; ++p) info->sort_tile_ctr[p] = 0;
        for (int p = 1; p < 8; ++p) info->misc_ctr[p] = 0;
        info->n_cells = 0;
        info->n_leaves = 0;
        info->max_depth = 0;
        __threadfence();
        info->misc_ctr[0] = 0;
    }
}

template <int RADIX_BITS, bool HILBERT>
__global__ void __launch_bounds__(kKeysThreads, 6) keys_kernel(const float *__restrict__ pos,
                                                            const float *__restrict__ mass,
                                                            float m_eq, int64_t n, bool vec,
                                                            uint64_t *__restrict__ keys,
                                                            float4 *__restrict__ xm,
                                                            uint32_t *hist, int passes, int shift0,
                                                            DevInfo *info) {
    constexpr int RADIX = 1 << RADIX_BITS;
    extern __shared__ uint32_t s_hist[];   // [passes][RADIX]
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) s_hist[i] = 0;
    __shared__ float s_lo[3];
    __shared__ float s_shi, s_slo;
    __shared__ double s_scale;
    __shared__ bool s_exact, s_f32, s_last;
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) s_lo[a] = info->lo[a];
        s_shi = info->s_hi;
        s_slo = info->s_lo;
        s_scale = info->scale;
        s_exact = info->exact_only != 0;
        s_f32 = info->s_fp32 != 0;
    }
    __syncthreads();
    const float lx = s_lo[0], ly = s_lo[1], lz = s_lo[2];
    const float shi = s_shi, slo = s_slo;
    const double sc = s_scale;
    const bool exact = s_exact, f32 = s_f32;

    auto count = [&](uint64_t k) {
        for (int p = 0; p < passes; ++p)
            atomicAdd(&s_hist[p * RADIX + (int)((k >> (shift0 + p * RADIX_BITS)) & (RADIX - 1))], 1u);
    };
    auto key_of = [&](float x, float y, float z) {
        const uint32_t qx = quantise(x, lx, shi, slo, sc, exact, f32),
                       qy = quantise(y, ly, shi, slo, sc, exact, f32),
                       qz = quantise(z, lz, shi, slo, sc, exact, f32);
        return HILBERT ? hilbert_key(qx, qy, qz) : morton_key(qx, qy, qz);
    };

    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const float4 *p4 = reinterpret_cast<const float4 *>(pos);
        ulonglong2 *k2 = reinterpret_cast<ulonglong2 *>(keys);
        const int64_t groups = n / 4;
        const float4 *m4 = reinterpret_cast<const float4 *>(mass);
        for (int64_t g = tid; g < groups; g += stride) {
            float4 a = __ldcs(p4 + 3 * g), c = __ldcs(p4 + 3 * g + 1), d = __ldcs(p4 + 3 * g + 2);
            float4 w = mass ? __ldcs(m4 + g) : make_float4(m_eq, m_eq, m_eq, m_eq);
            uint64_t k0 = key_of(a.x, a.y, a.z);
            uint64_t k1 = key_of(a.w, c.x, c.y);
            uint64_t k2v = key_of(c.z, c.w, d.x);
            uint64_t k3 = key_of(d.y, d.z, d.w);
            k2[2 * g] = make_ulonglong2(k0, k1);
            k2[2 * g + 1] = make_ulonglong2(k2v, k3);
            xm[4 * g] = make_float4(a.x, a.y, a.z, w.x);
            xm[4 * g + 1] = make_float4(a.w, c.x, c.y, w.y);
            xm[4 * g + 2] = make_float4(c.z, c.w, d.x, w.z);
            xm[4 * g + 3] = make_float4(d.y, d.z, d.w, w.w);
            count(k0); count(k1); count(k2v); count(k3);
        }
        done = groups * 4;
    }
    for (int64_t i = done + tid; i < n; i += stride) {
        float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        uint64_t k = key_of(x, y, z);
        keys[i] = k;
        xm[i] = make_float4(x, y, z, mass ? mass[i] : m_eq);
        count(k);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&info->misc_ctr[4], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: counts -> exclusive offsets, one pass at a time
    __shared__ uint32_t s_warp[kKeysThreads / 32];
    for (int p = 0; p < passes; ++p) {
        uint32_t carry = 0;
        for (int base = 0; base < RADIX; base += kKeysThreads) {
            int d = base + threadIdx.x;
            uint32_t v = (d < RADIX) ? __ldcg(&hist[p * RADIX + d]) : 0u;
            uint32_t x = v;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int off = 1; off < 32; off <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            if (lane == 31) s_warp[warp] = x;
            __syncthreads();
            uint32_t wpre = 0, tot = 0;
            for (int w = 0; w < kKeysThreads / 32; ++w) {
                if (w < warp) wpre += s_warp[w];
                tot += s_warp[w];
            }
            if (d < RADIX) hist[p * RADIX + d] = carry + wpre + x - v;
            carry += tot;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) info->misc_ctr[4] = 0;
}

}  // namespace

int64_t bbox_grid() { return 152 * 4; }

cudaError_t launch_root(const float *pos, int64_t n, Workspace &ws, int hist_len, cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(pos) & 15u) == 0;
    int64_t grid = bbox_grid();
    int64_t need = (n + 4 * kRootThreads - 1) / (4 * kRootThreads);
    if (need < grid) grid = need < 1 ? 1 : need;
    root_kernel<<<(unsigned)grid, kRootThreads, 0, s>>>(pos, n, vec, ws.bbox_part, ws.info, ws.hist,
                                                        hist_len, ws.root_pow2);
    ++g_launches;
    return cudaGetLastError();
}

template <int B, bool H>
static cudaError_t keys_impl(const float *pos, const float *mass, int64_t n, uint64_t *keys,
                             Workspace &ws, int passes, int shift0, cudaStream_t s) {
    const bool vec = (reinterpret_cast<uintptr_t>(pos) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(mass) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    const float m_eq = (float)(1.0 / (double)(n > 0 ? n : 1));
    size_t smem = sizeof(uint32_t) * passes * (1 << B);
    static std::atomic<uint64_t> attr_done{0};
    if (first_on_device(attr_done)) {
        cudaFuncSetAttribute(keys_kernel<B, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    }
    // six resident blocks per SM (42 registers), one wave
    int64_t grid = 152 * 6;
    int64_t need = (n + 4 * kKeysThreads - 1) / (4 * kKeysThreads);
    if (need < grid) grid = need < 1 ? 1 : need;
    keys_kernel<B, H><<<(unsigned)grid, kKeysThreads, smem, s>>>(pos, mass, m_eq, n, vec, keys, ws.xm,
                                                              ws.hist, passes, shift0, ws.info);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_keys(const float *pos, const float *mass, int64_t n, uint64_t *keys,
                        Workspace &ws, const SortCfg &cfg, int key_order, cudaStream_t s) {
    const SortPlan plan = sort_plan(cfg);
    const int passes = plan.passes, shift0 = plan.shift0;
    const bool h = key_order == TB_KEYS_HILBERT;
    switch (cfg.radix_bits) {
        case 8: return h ? keys_impl<8, true>(pos, mass, n, keys, ws, passes, shift0, s)
                         : keys_impl<8, false>(pos, mass, n, keys, ws, passes, shift0, s);
        case 9: return h ? keys_impl<9, true>(pos, mass, n, keys, ws, passes, shift0, s)
                         : keys_impl<9, false>(pos, mass, n, keys, ws, passes, shift0, s);
        case 10: return h ? keys_impl<10, true>(pos, mass, n, keys, ws, passes, shift0, s)
                          : keys_impl<10, false>(pos, mass, n, keys, ws, passes, shift0, s);
        case 11: return h ? keys_impl<11, true>(pos, mass, n, keys, ws, passes, shift0, s)
                          : keys_impl<11, false>(pos, mass, n, keys, ws, passes, shift0, s);
        default: return cudaErrorInvalidValue;
    }
}

// (x, y, z, m) of each particle in input order, for moment calls whose
// arrays differ from the ones the keys were made from.
__global__ void pack_kernel(const float *__restrict__ pos, const float *__restrict__ mass,
                            float m_eq, int64_t n, float4 *__restrict__ xm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        xm[i] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], mass ? mass[i] : m_eq);
}

cudaError_t launch_pack(const float *pos, const float *mass, int64_t n, float4 *xm,
                        cudaStream_t s) {
    const float m_eq = (float)(1.0 / (double)(n > 0 ? n : 1));
    int64_t grid = (n + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    pack_kernel<<<(unsigned)grid, 256, 0, s>>>(pos, mass, m_eq, n, xm);
    ++g_launches;
    return cudaGetLastError();
}


}  // namespace tb
