// tb_device.cuh -- device-side building blocks shared by the tree kernels.
//
// Nothing here is a kernel.  It holds the key arithmetic of Sec. 2.2, the
// minimum distinguished depth of Sec. 2.3.1, the FP32 error-free transforms
// used by the compensated moments, and the bounded wait every spin uses.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tb_internal.h"

namespace tb {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// ----------------------------------------------------------------- keys

// Minimum distinguished depth (Sec. 2.3.1): ceil(clz(a ^ b) / 3); __clzll(0)
// is 64, so identical keys give 22 ("never separated").
__device__ __forceinline__ int min_depth(uint64_t a, uint64_t b) {
    return (__clzll(a ^ b) + 2) / 3;
}

// The smallest power of two >= L, for L > 0 (the power-of-two root cube of
// Sec. 2.2): L = m 2^e with m in [1/2, 1), exactly.
__device__ __forceinline__ double pow2_ceil(double L) {
    int e;
    const double m = frexp(L, &e);
    return m == 0.5 ? L : ldexp(1.0, e);
}

// Depth-d cell key of a particle key: its upper 3d+1 bits (Sec. 2.3.1).
__device__ __forceinline__ uint64_t cell_key(uint64_t key, int d) {
    return key >> (63 - 3 * d);
}

// Spread bits 0..9 of v to every third bit (bit b -> bit 3b), in 32-bit
// words.
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Key: a leading 1, then the 21 octant digits, x the most significant bit
// of each digit (Sec. 2.2).  Interleaved in 32-bit pieces: key bits 0..29
// from coordinate bits 0..9, bits 30..59 from bits 10..19, 60..62 from bit 20.
__device__ __forceinline__ uint64_t morton_key(uint32_t qx, uint32_t qy, uint32_t qz) {
    const uint32_t lo = (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
    const uint32_t hx = qx >> 10, hy = qy >> 10, hz = qz >> 10;
    const uint32_t hi = (spread10(hx) << 2) | (spread10(hy) << 1) | spread10(hz);
    const uint32_t top = ((hx >> 10) << 2) | ((hy >> 10) << 1) | (hz >> 10);
    return (1ull << 63) | ((uint64_t)top << 60) | ((uint64_t)hi << 30) | lo;
}

// Peano-Hilbert key (the alternative order of the footnote in Sec. 2.2):
// Skilling's transform of the coordinates (J. Skilling, AIP Conf. Proc. 707,
// 381, 2004) -- from the top level down, an axis whose bit is set inverts the
// lower bits of the first axis, any other axis swaps its lower bits with the
// first axis's; then a Gray code across the axes and a correction by the
// parity of the last axis -- interleaved like a Morton key.  The points of a
// depth-d cube keep a common key prefix, so the whole pipeline takes these
// keys unchanged.
__device__ __forceinline__ uint64_t hilbert_key(uint32_t x, uint32_t y, uint32_t z) {
#pragma unroll
    for (int lev = 20; lev >= 1; --lev) {
        const uint32_t Q = 1u << lev, P = Q - 1;
        x ^= (x & Q) ? P : 0u;
        const uint32_t ty = (x ^ y) & P;
        const bool by = (y & Q) != 0u;
        x ^= by ? P : ty;
        y ^= by ? 0u : ty;
        const uint32_t tz = (x ^ z) & P;
        const bool bz = (z & Q) != 0u;
        x ^= bz ? P : tz;
        z ^= bz ? 0u : tz;
    }
    y ^= x;
    z ^= y;
    uint32_t t = 0;
#pragma unroll
    for (int lev = 20; lev >= 1; --lev)
        if (z & (1u << lev)) t ^= (1u << lev) - 1u;
    return morton_key(x ^ t, y ^ t, z ^ t);
}

// Exact error-free sum a + b = s + e (Knuth's TwoSum, no branch).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b when |a| >= |b| (Dekker's Fast2Sum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Exact product a * b = p + e with one FMA.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// 21-bit quantisation of one coordinate, equal bit for bit to the FP64
// definition q = min(2^21-1, floor(fl64(fl64(x - lo) * s))).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the product is
// formed in FP32 double-float arithmetic: x - lo = dh + dl exactly (TwoSum),
// s ~ s_hi + s_lo, t ~ p + c with p = fl32(dh * s_hi).  The estimate is within
// 2^-22 of the FP64 value for t < 2^21.  When the fractional part of the
// estimate lies within 2^-18 of an integer the floor is ambiguous.  If s is an
// FP32 value (s_fp32: s == s_hi) and x - lo is one too (dl == 0), the product
// dh * s_hi = p + e (TwoProd) is exact, holds at most 48 significant bits and
// so equals its FP64 rounding: its floor is floor(p), less one when p is an
// integer and e < 0 (|e| is at most half an ulp of p, below 1/2).  Otherwise
// the FP64 operations themselves decide (a few particles in 10^5 on the tree
// workloads; every coordinate of an input on a grid aligned with a
// power-of-two root cube takes the exact FP32 route instead).
__device__ __forceinline__ uint32_t quantise(float x, float lo, float s_hi, float s_lo, double s,
                                             bool exact_only, bool s_fp32) {
    if (!exact_only) {
        float dh, dl;
        two_sum(x, -lo, dh, dl);
        float p, e;
        two_prod(dh, s_hi, p, e);
        float c = __fmaf_rn(dh, s_lo, __fmaf_rn(dl, s_hi, __fmaf_rn(dl, s_lo, e)));
        float fl = floorf(p);
        float f = __fadd_rn(__fsub_rn(p, fl), c);
        float k = floorf(f);
        float r = __fsub_rn(f, k);
        const float delta = 3.814697265625e-06f;  // 2^-18
        if (r > delta && r < 1.0f - delta) {
            float q = __fadd_rn(fl, k);
            if (q < 0.f) q = 0.f;
            if (q > 2097151.f) q = 2097151.f;
            return (uint32_t)q;
        }
        if (s_fp32 && dl == 0.f) {
            float q = (fl == p && e < 0.f) ? __fsub_rn(fl, 1.0f) : fl;
            if (q < 0.f) q = 0.f;
            if (q > 2097151.f) q = 2097151.f;
            return (uint32_t)q;
        }
    }
    double d = __dsub_rn((double)x, (double)lo);
    double t = __dmul_rn(d, s);
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    return (uint32_t)f;
}

// ------------------------------------------------------- bounded waits

// Spin limit for every wait on another block.  A wait that runs out sets
// TB_ERR_TIMEOUT in the status word and returns false; callers then carry
// on with a harmless value so that no block waits forever.
__device__ __forceinline__ bool poll_backoff(int64_t &iter, int64_t limit) {
    if (++iter > limit) return false;
    if (iter > 64) __nanosleep(iter > 4096 ? 256 : 32);
    return true;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void flag_error(uint32_t *status, uint32_t bit) {
    atomicOr(status, bit);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------ bulk copies (TMA, 1-D)

// Shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes an mbarrier's initialisation visible to the asynchronous (bulk copy)
// proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrives on the barrier (one of its expected arrivals) and adds `bytes` to
// the transfer count its current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier to complete, giving up after
// `limit` polls (each poll may itself suspend for a while); returns false
// when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int64_t limit) {
    for (int64_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned, source in this GPU's memory), completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared -> global bulk copy (same size and alignment rules), tracked by the
// issuing thread's bulk group.
__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// The issuing thread waits until its bulk stores have read their shared
// memory source (the block may then reuse it or exit).
__device__ __forceinline__ void bulk_store_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Asynchronous 16-byte global -> shared copy (no registers held while it is
// in flight); completion is awaited with cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later bulk
// copies (the asynchronous proxy) that touch the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace tb
