// tb_reorder.cu -- per-particle arrays into key order (Sec. 2.3 step 3).
//
// dst[k] = src[perm[k]], one row of row_bytes per particle.  Rows are moved
// in the widest word that divides them and the arrays' alignment (16, 8 or
// 4 bytes); every thread keeps four rows in flight, since with unordered
// input each row is a random read.
#include "tb_internal.h"

namespace tb {

namespace {

template <class W>
__global__ void __launch_bounds__(256)
    reorder_kernel(const int32_t *__restrict__ perm, const W *__restrict__ src, W *__restrict__ dst,
                   int64_t n, int words) {
    const int64_t total = n * words;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); g0 < total; g0 += 4 * stride) {
        W v[4];
        int64_t at[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t g = g0 + j * stride;
            at[j] = g;
            if (g < total) {
                const int64_t k = g / words;
                const int w = (int)(g - k * words);
                v[j] = __ldg(src + (int64_t)perm[k] * words + w);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (at[j] < total) dst[at[j]] = v[j];
    }
}

template <class W>
cudaError_t launch(const int32_t *perm, const void *src, void *dst, int64_t n, int64_t row_bytes,
                   cudaStream_t s) {
    const int words = (int)(row_bytes / (int64_t)sizeof(W));
    const int64_t total = n * words;
    int64_t grid = (total / 4 + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    reorder_kernel<W><<<(unsigned)grid, 256, 0, s>>>(perm, static_cast<const W *>(src),
                                                    static_cast<W *>(dst), n, words);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace

}  // namespace tb

using namespace tb;

extern "C" tb_status tb_reorder(const tb_tree *tree, const void *d_src, void *d_dst, int64_t row_bytes,
                                tb_stream stream) {
    if (!tree || tree->n_sets != 0 || row_bytes <= 0 || (row_bytes & 3) || row_bytes > (1 << 20))
        return TB_EINVAL;
    const int64_t n = tree->n_particles;
    if (n == 0) return TB_OK;
    if (!d_src || !d_dst || !tree->perm) return TB_EINVAL;
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_src), b = reinterpret_cast<uintptr_t>(d_dst);
    if ((a & 3) || (b & 3)) return TB_EINVAL;
    const uintptr_t bytes = (uintptr_t)n * (uintptr_t)row_bytes;
    if (a < b + bytes && b < a + bytes) return TB_EINVAL;   // overlapping arrays
    // the permutation is complete only after a build that enqueued every stage
    const Workspace *ws = static_cast<const Workspace *>(tree->internal);
    if (!ws || !ws->cells_ready) return TB_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (row_bytes % 16 == 0 && ((a | b) & 15) == 0)
        e = launch<uint4>(tree->perm, d_src, d_dst, n, row_bytes, s);
    else if (row_bytes % 8 == 0 && ((a | b) & 7) == 0)
        e = launch<uint2>(tree->perm, d_src, d_dst, n, row_bytes, s);
    else
        e = launch<uint32_t>(tree->perm, d_src, d_dst, n, row_bytes, s);
    return e == cudaSuccess ? TB_OK : TB_ECUDA;
}
