// tb_internal.h -- declarations shared by the library's translation units:
// the device-side build record, status bits, sizes and the host launchers of
// each kernel family.
#pragma once

#include <atomic>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/tb.h"

namespace tb {

constexpr int kLevels = TB_LEVELS;          // depths 0..21
constexpr int kDepthMax = TB_DEPTH_MAX;
constexpr int kLevelFields = kLevels + 1;   // 22 level counters + 1 leaf counter
constexpr int kMaxNcrit = 1024;
constexpr int64_t kMaxCells = 2147483647;   // cell indices are int32
constexpr int64_t kBigCell = int64_t(1) << 20;   // cells above this are summed in FP64
constexpr int64_t kMomentPad = 8;   // cells allocated past the capacity in the moment arrays

// device status bits (tb_dev_info::status)
constexpr uint32_t kErrNonFinite = 1u;
constexpr uint32_t kErrOverflow = 2u;
constexpr uint32_t kErrTimeout = 4u;
constexpr uint32_t kErrInvalid = 8u;    // batched: set offsets not a partition of [0, n)
constexpr uint32_t kErrWalk = 16u;      // tree walk: traversal stack full

// Record of one build, in device memory; written by the kernels, read back
// by the host after a synchronisation.
struct DevInfo {
    float lo[3];           // root corner (FP32 minima)
    float hi[3];
    double side;           // L = max_a (hi_a - lo_a), 1 if 0
    double scale;          // 2^21 / L
    float s_hi, s_lo;      // scale ~ s_hi + s_lo
    uint32_t exact_only;   // 1: quantise with FP64 only (extreme ranges)
    uint32_t status;       // kErr* bits
    uint32_t epoch;        // look-back epoch base of the current tree build
    uint32_t n_leaves;
    int32_t max_depth;
    uint32_t s_fp32;       // 1: the scale is an FP32 value (scale == s_hi exactly)
    int64_t n_cells;
    int64_t level_offset[kLevels + 1];
    uint32_t sort_tile_ctr[16];   // dynamic tile ids, one counter per sort pass
    uint32_t misc_ctr[8];         // [0] bbox blocks done, [1] level-scan blocks done,
                                  // [2] big-leaf queue length, [3] big-leaf tickets,
                                  // [4] key blocks done, [5] long sort runs, [6] their tickets
};

// Sort tuning: a compiled variant.
struct SortCfg {
    int radix_bits;
    int threads;
    int items;
    int tile() const { return threads * items; }
};


// Global radix passes of a variant and the lowest bit they sort from; the
// runs of equal key >> shift0 are finished by the run step.
struct SortPlan {
    int passes;
    int shift0;
};
SortPlan sort_plan(const SortCfg &c);

// Workspace of one tree (device pointers unless noted).
struct Workspace {
    int64_t n_cap = 0;         // particle capacity
    int64_t tiles_cap = 0;     // look-back tiles capacity
    int64_t cell_cap = 0;
    int64_t level_tiles_cap = 0;
    int64_t leaf_cap = 0;
    int64_t bbox_blocks = 0;
    int64_t cell_cap_request = 0;   // params.cell_capacity of the current build
    int64_t reorder_cap = 0;
    bool root_pow2 = false;          // root side forced to a power of two (this build)

    float4 *xm = nullptr;            // [n] (x, y, z, m) in input order, written with the keys
    float4 *xs = nullptr;            // [n] the same records in key order (reorder only)
    const float *xm_pos = nullptr;   // arrays xm was made from
    const float *xm_mass = nullptr;
    uint64_t *keys_alt = nullptr;
    int32_t *perm_alt = nullptr;
    uint32_t *hist = nullptr;        // [passes][radix]
    uint64_t *lookback = nullptr;    // [tiles][radix]
    float *bbox_part = nullptr;      // [blocks][8]
    uint32_t *level_cnt = nullptr;   // [level tiles][kLevelFields]
    uint16_t *ml = nullptr;          // [n] m_k | L_k << 8 of each sorted particle
    int32_t *long_runs = nullptr;    // [n / 1024 + 2] sort runs too long for the run step
    int32_t *big_leaf = nullptr;     // [n] queue of depth-21 leaves too long for one thread
    DevInfo *info = nullptr;
    DevInfo *h_info = nullptr;       // pinned host mirror

    // profiling: events recorded at stage boundaries, accumulated over
    // builds until read
    bool profile = false;
    size_t n_events = 0;
    size_t last_read = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<const char *> ev_name;

    // batched
    int64_t set_cap = 0;
    int32_t *set_order = nullptr;    // [S] processing order (largest first)
    uint32_t *set_cnt = nullptr;     // [S][kLevelFields] cells per level and leaves of each set
    int64_t *set_leaf_off = nullptr; // [S+1]
    uint32_t *set_ctr = nullptr;     // [8] work-queue tickets, grid-barrier words

    cudaStream_t last_stream = nullptr;
    // tree walk scratch and whether the moments match the current structure
    int32_t *walk = nullptr;
    int64_t walk_cap = 0;
    uint32_t *walk_ctr = nullptr;   // counters of the last walk (groups, tickets, interactions)
    bool moments_ready = false;
    bool xs_current = false;      // xs holds the records of the last moments in key order
    bool cells_ready = false;     // the last tb_build enqueued every stage
    bool host_current = false;    // the tree's host scalars match the last build
};

// ------------------------------------------------------------ launchers
// Each returns cudaSuccess or the launch error.

extern int64_t g_launches;
constexpr int64_t kDefaultWaitLimit = int64_t(1) << 26;
extern int64_t g_wait_limit;   // polls of a radix-pass look-back wait

cudaError_t launch_root(const float *pos, int64_t n, Workspace &ws, int hist_len, cudaStream_t s);
cudaError_t launch_keys(const float *pos, const float *mass, int64_t n, uint64_t *keys,
                        Workspace &ws, const SortCfg &cfg, int key_order, cudaStream_t s);
cudaError_t launch_pack(const float *pos, const float *mass, int64_t n, float4 *xm,
                        cudaStream_t s);
cudaError_t launch_sort(uint64_t *keys_in_place_a, uint64_t *keys_b, int32_t *perm_a,
                        int32_t *perm_b, int64_t n, Workspace &ws, const SortCfg &cfg,
                        uint64_t *&keys_out, int32_t *&perm_out, cudaStream_t s);
cudaError_t launch_levels(const uint64_t *skeys, int64_t n, int n_crit, Workspace &ws,
                          cudaStream_t s);
cudaError_t launch_emit(const uint64_t *skeys, int64_t n, int n_crit, Workspace &ws,
                        tb_tree &t, cudaStream_t s);
cudaError_t launch_moments(tb_tree &t, Workspace &ws, int mode, cudaStream_t s);
cudaError_t launch_gather_records(const int32_t *perm, const float4 *xm, float4 *xs, int64_t n,
                                  cudaStream_t s);
cudaError_t launch_wait_selftest(int64_t limit, uint32_t *status, uint32_t *flag, cudaStream_t s);

int level_tile_size();
int64_t bbox_grid();
SortCfg default_sort_cfg(int radix_bits);
const SortCfg *sort_variant(int i);
bool sort_cfg_valid(const SortCfg &c);

cudaError_t launch_batched(const float *pos, const float *mass, const int64_t *off, int32_t S,
                           int ncrit, int threads, tb_tree &t, Workspace &ws, int64_t cell_cap,
                           int phase, int mode, cudaStream_t s);
bool batch_threads_valid(int threads);   // 0 (default), 512 or 1024
// The whole batched build (fixed cell capacity) in one cooperative launch;
// an error return leaves nothing enqueued, and the caller may fall back to
// the multi-launch path.
cudaError_t launch_batched_one(const float *pos, const float *mass, const int64_t *off, int32_t S,
                               int64_t n_total, int ncrit, int threads, tb_tree &t, Workspace &ws,
                               int64_t cell_cap, int mode, cudaStream_t s);
cudaError_t launch_set_check(const int64_t *off, int32_t S, int64_t n_total, Workspace &ws,
                             cudaStream_t s);

cudaError_t launch_runs(uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v, int64_t n,
                        int shift0, int32_t *long_runs, Workspace &ws, cudaStream_t s);
int64_t long_run_capacity(int64_t n);

// tree walk: int32 words of its scratch (counters, groups, per-warp stacks)
int64_t walk_buffer_words(int64_t n_cells);
cudaError_t launch_walk(const tb_tree &t, Workspace &ws, float theta, float eps, int n_group,
                        int use_quad, float *acc, int32_t *buf, cudaStream_t s);

void mark(Workspace &ws, const char *name, cudaStream_t s);

// Kernel attributes (dynamic shared memory above 48 KB, carve-out) belong to
// a device.  A launcher keeps one bit per device in `done` and sets its
// attributes the first time it runs on each device; two host threads that
// race here both set the same values, which is harmless.
inline bool first_on_device(std::atomic<uint64_t> &done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
    const uint64_t bit = uint64_t(1) << dev;
    if (done.load(std::memory_order_acquire) & bit) return false;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

}  // namespace tb
