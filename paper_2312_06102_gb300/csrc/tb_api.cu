// tb_api.cu -- host side of the C ABI declared in include/tb.h: argument
// checks, buffer management, the launch sequence of a build, status
// read-back and stage timing.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "tb_internal.h"

namespace tb {

int64_t g_launches = 0;

namespace {

// Test hook: TB_FAULT_ALLOC=k makes the k-th device allocation of the
// process fail (k counted from 1), to exercise the TB_ENOMEM paths.
int64_t g_alloc_calls = 0;
int64_t fault_alloc_at() {
    static int64_t v = -2;
    if (v == -2) {
        const char *e = std::getenv("TB_FAULT_ALLOC");
        v = e ? std::atoll(e) : -1;
    }
    return v;
}

template <class T>
bool dev_alloc(T *&p, int64_t count) {
    ++g_alloc_calls;
    if (fault_alloc_at() > 0 && g_alloc_calls == fault_alloc_at()) return false;
    void *q = nullptr;
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p = static_cast<T *>(q);
    return true;
}

template <class T>
void dev_free(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

struct TreeState {
    tb_tree pub;
    Workspace ws;
    tb_params params;
    int radix_bits = 8;
};

TreeState *state_of(tb_tree *t) { return reinterpret_cast<TreeState *>(t); }

tb_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TB_OK;
    if (e == cudaErrorMemoryAllocation) return TB_ENOMEM;
    return TB_ECUDA;
}

tb_status from_dev(uint32_t st) {
    if (st & kErrInvalid) return TB_EINVAL;
    if (st & kErrNonFinite) return TB_ENONFINITE;
    if (st & kErrTimeout) return TB_ETIMEOUT;
    if (st & (kErrOverflow | kErrWalk)) return TB_EOVERFLOW;
    return TB_OK;
}

void free_cells(TreeState &S) {
    tb_tree &t = S.pub;
    dev_free(t.ckey); dev_free(t.level); dev_free(t.parent); dev_free(t.child_first);
    dev_free(t.child_end); dev_free(t.pfirst); dev_free(t.pend);
    dev_free(t.mass); dev_free(t.com); dev_free(t.com_lo); dev_free(t.quad); dev_free(t.aabb);
    dev_free(t.mass64); dev_free(t.com64); dev_free(t.quad64);
    t.cell_capacity = 0;
    S.ws.cell_cap = 0;
}

void free_particles(TreeState &S) {
    tb_tree &t = S.pub;
    Workspace &ws = S.ws;
    dev_free(t.pkey); dev_free(t.perm); dev_free(ws.keys_alt); dev_free(ws.perm_alt);
    dev_free(ws.xm);
    dev_free(ws.xs);
    t.pos_sorted = nullptr;
    ws.xm_pos = ws.xm_mass = nullptr;
    dev_free(t.leaf_cell); dev_free(ws.big_leaf);
    dev_free(ws.level_cnt); dev_free(ws.lookback); dev_free(ws.ml); dev_free(ws.long_runs);
    ws.n_cap = 0;
    ws.tiles_cap = 0;
    ws.level_tiles_cap = 0;
}

tb_status ensure_fixed(TreeState &S) {
    Workspace &ws = S.ws;
    if (ws.info) return TB_OK;
    if (!dev_alloc(ws.info, 1) || !dev_alloc(ws.hist, 16 * 2048) ||
        !dev_alloc(ws.bbox_part, bbox_grid() * 8))
        return TB_ENOMEM;
    if (cudaMallocHost(&ws.h_info, sizeof(DevInfo)) != cudaSuccess) {
        cudaGetLastError();
        return TB_ENOMEM;
    }
    if (cudaMemset(ws.info, 0, sizeof(DevInfo)) != cudaSuccess) return TB_ECUDA;
    std::memset(ws.h_info, 0, sizeof(DevInfo));
    return TB_OK;
}

// need_xs: the key-ordered records are scratch of the batched build's moments
tb_status ensure_particles(TreeState &S, int64_t n, const SortCfg &cfg, bool reorder,
                           bool need_xs) {
    Workspace &ws = S.ws;
    tb_tree &t = S.pub;
    const int64_t tiles = (n + cfg.tile() - 1) / cfg.tile();
    const int64_t need_lb = tiles * (int64_t(1) << cfg.radix_bits);
    const int64_t ltiles = (n + level_tile_size() - 1) / level_tile_size();
    if (n > ws.n_cap || need_lb > ws.tiles_cap || ltiles > ws.level_tiles_cap) {
        cudaDeviceSynchronize();
        free_particles(S);
        int64_t cap = n;
        int64_t lb = need_lb > 0 ? need_lb : 1;
        if (!dev_alloc(t.pkey, cap) || !dev_alloc(t.perm, cap) || !dev_alloc(ws.keys_alt, cap) ||
            !dev_alloc(ws.perm_alt, cap) || !dev_alloc(t.leaf_cell, cap) || !dev_alloc(ws.xm, cap) ||
            !dev_alloc(ws.big_leaf, cap) || !dev_alloc(ws.ml, cap) ||
            !dev_alloc(ws.long_runs, long_run_capacity(cap)) ||
            !dev_alloc(ws.level_cnt, (ltiles + 1) * kLevelFields) || !dev_alloc(ws.lookback, lb))
            return TB_ENOMEM;
        if (cudaMemset(ws.lookback, 0, sizeof(uint64_t) * lb) != cudaSuccess) return TB_ECUDA;
        ws.n_cap = cap;
        ws.tiles_cap = lb;
        ws.level_tiles_cap = ltiles;
    }
    // the particles in key order (the reorder output of Sec. 2.3 step 3) are
    // written out by the leaf pass only when asked for
    if ((reorder || need_xs) && !ws.xs && !dev_alloc(ws.xs, ws.n_cap)) return TB_ENOMEM;
    t.pos_sorted = reorder ? reinterpret_cast<float *>(ws.xs) : nullptr;
    return TB_OK;
}

tb_status ensure_cells(TreeState &S, int64_t cells, bool fp64) {
    Workspace &ws = S.ws;
    tb_tree &t = S.pub;
    if (cells > ws.cell_cap || (fp64 && !t.mass64)) {
        cudaDeviceSynchronize();
        int64_t cap = cells > ws.cell_cap ? cells : ws.cell_cap;
        // the parent pass bulk-copies children's moments and parent links in
        // whole groups of four cells, up to three cells past the last one
        const int64_t pad = kMomentPad;
        free_cells(S);
        if (!dev_alloc(t.ckey, cap) || !dev_alloc(t.level, cap) || !dev_alloc(t.parent, cap + pad) ||
            !dev_alloc(t.child_first, cap) || !dev_alloc(t.child_end, cap) ||
            !dev_alloc(t.pfirst, cap) || !dev_alloc(t.pend, cap) || !dev_alloc(t.mass, cap + pad) ||
            !dev_alloc(t.com, 3 * (cap + pad)) || !dev_alloc(t.com_lo, 3 * (cap + pad)) ||
            !dev_alloc(t.quad, 6 * (cap + pad)) || !dev_alloc(t.aabb, 6 * (cap + pad)))
            return TB_ENOMEM;
        if (fp64 && (!dev_alloc(t.mass64, cap) || !dev_alloc(t.com64, 3 * cap) ||
                     !dev_alloc(t.quad64, 6 * cap)))
            return TB_ENOMEM;
        ws.cell_cap = cap;
        t.cell_capacity = cap;
    }
    return TB_OK;
}

void refresh_host(TreeState &S) {
    const DevInfo &h = *S.ws.h_info;
    tb_tree &t = S.pub;
    S.ws.host_current = true;
    t.n_cells = h.n_cells;
    t.n_leaves = h.n_leaves;
    t.max_depth = h.max_depth;
    for (int d = 0; d <= kLevels; ++d) t.level_offset[d] = h.level_offset[d];
    for (int a = 0; a < 3; ++a) t.lo[a] = (double)h.lo[a];
    t.side = h.side;
}

// Cell indices (parent, children, leaf_cell) are int32: a tree with more
// cells is refused before anything is allocated or written.  The overflow bit
// also goes into the device status, so later calls on the tree do nothing
// and report it.
tb_status refuse_cell_count(TreeState &S, cudaStream_t s) {
    if (S.ws.h_info->n_cells <= kMaxCells) return TB_OK;
    S.ws.h_info->status |= kErrOverflow;
    cudaError_t e = cudaMemcpyAsync(&S.ws.info->status, &S.ws.h_info->status, sizeof(uint32_t),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? TB_EOVERFLOW : from_cuda(e);
}

tb_status read_info(TreeState &S, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(S.ws.h_info, S.ws.info, sizeof(DevInfo),
                                    cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    refresh_host(S);
    return from_dev(S.ws.h_info->status);
}

SortCfg pick_cfg(const tb_params *p) {
    SortCfg c = default_sort_cfg(p->radix_bits ? p->radix_bits : 8);
    if (p->sort_threads) c.threads = p->sort_threads;
    if (p->sort_items) c.items = p->sort_items;
    return c;
}

bool valid_params(const tb_params *p) {
    return p && p->n_crit >= 1 && p->n_crit <= kMaxNcrit && p->mom_mode >= 0 && p->mom_mode <= 2 &&
           p->cell_capacity >= 0 && p->cell_capacity <= kMaxCells &&
           (p->radix_bits == 0 || (p->radix_bits >= 8 && p->radix_bits <= 11)) &&
           (p->key_order == TB_KEYS_MORTON || p->key_order == TB_KEYS_HILBERT) &&
           batch_threads_valid(p->batch_threads) &&
           (p->batch_one_launch == 0 || p->batch_one_launch == 1) &&
           (p->root_pow2 == 0 || p->root_pow2 == 1) &&
           sort_cfg_valid(pick_cfg(p));
}

}  // namespace

void mark(Workspace &ws, const char *name, cudaStream_t s) {
    if (!ws.profile || ws.n_events >= 200000) return;
    if (ws.n_events == ws.ev.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        ws.ev.push_back(e);
        ws.ev_name.push_back(name);
    }
    cudaEventRecord(ws.ev[ws.n_events], s);
    ws.ev_name[ws.n_events] = name;
    ++ws.n_events;
}

}  // namespace tb

using namespace tb;

extern "C" {

tb_params tb_default_params(void) {
    tb_params p;
    std::memset(&p, 0, sizeof(p));
    p.n_crit = 16;
    p.mom_mode = TB_MOM_FP32_COMP;
    return p;
}

const char *tb_status_string(tb_status s) {
    switch (s) {
        case TB_OK: return "ok";
        case TB_EINVAL: return "invalid argument";
        case TB_ENOMEM: return "device allocation failed";
        case TB_ECUDA: return "CUDA runtime error";
        case TB_EOVERFLOW: return "cell capacity exceeded";
        case TB_ETIMEOUT: return "bounded device wait ran out";
        case TB_ENONFINITE: return "non-finite coordinate";
    }
    return "unknown status";
}

int64_t tb_kernel_launches(void) { return g_launches; }

int32_t tb_sort_variant(int32_t i, int32_t *radix_bits, int32_t *threads, int32_t *items) {
    const SortCfg *c = sort_variant(i);
    if (!c) return 0;
    if (radix_bits) *radix_bits = c->radix_bits;
    if (threads) *threads = c->threads;
    if (items) *items = c->items;
    return 1;
}

tb_status tb_build(const float *d_pos, const float *d_mass, int64_t n, const tb_params *params,
                   tb_stream stream, tb_tree **tree) {
    if (!tree || !valid_params(params) || n < 0 || n > 2147483647LL) return TB_EINVAL;
    if (n > 0 && (!d_pos || (reinterpret_cast<uintptr_t>(d_pos) & 3u))) return TB_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_mass) & 3u) return TB_EINVAL;
    if (*tree && (*tree)->n_sets != 0) return TB_EINVAL;   // a batched tree
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TreeState *S = *tree ? state_of(*tree) : nullptr;
    if (!S) {
        S = new (std::nothrow) TreeState();
        if (!S) return TB_ENOMEM;
        std::memset(&S->pub, 0, sizeof(tb_tree));
        S->pub.internal = &S->ws;
        *tree = &S->pub;
    }
    tb_status st = ensure_fixed(*S);
    if (st != TB_OK) return st;
    Workspace &ws = S->ws;
    tb_tree &t = S->pub;
    S->params = *params;
    const SortCfg cfg = pick_cfg(params);
    S->radix_bits = cfg.radix_bits;
    ws.last_stream = s;
    ws.moments_ready = false;
    ws.xs_current = false;
    ws.cells_ready = false;
    ws.host_current = false;
    t.n_particles = n;
    t.n_crit = params->n_crit;
    ws.cell_cap_request = params->cell_capacity;
    if (n == 0) {
        t.n_cells = t.n_leaves = 0;
        t.max_depth = 0;
        for (int d = 0; d <= kLevels; ++d) t.level_offset[d] = 0;
        for (int a = 0; a < 3; ++a) t.lo[a] = 0.0;
        t.side = 1.0;
        cudaError_t e = cudaMemsetAsync(ws.info, 0, offsetof(DevInfo, sort_tile_ctr), s);
        ws.cells_ready = ws.host_current = e == cudaSuccess;
        return from_cuda(e);
    }
    st = ensure_particles(*S, n, cfg, params->reorder != 0, false);
    if (st != TB_OK) return st;
    if (params->cell_capacity > 0) {
        st = ensure_cells(*S, params->cell_capacity, params->mom_mode == TB_MOM_FP64);
        if (st != TB_OK) return st;
    }
    const int passes = sort_plan(cfg).passes;
    mark(ws, "start", s);
    ws.root_pow2 = params->root_pow2 != 0;
    cudaError_t e = launch_root(d_pos, n, ws, passes << cfg.radix_bits, s);
    if (e != cudaSuccess) return from_cuda(e);
    mark(ws, "root", s);
    // the unsorted keys go where the last pass will read from the other buffer
    uint64_t *ka = (passes & 1) ? ws.keys_alt : t.pkey;
    uint64_t *kb = (passes & 1) ? t.pkey : ws.keys_alt;
    int32_t *pa = (passes & 1) ? ws.perm_alt : t.perm;
    int32_t *pb = (passes & 1) ? t.perm : ws.perm_alt;
    e = launch_keys(d_pos, d_mass, n, ka, ws, cfg, params->key_order, s);
    if (e != cudaSuccess) return from_cuda(e);
    ws.xm_pos = d_pos;
    ws.xm_mass = d_mass;
    mark(ws, "keys", s);
    uint64_t *kout = nullptr;
    int32_t *pout = nullptr;
    e = launch_sort(ka, kb, pa, pb, n, ws, cfg, kout, pout, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (kout != t.pkey || pout != t.perm) return TB_ECUDA;
    e = launch_levels(t.pkey, n, params->n_crit, ws, s);
    if (e != cudaSuccess) return from_cuda(e);
    mark(ws, "levels", s);
    if (params->cell_capacity == 0) {
        st = read_info(*S, s);
        if (st != TB_OK) return st;
        st = refuse_cell_count(*S, s);
        if (st != TB_OK) return st;
        st = ensure_cells(*S, ws.h_info->n_cells, params->mom_mode == TB_MOM_FP64);
        if (st != TB_OK) return st;
    }
    e = launch_emit(t.pkey, n, params->n_crit, ws, t, s);
    if (e != cudaSuccess) return from_cuda(e);
    mark(ws, "emit", s);
    ws.cells_ready = true;
    return TB_OK;
}

tb_status tb_walk(tb_tree *tree, float theta, float eps, int32_t n_group, int32_t use_quad,
                  float *d_acc, tb_stream stream) {
    if (!tree || tree->n_sets != 0 || !(theta >= 0.f) || !(theta < 1e30f) || !(eps >= 0.f) ||
        !(eps < 1e30f) || n_group < 1 || n_group > (1 << 20))
        return TB_EINVAL;
    TreeState *S = state_of(tree);
    if (tree->n_particles == 0) return TB_OK;
    if (!d_acc || (reinterpret_cast<uintptr_t>(d_acc) & 3u)) return TB_EINVAL;
    if (!S->ws.moments_ready) return TB_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the walk sizes its groups, records and buffer by the cell count: after
    // a fixed-capacity build that count is read back first (one stream wait)
    if (!S->ws.host_current) {
        tb_status st = read_info(*S, s);
        if (st != TB_OK) return st;
    }
    const int64_t need = walk_buffer_words(tree->n_cells);
    if (S->ws.walk_cap < need) {
        dev_free(S->ws.walk);
        S->ws.walk_cap = 0;
        if (!dev_alloc(S->ws.walk, need)) return TB_ENOMEM;
        S->ws.walk_cap = need;
    }
    // the walk reads the particles in key order: written by the moments only
    // when pos_sorted was asked for, else gathered here once per moments call
    if (!S->ws.xs_current) {
        if (!S->ws.xs && !dev_alloc(S->ws.xs, S->ws.n_cap)) return TB_ENOMEM;
        cudaError_t e = launch_gather_records(tree->perm, S->ws.xm, S->ws.xs, tree->n_particles, s);
        if (e != cudaSuccess) return from_cuda(e);
        S->ws.xs_current = true;
    }
    return from_cuda(launch_walk(*tree, S->ws, theta, eps, n_group, use_quad, d_acc, S->ws.walk, s));
}

tb_status tb_moments(tb_tree *tree, const float *d_pos, const float *d_mass, tb_stream stream) {
    if (!tree || (tree->n_particles > 0 && !d_pos)) return TB_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_pos) & 3u) return TB_EINVAL;
    TreeState *S = state_of(tree);
    if (tree->n_sets != 0) return TB_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (tree->n_particles == 0) return TB_OK;
    if (!S->ws.cells_ready) return TB_EINVAL;   // the last build did not complete
    const bool fp64 = S->params.mom_mode == TB_MOM_FP64;
    if (fp64 && !tree->mass64) {
        tb_status st = ensure_cells(*S, S->ws.cell_cap, true);
        if (st != TB_OK) return st;
    }
    if (S->params.reorder && !tree->pos_sorted) return TB_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_mass) & 3u) return TB_EINVAL;
    S->ws.last_stream = s;
    cudaError_t e = cudaSuccess;
    if (d_pos != S->ws.xm_pos || d_mass != S->ws.xm_mass) {
        e = launch_pack(d_pos, d_mass, tree->n_particles, S->ws.xm, s);
        if (e != cudaSuccess) return from_cuda(e);
        S->ws.xm_pos = d_pos;
        S->ws.xm_mass = d_mass;
    }
    e = launch_moments(*tree, S->ws, S->params.mom_mode, s);
    if (e != cudaSuccess) return from_cuda(e);
    S->ws.moments_ready = true;
    S->ws.xs_current = tree->pos_sorted != nullptr;
    return TB_OK;
}

tb_status tb_build_batched(const float *d_pos, const float *d_mass, const int64_t *d_set_offsets,
                           int32_t n_sets, int64_t n_total, const tb_params *params,
                           tb_stream stream, tb_tree **tree) {
    if (!tree || !valid_params(params) || n_sets < 0 || n_total < 0 || n_total > 2147483647LL)
        return TB_EINVAL;
    if (params->key_order != TB_KEYS_MORTON) return TB_EINVAL;   // batched: Morton keys only
    if (n_sets > 0 && !d_set_offsets) return TB_EINVAL;
    if (n_total > 0 && (!d_pos || (reinterpret_cast<uintptr_t>(d_pos) & 3u))) return TB_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_mass) & 3u) return TB_EINVAL;
    if (*tree && (*tree)->n_sets == 0 && (*tree)->n_particles > 0) return TB_EINVAL;   // a single tree
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TreeState *S = *tree ? state_of(*tree) : nullptr;
    if (!S) {
        S = new (std::nothrow) TreeState();
        if (!S) return TB_ENOMEM;
        std::memset(&S->pub, 0, sizeof(tb_tree));
        S->pub.internal = &S->ws;
        *tree = &S->pub;
    }
    tb_status st = ensure_fixed(*S);
    if (st != TB_OK) return st;
    Workspace &ws = S->ws;
    tb_tree &t = S->pub;
    S->params = *params;
    ws.last_stream = s;
    ws.root_pow2 = params->root_pow2 != 0;
    t.n_particles = n_total;
    t.n_crit = params->n_crit;
    t.n_sets = n_sets;
    st = ensure_particles(*S, n_total, default_sort_cfg(8), false, true);
    if (st != TB_OK) return st;
    if (n_sets > ws.set_cap || !t.set_cell_offset) {
        cudaDeviceSynchronize();
        dev_free(ws.set_order); dev_free(ws.set_cnt); dev_free(ws.set_leaf_off); dev_free(ws.set_ctr);
        dev_free(t.set_particle_offset); dev_free(t.set_cell_offset); dev_free(t.set_root);
        const int64_t cap = n_sets > 0 ? n_sets : 1;
        if (!dev_alloc(ws.set_order, cap) || !dev_alloc(ws.set_cnt, cap * kLevelFields) ||
            !dev_alloc(ws.set_leaf_off, cap + 1) || !dev_alloc(ws.set_ctr, 8) ||
            !dev_alloc(t.set_particle_offset, cap + 1) || !dev_alloc(t.set_cell_offset, cap + 1) ||
            !dev_alloc(t.set_root, 4 * cap))
            return TB_ENOMEM;
        ws.set_cap = cap;
    }
    if (params->cell_capacity > 0) {
        st = ensure_cells(*S, params->cell_capacity, params->mom_mode == TB_MOM_FP64);
        if (st != TB_OK) return st;
    }
    cudaError_t e = cudaMemsetAsync(ws.info, 0, sizeof(DevInfo), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.set_ctr, 0, 8 * sizeof(uint32_t), s);
    if (e == cudaSuccess && n_sets > 0)
        e = cudaMemcpyAsync(t.set_particle_offset, d_set_offsets, sizeof(int64_t) * (n_sets + 1),
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (n_sets == 0 || n_total == 0) {
        // nothing to build: offsets of the (empty) sets are all zero
        if (n_sets > 0) {
            e = cudaMemsetAsync(t.set_cell_offset, 0, sizeof(int64_t) * (n_sets + 1), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(t.set_root, 0, sizeof(double) * 4 * n_sets, s);
            if (e != cudaSuccess) return from_cuda(e);
        }
        t.n_cells = t.n_leaves = 0;
        t.max_depth = 0;
        return TB_OK;
    }
    mark(ws, "start", s);
    if (params->cell_capacity > 0 && params->batch_one_launch) {
        // fixed capacity: the whole build in one cooperative launch
        e = launch_batched_one(d_pos, d_mass, t.set_particle_offset, n_sets, n_total,
                               params->n_crit, params->batch_threads, t, ws, params->cell_capacity,
                               params->mom_mode, s);
        if (e == cudaSuccess) return TB_OK;
        // a device that cannot take it: the same build in separate launches
        cudaGetLastError();
    }
    e = launch_set_check(t.set_particle_offset, n_sets, n_total, ws, s);
    if (e == cudaSuccess)
        e = launch_batched(d_pos, d_mass, t.set_particle_offset, n_sets, params->n_crit,
                           params->batch_threads, t, ws, params->cell_capacity, 0,
                           params->mom_mode, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (params->cell_capacity == 0) {
        st = read_info(*S, s);
        if (ws.h_info->status & kErrInvalid) return TB_EINVAL;
        if (st != TB_OK) return st;
        st = refuse_cell_count(*S, s);
        if (st != TB_OK) return st;
        st = ensure_cells(*S, ws.h_info->n_cells > 0 ? ws.h_info->n_cells : 1,
                          params->mom_mode == TB_MOM_FP64);
        if (st != TB_OK) return st;
    }
    e = launch_batched(d_pos, d_mass, t.set_particle_offset, n_sets, params->n_crit,
                       params->batch_threads, t, ws, params->cell_capacity, 1, params->mom_mode, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (params->cell_capacity == 0) {
        st = read_info(*S, s);
        if (st != TB_OK) return st;
    }
    return TB_OK;
}

void tb_free(tb_tree *tree) {
    if (!tree) return;
    TreeState *S = state_of(tree);
    cudaDeviceSynchronize();
    free_cells(*S);
    free_particles(*S);
    Workspace &ws = S->ws;
    dev_free(ws.info); dev_free(ws.hist); dev_free(ws.bbox_part);
    if (ws.h_info) cudaFreeHost(ws.h_info);
    for (cudaEvent_t e : ws.ev) cudaEventDestroy(e);
    dev_free(ws.walk);
    dev_free(ws.set_order); dev_free(ws.set_cnt); dev_free(ws.set_leaf_off); dev_free(ws.set_ctr);
    dev_free(tree->set_particle_offset); dev_free(tree->set_cell_offset); dev_free(tree->set_root);
    delete S;
}

tb_status tb_tree_status(tb_tree *tree, tb_stream stream) {
    if (!tree) return TB_EINVAL;
    TreeState *S = state_of(tree);
    if (!S->ws.info) return TB_OK;
    return read_info(*S, reinterpret_cast<cudaStream_t>(stream));
}

tb_status tb_profile(tb_tree *tree, int32_t enable) {
    if (!tree) return TB_EINVAL;
    state_of(tree)->ws.profile = enable != 0;
    return TB_OK;
}

int32_t tb_stage_times(tb_tree *tree, tb_stream stream, float *ms, int32_t max) {
    if (!tree || !ms) return 0;
    Workspace &ws = state_of(tree)->ws;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return 0;
    int32_t k = 0;
    for (size_t i = 1; i < ws.n_events && k < max; ++i, ++k) {
        float v = 0.f;
        cudaEventElapsedTime(&v, ws.ev[i - 1], ws.ev[i]);
        ms[k] = v;
    }
    // names stay readable until the next record; restart the accumulation
    ws.last_read = ws.n_events;
    ws.n_events = 0;
    return k;
}

const char *tb_stage_name(tb_tree *tree, int32_t i) {
    if (!tree) return "";
    Workspace &ws = state_of(tree)->ws;
    if (i < 0 || (size_t)i + 1 >= ws.last_read) return "";
    return ws.ev_name[i + 1];
}

tb_status tb_walk_counts(tb_tree *tree, tb_stream stream, int64_t *cell_interactions,
                         int64_t *particle_interactions) {
    if (!tree || !cell_interactions || !particle_interactions) return TB_EINVAL;
    Workspace &ws = state_of(tree)->ws;
    *cell_interactions = *particle_interactions = 0;
    if (!ws.walk_ctr) return TB_OK;
    unsigned long long h[2] = {0, 0};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h, ws.walk_ctr + 2, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    *cell_interactions = (int64_t)h[0];
    *particle_interactions = (int64_t)h[1];
    return TB_OK;
}

tb_status tb_set_wait_limit(int64_t polls) {
    if (polls < 0) return TB_EINVAL;
    g_wait_limit = polls > 0 ? polls : kDefaultWaitLimit;
    return TB_OK;
}

tb_status tb_selftest_wait(int64_t spin_limit, tb_stream stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *buf = nullptr;
    if (cudaMalloc(&buf, 2 * sizeof(uint32_t)) != cudaSuccess) return TB_ENOMEM;
    cudaMemsetAsync(buf, 0, 2 * sizeof(uint32_t), s);
    cudaError_t e = launch_wait_selftest(spin_limit, buf, buf + 1, s);
    uint32_t h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, buf, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) return from_cuda(e);
    return from_dev(h[0]);
}

}  // extern "C"
