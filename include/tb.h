/*
 * tb.h -- C ABI of the GB300 oct-tree builder.
 *
 * The library builds the hashed oct-tree of Tokuue & Ishiyama (MNRAS 2023,
 * arXiv:2312.06102) on one GPU: particles in, cells out, each cell with its
 * level, key, parent, children, particle range and multipole moments.
 *
 * Pipeline (paper section in brackets):
 *   root cell + 64-bit particle keys                      [Sec. 2.2; Sec. 2.3 step 1]
 *   stable sort of (key, original index)                  [Sec. 2.3 step 2]
 *   leaves straight from the sorted keys                  [Sec. 2.3.1, Alg. 1, App. A]
 *   remaining cells bottom-up, with links                 [Sec. 2.3.2, Alg. 2]
 *   moments computed from children, never re-traversing   [Sec. 2.3, last paragraph;
 *                                                          footnote on the centre of mass]
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers.  Inputs stay owned by the caller,
 *    are only read, and must stay valid until the work enqueued on the
 *    caller's stream has finished.
 *  - Every array a tb_tree points to is DEVICE memory owned by the library;
 *    tb_free releases it.  A tree may be passed back to tb_build /
 *    tb_build_batched to be rebuilt in place (its buffers grow when needed).
 *  - Work is enqueued on the caller's stream and runs asynchronously.  The
 *    host waits only in these places: the cell-count read-back of a build
 *    whose params.cell_capacity is 0; a build or walk that must grow a tree's
 *    buffers (the device is synchronised before the old ones are freed);
 *    tb_free; tb_walk on a tree last built with a fixed capacity whose cell
 *    count has not been read back (it reads it first); and the calls that
 *    return device results to the host (tb_tree_status, tb_stage_times,
 *    tb_selftest_wait, tb_keys_sorted_noalloc).  A rebuild with a fixed capacity into buffers
 *    that are large enough never waits, and can be captured in a CUDA graph.
 *  - Threads: the library keeps process-wide state (kernel attributes set
 *    on first use on each device, the launch counter, the wait limit, the
 *    scratch of tb_keys_sorted_noalloc).  Calls from several host threads must be
 *    serialised by the caller; one thread may drive many trees on many
 *    streams.
 *  - Argument errors are returned at once.  Errors the GPU detects
 *    (non-finite coordinate, cell capacity exceeded, a look-back wait that
 *    ran out) are written to a device status word; the next call that
 *    synchronises returns them, as does tb_tree_status().
 *  - Sizes: 0 <= n <= 2^31 - 1 particles.  n = 0 gives an empty tree.
 *    1 <= n_crit <= 1024.  A NULL mass array means equal masses
 *    fp32(1.0 / n) (the FP64 quotient rounded once to FP32).
 *  - Positions are FP32, row-major [n][3], 4-byte aligned (16-byte alignment
 *    takes the vectorised load path).
 */
#ifndef TB_H
#define TB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tb_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    TB_OK = 0,
    TB_EINVAL = 1,       /* bad argument (NULL pointer, size out of range, bad mode) */
    TB_ENOMEM = 2,       /* device allocation failed */
    TB_ECUDA = 3,        /* a CUDA runtime call failed */
    TB_EOVERFLOW = 4,    /* more cells than params.cell_capacity (outputs not written) */
    TB_ETIMEOUT = 5,     /* a bounded device wait ran out (results not valid) */
    TB_ENONFINITE = 6    /* a coordinate is NaN or infinite (tree not built) */
} tb_status;

typedef enum {
    TB_MOM_FP32_COMP = 0,   /* FP32 with two-sum / two-product compensation (default) */
    TB_MOM_FP32_PLAIN = 1,  /* FP32, uncompensated (reported for comparison) */
    TB_MOM_FP64 = 2         /* FP64 accumulation; also fills mass64 / com64 / quad64 */
} tb_mom_mode;

/* Particle key order (Sec. 2.2 and its footnote).  Either way a key is a
 * leading 1 bit and 21 octant digits, and the particles of a depth-d cell
 * share the key's upper 3d + 1 bits, which is all the build relies on; the
 * cells are the same, ordered within a level by the chosen key.  Peano-Hilbert
 * keys follow Skilling's transform (AIP Conf. Proc. 707, 381, 2004). */
typedef enum {
    TB_KEYS_MORTON = 0,
    TB_KEYS_HILBERT = 1
} tb_key_order;

/* Maximum depth: 1 + 3 * 21 = 64 key bits (Sec. 2.2). */
#define TB_DEPTH_MAX 21
#define TB_LEVELS 22

typedef struct {
    int32_t n_crit;          /* a cell with more particles than this is split (Sec. 2.1) */
    int32_t mom_mode;        /* tb_mom_mode */
    int64_t cell_capacity;   /* 0: size the cell arrays exactly (one stream sync);
                                >0: fixed capacity, no host sync (graph-capturable);
                                at most 2^31 - 1 (cell indices are int32: a tree
                                with more cells gives TB_EOVERFLOW) */
    int32_t reorder;         /* 1: tb_moments also writes pos_sorted (particles in key
                                order, Sec. 2.3 step 3) */
    int32_t radix_bits;      /* 0 = tuned default; else 8..11 (sort digit width);
                                tb_build only */
    int32_t sort_threads;    /* 0 = tuned default; else threads per sort tile; tb_build only */
    int32_t sort_items;      /* 0 = tuned default; else keys per thread of a sort tile
                                (compiled variants: see tb_sort_variant); tb_build only */
    int32_t batch_threads;   /* tb_build_batched only: threads of the block that builds
                                one set, 512 (two sets per SM at a time; the default
                                for 0) or 1024 (one) */
    int32_t key_order;       /* tb_key_order: TB_KEYS_MORTON (default) or TB_KEYS_HILBERT
                                (tb_build only; tb_build_batched takes Morton keys) */
    int32_t batch_one_launch; /* tb_build_batched with cell_capacity > 0 only: 1 runs the
                                whole build as one cooperative launch (phases separated
                                by grid barriers); 0 (default) runs it as separate
                                launches, which measured faster */
    int32_t root_pow2;       /* 0 (default): the root cube's side is the largest extent
                                of the particles' bounding box; 1: it is forced to the
                                smallest power of two at least that extent (Sec. 2.2),
                                the corner staying at the per-axis minimum (tb_build
                                and, per set, tb_build_batched) */
} tb_params;

/* Host-side description of a tree.  Scalars are valid after a build with
 * cell_capacity == 0, or after tb_tree_status(); every pointer is a DEVICE
 * pointer owned by the library. */
typedef struct tb_tree {
    int64_t n_particles;
    int64_t n_cells;
    int64_t n_leaves;
    int32_t max_depth;
    int32_t n_crit;
    int64_t level_offset[TB_LEVELS + 1];  /* cells of level d: [level_offset[d], level_offset[d+1]) */
    double lo[3];                         /* root cube corner (FP32 minima, exact in FP64) */
    double side;                          /* root cube side L (FP64) */
    int64_t cell_capacity;                /* allocated length of the per-cell arrays */

    /* particles in key order: pkey[k] is the k-th smallest key, perm[k] the
       original index of that particle (ties keep ascending original index) */
    uint64_t *pkey;
    int32_t *perm;

    /* cells, canonical order: level ascending, key ascending within a level */
    uint64_t *ckey;          /* cell key: upper 3*level + 1 bits of its particles' keys; root = 1 */
    uint8_t *level;
    int32_t *parent;         /* -1 for the root */
    int32_t *child_first;    /* children are [child_first, child_end); -1/-1 for a leaf */
    int32_t *child_end;
    int32_t *pfirst;         /* particles are sorted positions [pfirst, pend) */
    int32_t *pend;
    int32_t *leaf_cell;      /* the j-th leaf in key order (n_leaves entries) */

    /* moments (tb_moments / tb_build_batched) */
    float *mass;             /* [C] total mass */
    float *com;              /* [C][3] centre of mass, rounded to FP32 */
    float *com_lo;           /* [C][3] com + com_lo is the centre of mass to ~2^-44 relative */
    float *quad;             /* [C][6] central second moment sum m (x-c)(x-c)^T: xx xy xz yy yz zz */
    float *aabb;             /* [C][6] member bounding box: min x y z, max x y z (exact) */
    double *mass64;          /* FP64 mode only, else NULL */
    double *com64;
    double *quad64;
    float *pos_sorted;       /* reorder only: [n][4] x, y, z, m in key order (Sec. 2.3
                                step 3), written by tb_moments; else NULL */

    /* batched builds only (NULL / 0 otherwise) */
    int32_t n_sets;
    int64_t *set_particle_offset;  /* [S+1] device copy of the caller's offsets */
    int64_t *set_cell_offset;      /* [S+1] cells of set s: [off[s], off[s+1]) */
    double *set_root;              /* [S][4] per-set root cube: lo x y z, side */

    void *internal;                /* library workspace */
} tb_tree;

/* Build the tree structure: root cell, keys, sort, leaves, cells and links
 * (Sec. 2.2, Sec. 2.3 steps 1, 2 and 4, Alg. 1, Alg. 2).
 *   d_pos   [n][3] FP32 positions (device)
 *   d_mass  [n] FP32 masses or NULL; only used by a later tb_moments
 *   n       number of particles
 *   params  n_crit, capacity, tuning (must not be NULL)
 *   stream  caller's stream
 *   tree    in: NULL to allocate a new tree, or a tree to rebuild in place;
 *           out: the tree (owned by the library until tb_free)
 * Returns TB_OK, TB_EINVAL, TB_ENOMEM, TB_ECUDA, or (capacity 0 only)
 * TB_ENONFINITE / TB_ETIMEOUT detected during the build. */
tb_status tb_build(const float *d_pos, const float *d_mass, int64_t n, const tb_params *params,
                   tb_stream stream, tb_tree **tree);

/* Fill mass, com, com_lo, quad and aabb of every cell of a built tree:
 * leaves by summation over their members in key order, every other cell
 * from its children (Sec. 2.3: properties are computed as cells are made,
 * the centre of mass of a parent from those of its children; higher
 * multipoles likewise).  tb_build keeps a snapshot of (x, y, z, m) taken
 * while it made the keys; when d_pos and d_mass are the same pointers the
 * build was given, that snapshot is used and the arrays are not read again
 * (new contents written in between are not seen: the moments are those of
 * the particles the tree was built from).  So once the build's work on the
 * stream has completed, the caller may refill those arrays, e.g. with the
 * next step's copy.  Other pointers are read afresh.  Leaves of more than
 * 2^20 particles are summed in FP64 in every mode (parents of that many in
 * the FP32-plain mode too).  Calling it again on the same build gives the
 * same moments bit for bit.  Returns TB_EINVAL when the
 * tree's last tb_build returned an error before it enqueued every stage. */
tb_status tb_moments(tb_tree *tree, const float *d_pos, const float *d_mass, tb_stream stream);

/* Build S independent trees in one call, moments included.  Particles of set
 * s are d_pos[d_set_offsets[s] .. d_set_offsets[s+1]); each set has its own
 * root cube (the tight one, or with root_pow2 its side forced to a power of
 * two).  Cells of each set are contiguous and canonical within the
 * set; parent / child / particle indices are global (into the whole arrays).
 *   d_set_offsets  [S+1] int64, device, non-decreasing, d_set_offsets[0] = 0
 *   n_total        d_set_offsets[S] (the host must know it for allocation)
 * Every set must hold at most 2^31 - 1 particles.  With
 * params.cell_capacity > 0 and a tree from an earlier call with the same S
 * and n_total, nothing is allocated and nothing synchronises, so the call can
 * be captured into a CUDA graph and replayed.  With batch_one_launch set the
 * whole build is then one cooperative launch (persistent blocks taking sets
 * from work queues, phases separated by grid barriers with bounded waits);
 * otherwise, and always with cell_capacity 0, it takes separate launches.
 * Of params it reads n_crit, mom_mode, cell_capacity and batch_threads;
 * key_order must be TB_KEYS_MORTON.  Each set is sorted by one block (five
 * 8-bit passes over the upper 40 key bits, then its runs of equal upper
 * bits), so radix_bits, sort_threads, sort_items and reorder are not used. */
tb_status tb_build_batched(const float *d_pos, const float *d_mass, const int64_t *d_set_offsets,
                           int32_t n_sets, int64_t n_total, const tb_params *params,
                           tb_stream stream, tb_tree **tree);

/* Gravitational accelerations (G = 1) of every particle from the tree
 * (Sec. 2.1): the Barnes-Hut walk with the opening test l / d < theta of Eq.
 * 1, cells taken as monopole + quadrupole (use_quad != 0) or monopole only,
 * and Barnes' modified algorithm -- the particles of a group share one
 * interaction list.  Groups are the cells holding at most n_group particles
 * whose parent holds more; a group is walked 32 particles at a time, and for
 * each such chunk a cell is accepted when l < theta * d_min, with d_min the
 * distance from the cell's centre of mass to the chunk's bounding box (so the
 * test of Eq. 1 holds for every particle of the chunk), and never when its
 * particles meet the chunk's.  Opened leaves contribute particle by particle.
 * Point masses are Plummer-softened with length eps; the quadrupole term,
 * T r / |r|^5 - (5/2) (r.T r) r / |r|^7 with T = 3 Q - tr(Q) I and r = x -
 * COM, is not.  Arithmetic is FP32.
 *   tree     a single tree (tb_build) whose moments are current (tb_moments
 *            called after the last build), else TB_EINVAL
 *   theta    opening parameter >= 0 (0 opens every cell: direct summation)
 *   eps      softening length >= 0
 *   n_group  group size bound, 1 <= n_group <= 2^20
 *   d_acc    [n_particles][3] FP32 out, device, caller-owned, in the
 *            caller's original particle order
 * Scratch (per-warp traversal stacks of about 30 MB, plus 84 B per cell for
 * the group list and a packed copy of the moments) is allocated on first use
 * and kept with the tree.  A traversal stack
 * that fills (not expected for trees of depth <= 21) sets a device status that
 * tb_tree_status reports as TB_EOVERFLOW. */
tb_status tb_walk(tb_tree *tree, float theta, float eps, int32_t n_group, int32_t use_quad,
                  float *d_acc, tb_stream stream);

/* Interactions evaluated by the last tb_walk of `tree` made while profiling
 * was enabled on it (tb_profile; counting costs such a walk about 15%):
 * target particle x accepted cell, and target particle x source particle
 * (self pairs excluded).  With theta = 0 no cell is accepted and the second
 * count is n (n - 1).  Both are 0 before the first walk; after a walk made
 * without profiling they are 0 too.  Synchronises `stream`.
 * Returns TB_OK, TB_EINVAL (NULL argument) or TB_ECUDA. */
tb_status tb_walk_counts(tb_tree *tree, tb_stream stream, int64_t *cell_interactions,
                         int64_t *particle_interactions);

/* Reorder a per-particle array into the key order of a built single tree
 * (Sec. 2.3 step 3; done "every few steps" in a simulation so that later
 * builds start from nearly sorted particles):
 *   d_dst[k] = d_src[perm[k]] for k < n_particles, row by row.
 *   d_src, d_dst  [n_particles][row_bytes] device arrays, caller-owned; they
 *                 must not overlap; 4-byte aligned (16-byte rows on 16-byte
 *                 aligned arrays take the vector path)
 *   row_bytes     bytes per particle, a positive multiple of 4 (e.g. 12 for
 *                 [n][3] FP32 positions, 4 for masses)
 * The tree must come from tb_build (not tb_build_batched); its perm is read
 * on `stream`, so the build must be ordered before this call.  Returns TB_OK
 * or TB_EINVAL (bad pointer, size or alignment, a batched tree, or a tree
 * whose last tb_build did not complete) / TB_ECUDA. */
tb_status tb_reorder(const tb_tree *tree, const void *d_src, void *d_dst, int64_t row_bytes,
                     tb_stream stream);

/* Release a tree (NULL-safe).  Synchronises with the device before freeing. */
void tb_free(tb_tree *tree);

/* Synchronise `stream`, refresh the tree's host scalars from the device and
 * return the device status (TB_OK, TB_ENONFINITE, TB_EOVERFLOW, TB_ETIMEOUT). */
tb_status tb_tree_status(tb_tree *tree, tb_stream stream);

const char *tb_status_string(tb_status s);

/* Default parameters: n_crit 16, compensated FP32 moments, exact sizing. */
tb_params tb_default_params(void);

/* The i-th compiled radix-sort variant (digit bits, threads, keys per
 * thread); returns 0 past the last one.  Any of them may be named in
 * tb_params; the autotuner times them. */
int32_t tb_sort_variant(int32_t i, int32_t *radix_bits, int32_t *threads, int32_t *items);

/* Number of kernels this library has launched in this process so far. */
int64_t tb_kernel_launches(void);

/* Per-stage timing of the most recent builds of `tree`.  When enabled the
 * library records CUDA events on the build stream at each stage boundary,
 * and tb_walk counts its interactions (tb_walk_counts).
 * tb_stage_times synchronises the stream and writes up to `max` elapsed
 * times (ms) of the last build and moment call, returning the count; names
 * come from tb_stage_name.  Stage 0 is the root cell, 1 the keys, 2..1+P the
 * P sort passes, then level counts, cell emission and moments. */
tb_status tb_profile(tb_tree *tree, int32_t enable);
int32_t tb_stage_times(tb_tree *tree, tb_stream stream, float *ms, int32_t max);
const char *tb_stage_name(tb_tree *tree, int32_t i);

/* Self-test of the bounded device wait: launches one kernel that waits on a
 * flag nothing sets, giving up after `spin_limit` polls.  Returns
 * TB_ETIMEOUT when the wait ran out and the context is still usable. */
tb_status tb_selftest_wait(int64_t spin_limit, tb_stream stream);

/* Test hook for the bounded waits of the radix sort (Sec. 2.3 step 2): each
 * pass's look-back on earlier tiles gives up after `polls` polls of a
 * predecessor that has not published yet (the default, 2^26 polls with a
 * back-off, is about 17 s) and the build then reports TB_ETIMEOUT.  A small
 * limit makes a multi-tile sort run out on purpose; its keys and cells are
 * then not valid, but every access stays in bounds and the next build with
 * the default limit is correct.  polls = 0 restores the default.  The
 * setting is process-wide and applies to sorts enqueued after the call.
 * Returns TB_OK, or TB_EINVAL for polls < 0. */
tb_status tb_set_wait_limit(int64_t polls);

/* Allocation-free keys and sort.  The paper has no counterpart to this entry
 * point: it serves callers of this library that cannot allocate device
 * memory when they call -- for example code that runs while another
 * component's caching allocator holds the device's free memory, or inside a
 * loop that must not pay cudaMalloc's implicit synchronisation.
 * Computes the same root cube, keys and stable (key, index) sort as tb_build:
 *   d_pos   [n][3] FP32 positions (device, caller-owned)
 *   n       0 <= n <= TB_NOALLOC_MAX_N, else TB_EINVAL before any GPU work
 *   d_pkey  [n] out: sorted keys (device, caller-owned, 8-byte aligned)
 *   d_perm  [n] out: original index of each sorted key (device, caller-owned)
 *   h_root  [4] out, host, optional: root corner x y z and side
 * Scratch lives in one fixed file-scope device array of about 15 MB.  CUDA
 * loads the library's code lazily, so a device reserves that array at the
 * first call on it (the call looks up the array's address with the device
 * current), and loads the kernels at the first call that sorts (n >= 2):
 * those first calls can return TB_ENOMEM or TB_ECUDA when the device's
 * memory is already taken.  Make one call with n >= 2 at start-up, before
 * any stream capture; after it the device holds the array and the kernels
 * until the process exits and calls allocate nothing.  Every call shares
 * the array, so calls whose GPU work overlaps race; order them on one
 * stream.  The call synchronises `stream` before it returns TB_OK,
 * TB_EINVAL, TB_ENOMEM (first calls on a device only), TB_ECUDA,
 * TB_ENONFINITE or TB_ETIMEOUT. */
#define TB_NOALLOC_MAX_N 524288
tb_status tb_keys_sorted_noalloc(const float *d_pos, int64_t n, uint64_t *d_pkey, int32_t *d_perm,
                                 double *h_root, tb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TB_H */
