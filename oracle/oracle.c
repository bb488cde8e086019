/*
 * oracle.c -- plain, single-threaded FP64 CPU oracle for the hashed
 * oct-tree build of Tokuue & Ishiyama (MNRAS 2023, arXiv:2312.06102).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or constant with the CUDA library: every step below is
 * written from the paper's definitions, slowly and directly, so that a
 * reader can check it against the text by eye.
 *
 * What it computes (paper section in brackets):
 *   ora_keys        root cell and 64-bit particle keys          [Sec. 2.2]
 *   ora_hilbert     Peano-Hilbert key of three 21-bit integers  [Sec. 2.2 footnote]
 *   ora_sort        stable sort of (key, index) pairs            [Sec. 2.3, step 2]
 *   ora_build       Barnes-Hut top-down build: a cell holding more
 *                   than n_crit particles is halved along each axis
 *                   (8 children, empty ones not created)        [Sec. 2.1]
 *                   then cells in canonical (level, key) order with
 *                   parent / child / particle-range links        [Sec. 2.3.2 footnotes]
 *   ora_moments     direct FP64 sums over each cell's members:
 *                   mass, centre of mass, central second moment,
 *                   member bounding box                          [Sec. 2.3, footnote on COM]
 *   ora_paper_build the leaf scan of Algorithm 1 and the per-depth
 *                   parent creation of Algorithm 2, as a second,
 *                   independent route to the same cells          [Alg. 1, Alg. 2, App. A]
 *   ora_tree_walk   monopole + quadrupole tree walk with the opening
 *                   test l/d < theta of Eq. (1)                  [Sec. 2.1, Eq. 1]
 *   ora_direct_acc  O(N^2) softened direct summation (check of the walk)
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes):
 *   - root cell: tight bounding box; corner lo = per-axis minimum, side
 *     L = largest per-axis extent (1 if all extents are 0).  With pow2 set,
 *     the side is forced to the smallest power of two >= L (Sec. 2.2), the
 *     corner staying at the minimum; keys taken from that corner are the
 *     paper's keys about the root's centre shifted by 2^20 on every axis.
 *   - quantisation: q = min(2^21 - 1, floor((double(x) - double(lo)) * s)),
 *     s = 2^21 / L, every operation FP64 round-to-nearest, no contraction.
 *   - octant digit: (x bit << 2) | (y bit << 1) | (z bit), x most significant.
 *   - minDepth(i,j) = ceil(clz64(key_i ^ key_j) / 3) with clz64(0) = 64, so
 *     identical keys give 22; the deepest level is 21 (1 + 3*21 = 64 bits) and
 *     a depth-21 cell is never split, so it may hold more than n_crit
 *     particles, all with the same key.
 *   - equal keys keep ascending original index (stable sort).
 *   - cells with zero total mass: centre of mass = first member (in key
 *     order), second moment 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_DEPTH_MAX 21
#define ORA_LEVELS 22

/* ------------------------------------------------------------------ */
/* Sec. 2.2: keys                                                      */
/* ------------------------------------------------------------------ */

/* minimum distinguished depth of two keys (Sec. 2.3.1): ceil(clz(a^b)/3) */
int ora_min_depth(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    int clz = 0;
    /* count leading zero bits one at a time; clz(0) = 64 */
    for (int bit = 63; bit >= 0; --bit) {
        if ((x >> bit) & 1u) break;
        ++clz;
    }
    return (clz + 2) / 3;
}

/* interleave three 21-bit integers below a leading 1 bit (Sec. 2.2) */
uint64_t ora_interleave(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t key = 1;
    for (int b = 20; b >= 0; --b) {
        key = (key << 1) | ((qx >> b) & 1u);
        key = (key << 1) | ((qy >> b) & 1u);
        key = (key << 1) | ((qz >> b) & 1u);
    }
    return key;
}

/* Peano-Hilbert key (the alternative order of the footnote in Sec. 2.2):
 * Skilling's transform of the three 21-bit coordinates (J. Skilling, AIP
 * Conf. Proc. 707, 381, 2004: "Programming the Hilbert curve") -- undo the
 * excess work level by level from the top (invert the low bits of the first
 * axis when an axis has the level's bit set, else exchange the low bits of
 * the first axis and that axis), then Gray-encode across the axes and
 * correct by the parity of the last axis -- and the result interleaved like a
 * Morton key, first axis most significant, below the leading 1 bit.  Keys of
 * the points of one depth-d cube share their upper 3d + 1 bits, and
 * consecutive grid points along the key order are face neighbours. */
uint64_t ora_hilbert(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint32_t X[3] = {qx, qy, qz};
    const uint32_t M = 1u << 20;
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    return ora_interleave(X[0], X[1], X[2]);
}

/* one coordinate to a 21-bit integer */
uint32_t ora_quantise(float x, double lo, double scale)
{
    volatile double d = (double)x - lo;  /* volatile: keep each FP64 op separate */
    volatile double t = d * scale;
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    return (uint32_t)f;
}

/* smallest power of two >= L, for L > 0 (exact: frexp gives L = m 2^e,
 * m in [1/2, 1)) */
static double pow2_ceil(double L)
{
    int e;
    double m = frexp(L, &e);
    return (m == 0.5) ? L : ldexp(1.0, e);
}

/* root cell: corner lo[3] and side; returns 0, or 1 if a coordinate is not
 * finite.  pow2: side forced to a power of two (Sec. 2.2). */
int ora_root_mode(const float *pos, int64_t n, double lo[3], double *side, int pow2)
{
    double hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = 0.0; hi[a] = 0.0; }
    if (n <= 0) { *side = 1.0; return 0; }
    for (int a = 0; a < 3; ++a) { lo[a] = pos[a]; hi[a] = pos[a]; }
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            float x = pos[3 * i + a];
            if (!isfinite(x)) return 1;
            if (x < lo[a]) lo[a] = x;
            if (x > hi[a]) hi[a] = x;
        }
    }
    double L = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = hi[a] - lo[a];
        if (e > L) L = e;
    }
    *side = (L > 0.0) ? (pow2 ? pow2_ceil(L) : L) : 1.0;
    return 0;
}

int ora_root(const float *pos, int64_t n, double lo[3], double *side)
{
    return ora_root_mode(pos, n, lo, side, 0);
}

/* keys in Morton order (order 0) or Peano-Hilbert order (order 1), from the
 * tight root cell or (pow2) the power-of-two one */
int ora_keys_root(const float *pos, int64_t n, double lo[3], double *side, uint64_t *keys,
                  int order, int pow2)
{
    if (ora_root_mode(pos, n, lo, side, pow2)) return 1;
    double scale = 2097152.0 / *side;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) q[a] = ora_quantise(pos[3 * i + a], lo[a], scale);
        keys[i] = order ? ora_hilbert(q[0], q[1], q[2]) : ora_interleave(q[0], q[1], q[2]);
    }
    return 0;
}

int ora_keys_ordered(const float *pos, int64_t n, double lo[3], double *side, uint64_t *keys,
                     int order)
{
    return ora_keys_root(pos, n, lo, side, keys, order, 0);
}

int ora_keys(const float *pos, int64_t n, double lo[3], double *side, uint64_t *keys)
{
    return ora_keys_ordered(pos, n, lo, side, keys, 0);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3 step 2: sort (key, index) pairs; ties by index             */
/* ------------------------------------------------------------------ */

typedef struct { uint64_t key; int64_t idx; } ora_pair;

static int pair_cmp(const void *pa, const void *pb)
{
    const ora_pair *a = (const ora_pair *)pa, *b = (const ora_pair *)pb;
    if (a->key != b->key) return (a->key < b->key) ? -1 : 1;
    if (a->idx != b->idx) return (a->idx < b->idx) ? -1 : 1;
    return 0;
}

void ora_sort(const uint64_t *keys, int64_t n, uint64_t *sorted, int32_t *perm)
{
    ora_pair *p = (ora_pair *)malloc(sizeof(ora_pair) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { p[i].key = keys[i]; p[i].idx = i; }
    qsort(p, (size_t)n, sizeof(ora_pair), pair_cmp);
    for (int64_t i = 0; i < n; ++i) { sorted[i] = p[i].key; perm[i] = (int32_t)p[i].idx; }
    free(p);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1: top-down Barnes-Hut build over the sorted keys            */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    int32_t level;
    int64_t pfirst, pend;
    int64_t parent;   /* index in emission order, -1 for the root */
} ora_cell;

typedef struct ora_tree {
    int64_t n, n_cells;
    int32_t n_crit;
    double lo[3], side;
    uint64_t *skeys;     /* sorted particle keys */
    int32_t *perm;       /* perm[k] = original index of the k-th sorted particle */
    /* canonical (level, key) order */
    uint64_t *ckey;
    uint8_t *level;
    int32_t *parent, *child_first, *child_end, *pfirst, *pend;
    int64_t level_offset[ORA_LEVELS + 1];
    int status;
} ora_tree;

typedef struct { ora_cell *v; int64_t n, cap; } cell_vec;

static int64_t push_cell(cell_vec *cv, ora_cell c)
{
    if (cv->n == cv->cap) {
        cv->cap = cv->cap ? 2 * cv->cap : 1024;
        cv->v = (ora_cell *)realloc(cv->v, sizeof(ora_cell) * (size_t)cv->cap);
    }
    cv->v[cv->n] = c;
    return cv->n++;
}

/* depth-d cell key of a particle key: its upper 3d+1 bits */
static uint64_t prefix(uint64_t key, int d) { return key >> (63 - 3 * d); }

static void split_cell(cell_vec *cv, const uint64_t *sk, int64_t a, int64_t b, int d,
                       int64_t parent, int32_t n_crit)
{
    ora_cell c;
    c.key = prefix(sk[a], d);
    c.level = d;
    c.pfirst = a;
    c.pend = b;
    c.parent = parent;
    int64_t me = push_cell(cv, c);
    if (b - a <= n_crit || d >= ORA_DEPTH_MAX) return;   /* a leaf */
    /* halve along each axis: the octant is the 3-bit digit at depth d+1;
     * sorted keys keep each octant contiguous */
    int64_t s = a;
    while (s < b) {
        uint64_t oct = prefix(sk[s], d + 1);
        int64_t e = s;
        while (e < b && prefix(sk[e], d + 1) == oct) ++e;
        split_cell(cv, sk, s, e, d + 1, me, n_crit);
        s = e;
    }
}

static const ora_cell *g_sort_cells;   /* single-threaded oracle: plain global */
static int idx_cmp(const void *pa, const void *pb)
{
    const ora_cell *a = &g_sort_cells[*(const int64_t *)pa];
    const ora_cell *b = &g_sort_cells[*(const int64_t *)pb];
    if (a->level != b->level) return (a->level < b->level) ? -1 : 1;
    if (a->key != b->key) return (a->key < b->key) ? -1 : 1;
    return 0;
}

ora_tree *ora_build_root(const float *pos, int64_t n, int32_t n_crit, int key_order, int pow2)
{
    ora_tree *t = (ora_tree *)calloc(1, sizeof(ora_tree));
    t->n = n;
    t->n_crit = n_crit;
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    t->skeys = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    t->perm = (int32_t *)malloc(sizeof(int32_t) * nn);
    t->status = ora_keys_root(pos, n, t->lo, &t->side, keys, key_order, pow2);
    ora_sort(keys, n, t->skeys, t->perm);
    free(keys);

    cell_vec cv = {0, 0, 0};
    if (n > 0) split_cell(&cv, t->skeys, 0, n, 0, -1, n_crit);
    int64_t C = cv.n;
    t->n_cells = C;

    /* canonical order: level ascending, key ascending */
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C > 0 ? C : 1));
    int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)(C > 0 ? C : 1));
    for (int64_t i = 0; i < C; ++i) order[i] = i;
    g_sort_cells = cv.v;
    qsort(order, (size_t)C, sizeof(int64_t), idx_cmp);
    for (int64_t i = 0; i < C; ++i) rank[order[i]] = i;

    size_t cc = (size_t)(C > 0 ? C : 1);
    t->ckey = (uint64_t *)malloc(sizeof(uint64_t) * cc);
    t->level = (uint8_t *)malloc(cc);
    t->parent = (int32_t *)malloc(sizeof(int32_t) * cc);
    t->child_first = (int32_t *)malloc(sizeof(int32_t) * cc);
    t->child_end = (int32_t *)malloc(sizeof(int32_t) * cc);
    t->pfirst = (int32_t *)malloc(sizeof(int32_t) * cc);
    t->pend = (int32_t *)malloc(sizeof(int32_t) * cc);
    for (int64_t i = 0; i < C; ++i) {
        const ora_cell *c = &cv.v[order[i]];
        t->ckey[i] = c->key;
        t->level[i] = (uint8_t)c->level;
        t->parent[i] = (c->parent < 0) ? -1 : (int32_t)rank[c->parent];
        t->pfirst[i] = (int32_t)c->pfirst;
        t->pend[i] = (int32_t)c->pend;
        t->child_first[i] = -1;
        t->child_end[i] = -1;
    }
    /* children of a cell: the smallest and one past the largest canonical
     * index among the cells naming it as parent */
    for (int64_t i = 0; i < C; ++i) {
        int32_t p = t->parent[i];
        if (p < 0) continue;
        if (t->child_first[p] < 0 || i < t->child_first[p]) t->child_first[p] = (int32_t)i;
        if (t->child_end[p] < 0 || i + 1 > t->child_end[p]) t->child_end[p] = (int32_t)(i + 1);
    }
    for (int d = 0; d <= ORA_LEVELS; ++d) t->level_offset[d] = 0;
    for (int64_t i = 0; i < C; ++i) t->level_offset[t->level[i] + 1]++;
    for (int d = 0; d < ORA_LEVELS; ++d) t->level_offset[d + 1] += t->level_offset[d];

    free(order);
    free(rank);
    free(cv.v);
    return t;
}

ora_tree *ora_build_ordered(const float *pos, int64_t n, int32_t n_crit, int key_order)
{
    return ora_build_root(pos, n, n_crit, key_order, 0);
}

ora_tree *ora_build(const float *pos, int64_t n, int32_t n_crit)
{
    return ora_build_ordered(pos, n, n_crit, 0);
}

int64_t ora_n_cells(const ora_tree *t) { return t->n_cells; }
int ora_status(const ora_tree *t) { return t->status; }

void ora_get(const ora_tree *t, uint64_t *skeys, int32_t *perm, double *lo, double *side,
             uint64_t *ckey, uint8_t *level, int32_t *parent, int32_t *child_first,
             int32_t *child_end, int32_t *pfirst, int32_t *pend, int64_t *level_offset)
{
    size_t n = (size_t)t->n, C = (size_t)t->n_cells;
    if (skeys) memcpy(skeys, t->skeys, n * sizeof(uint64_t));
    if (perm) memcpy(perm, t->perm, n * sizeof(int32_t));
    if (lo) for (int a = 0; a < 3; ++a) lo[a] = t->lo[a];
    if (side) *side = t->side;
    if (ckey) memcpy(ckey, t->ckey, C * sizeof(uint64_t));
    if (level) memcpy(level, t->level, C);
    if (parent) memcpy(parent, t->parent, C * sizeof(int32_t));
    if (child_first) memcpy(child_first, t->child_first, C * sizeof(int32_t));
    if (child_end) memcpy(child_end, t->child_end, C * sizeof(int32_t));
    if (pfirst) memcpy(pfirst, t->pfirst, C * sizeof(int32_t));
    if (pend) memcpy(pend, t->pend, C * sizeof(int32_t));
    if (level_offset) memcpy(level_offset, t->level_offset, sizeof(t->level_offset));
}

void ora_free(ora_tree *t)
{
    if (!t) return;
    free(t->skeys); free(t->perm); free(t->ckey); free(t->level); free(t->parent);
    free(t->child_first); free(t->child_end); free(t->pfirst); free(t->pend);
    free(t);
}

/* ------------------------------------------------------------------ */
/* Moments by direct summation over each cell's member particles       */
/* ------------------------------------------------------------------ */

static void cell_moments(const ora_tree *t, int64_t c, const float *pos, const float *mass,
                         double m_eq, double *M_out, double com[3], double q[6], float bb[6])
{
    int64_t a = t->pfirst[c], b = t->pend[c];
    double M = 0.0, s[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < 3; ++ax) { bb[ax] = INFINITY; bb[3 + ax] = -INFINITY; }
    for (int64_t k = a; k < b; ++k) {
        int64_t i = t->perm[k];
        double m = mass ? (double)mass[i] : m_eq;
        M += m;
        for (int ax = 0; ax < 3; ++ax) {
            float x = pos[3 * i + ax];
            s[ax] += m * (double)x;
            if (x < bb[ax]) bb[ax] = x;
            if (x > bb[3 + ax]) bb[3 + ax] = x;
        }
    }
    if (M != 0.0) {
        for (int ax = 0; ax < 3; ++ax) com[ax] = s[ax] / M;
    } else {
        int64_t i0 = t->perm[a];
        for (int ax = 0; ax < 3; ++ax) com[ax] = (double)pos[3 * i0 + ax];
    }
    /* central second moment Q_ab = sum m (x_a - c_a)(x_b - c_b), order xx xy xz yy yz zz */
    for (int j = 0; j < 6; ++j) q[j] = 0.0;
    for (int64_t k = a; k < b; ++k) {
        int64_t i = t->perm[k];
        double m = mass ? (double)mass[i] : m_eq;
        double d0 = (double)pos[3 * i + 0] - com[0];
        double d1 = (double)pos[3 * i + 1] - com[1];
        double d2 = (double)pos[3 * i + 2] - com[2];
        q[0] += m * d0 * d0; q[1] += m * d0 * d1; q[2] += m * d0 * d2;
        q[3] += m * d1 * d1; q[4] += m * d1 * d2; q[5] += m * d2 * d2;
    }
    *M_out = M;
}

/* moments of the cells listed in cells[0..nc) (all cells when cells == NULL) */
void ora_moments(const ora_tree *t, const float *pos, const float *mass,
                 const int64_t *cells, int64_t nc, double *M, double *com, double *quad,
                 float *aabb)
{
    double m_eq = (double)(float)(1.0 / (double)(t->n > 0 ? t->n : 1));
    int64_t cnt = cells ? nc : t->n_cells;
    for (int64_t j = 0; j < cnt; ++j) {
        int64_t c = cells ? cells[j] : j;
        cell_moments(t, c, pos, mass, m_eq, &M[j], &com[3 * j], &quad[6 * j], &aabb[6 * j]);
    }
}

/* ------------------------------------------------------------------ */
/* Algorithms 1 and 2 on the sorted keys (second route to the cells)   */
/* ------------------------------------------------------------------ */

typedef struct { uint64_t *key; int64_t *count; int64_t n, cap; } key_list;

static void kl_push(key_list *l, uint64_t key, int64_t count)
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 256;
        l->key = (uint64_t *)realloc(l->key, sizeof(uint64_t) * (size_t)l->cap);
        l->count = (int64_t *)realloc(l->count, sizeof(int64_t) * (size_t)l->cap);
    }
    l->key[l->n] = key;
    l->count[l->n] = count;
    l->n++;
}

/* Leaves straight from the sorted keys (Alg. 1): the first particle k of a
 * leaf sits at depth D_k = max(minDepth(k-1,k), minDepth(k,k+n_leaf)) (the
 * first term only for k > 0, the second only when k+n_leaf < N; App. A),
 * capped at the deepest level 21; the leaf then takes every following
 * particle whose upper 3 D_k + 1 bits equal the leaf key.
 * Parents level by level (Alg. 2): at depth d the sorted leaf keys and the
 * sorted non-leaf keys are walked together, smallest key first; a child whose
 * key >> 3 differs from the parent created last opens a new parent at d-1.
 * Writes every cell as (level, key, particle count), level-major, keys
 * ascending within a level; returns the number of cells, or -1 when out
 * exceeds cap. */
int64_t ora_paper_build(const uint64_t *sk, int64_t n, int32_t n_leaf, int64_t cap,
                        uint8_t *out_level, uint64_t *out_key, int64_t *out_count)
{
    key_list leaves[ORA_LEVELS], inner[ORA_LEVELS];
    memset(leaves, 0, sizeof(leaves));
    memset(inner, 0, sizeof(inner));
    int dmax = 0;
    int64_t k = 0;
    while (k < n) {
        int D = 0;
        if (k > 0) D = ora_min_depth(sk[k - 1], sk[k]);
        if (k + n_leaf < n) {
            int d2 = ora_min_depth(sk[k], sk[k + n_leaf]);
            if (d2 > D) D = d2;
        }
        if (D > ORA_DEPTH_MAX) D = ORA_DEPTH_MAX;
        uint64_t leaf_key = prefix(sk[k], D);
        int64_t first = k;
        while (k < n && prefix(sk[k], D) == leaf_key) ++k;
        kl_push(&leaves[D], leaf_key, k - first);
        if (D > dmax) dmax = D;
    }
    for (int d = dmax; d >= 1; --d) {
        int64_t i = 0, j = 0;
        uint64_t last_parent = 0;   /* no cell key is 0: every key carries the leading 1 */
        while (i < leaves[d].n || j < inner[d].n) {
            uint64_t ck;
            int64_t cnt;
            int take_leaf;
            if (i < leaves[d].n && j < inner[d].n) take_leaf = leaves[d].key[i] < inner[d].key[j];
            else take_leaf = i < leaves[d].n;
            if (take_leaf) { ck = leaves[d].key[i]; cnt = leaves[d].count[i]; ++i; }
            else { ck = inner[d].key[j]; cnt = inner[d].count[j]; ++j; }
            uint64_t pk = ck >> 3;
            if (pk != last_parent) {
                kl_push(&inner[d - 1], pk, 0);
                last_parent = pk;
            }
            inner[d - 1].count[inner[d - 1].n - 1] += cnt;
        }
    }
    /* gather level-major, keys ascending (merge of the two sorted lists) */
    int64_t w = 0;
    for (int d = 0; d < ORA_LEVELS; ++d) {
        int64_t i = 0, j = 0;
        while (i < leaves[d].n || j < inner[d].n) {
            int take_leaf;
            if (i < leaves[d].n && j < inner[d].n) take_leaf = leaves[d].key[i] < inner[d].key[j];
            else take_leaf = i < leaves[d].n;
            if (w >= cap) { w = -1; goto done; }
            out_level[w] = (uint8_t)d;
            if (take_leaf) { out_key[w] = leaves[d].key[i]; out_count[w] = leaves[d].count[i]; ++i; }
            else { out_key[w] = inner[d].key[j]; out_count[w] = inner[d].count[j]; ++j; }
            ++w;
        }
    }
done:
    for (int d = 0; d < ORA_LEVELS; ++d) {
        free(leaves[d].key); free(leaves[d].count);
        free(inner[d].key); free(inner[d].count);
    }
    return w;
}

/* ------------------------------------------------------------------ */
/* Tree walk (Sec. 2.1, Eq. 1) and direct summation                    */
/* ------------------------------------------------------------------ */

static void acc_point(const double r[3], double m, double eps2, double acc[3])
{
    /* softened point mass at offset r = x_target - x_source */
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
    double inv = 1.0 / sqrt(r2);
    double f = m * inv * inv * inv;
    acc[0] -= f * r[0]; acc[1] -= f * r[1]; acc[2] -= f * r[2];
}

/* acceleration (G = 1) on target particle i (original index) from all others */
void ora_direct_acc(const float *pos, const float *mass, int64_t n, double eps,
                    const int64_t *targets, int64_t nt, double *acc)
{
    double m_eq = (double)(float)(1.0 / (double)(n > 0 ? n : 1));
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets[t];
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3];
            for (int ax = 0; ax < 3; ++ax) r[ax] = (double)pos[3 * i + ax] - (double)pos[3 * j + ax];
            acc_point(r, mass ? (double)mass[j] : m_eq, eps * eps, a);
        }
        for (int ax = 0; ax < 3; ++ax) acc[3 * t + ax] = a[ax];
    }
}

/* Walk from the root; a cell that holds the target is always opened; any other
 * cell whose side l = side/2^level and distance d = |x - COM| satisfy l/d < theta
 * is taken as a point mass (plus its quadrupole when use_quad); leaves that fail
 * the test are summed particle by particle.  The quadrupole term uses the
 * traceless tensor T = 3Q - tr(Q) I of the central second moment Q:
 *   a += T r / |r|^5 - (5/2) (r.T r) r / |r|^7,  r = x - COM. */
void ora_tree_walk(const ora_tree *t, const float *pos, const float *mass,
                   const double *cM, const double *ccom, const double *cquad,
                   double theta, double eps, int use_quad,
                   const int64_t *targets, int64_t nt, double *acc)
{
    int64_t n = t->n;
    double m_eq = (double)(float)(1.0 / (double)(n > 0 ? n : 1));
    int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k) inv[t->perm[k]] = k;
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(t->n_cells * 1 + 64));
    for (int64_t ti = 0; ti < nt; ++ti) {
        int64_t i = targets[ti];
        int64_t ki = inv[i];
        double x[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        double a[3] = {0.0, 0.0, 0.0};
        int64_t sp = 0;
        if (t->n_cells > 0) stack[sp++] = 0;
        while (sp > 0) {
            int64_t c = stack[--sp];
            int holds = (ki >= t->pfirst[c] && ki < t->pend[c]);
            double r[3];
            for (int ax = 0; ax < 3; ++ax) r[ax] = x[ax] - ccom[3 * c + ax];
            double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double l = ldexp(t->side, -(int)t->level[c]);
            if (!holds && l < theta * d) {
                acc_point(r, cM[c], eps * eps, a);
                if (use_quad) {
                    const double *q = &cquad[6 * c];
                    double tr = q[0] + q[3] + q[5];
                    double T[3][3] = {{3 * q[0] - tr, 3 * q[1], 3 * q[2]},
                                      {3 * q[1], 3 * q[3] - tr, 3 * q[4]},
                                      {3 * q[2], 3 * q[4], 3 * q[5] - tr}};
                    double Tr[3], rTr = 0.0;
                    for (int u = 0; u < 3; ++u) {
                        Tr[u] = T[u][0] * r[0] + T[u][1] * r[1] + T[u][2] * r[2];
                        rTr += r[u] * Tr[u];
                    }
                    double r2 = d * d, r5 = r2 * r2 * d, r7 = r5 * r2;
                    for (int u = 0; u < 3; ++u) a[u] += Tr[u] / r5 - 2.5 * rTr * r[u] / r7;
                }
            } else if (t->child_first[c] < 0) {
                for (int64_t k = t->pfirst[c]; k < t->pend[c]; ++k) {
                    int64_t j = t->perm[k];
                    if (j == i) continue;
                    double rr[3];
                    for (int ax = 0; ax < 3; ++ax) rr[ax] = x[ax] - (double)pos[3 * j + ax];
                    acc_point(rr, mass ? (double)mass[j] : m_eq, eps * eps, a);
                }
            } else {
                for (int32_t ch = t->child_end[c] - 1; ch >= t->child_first[c]; --ch) stack[sp++] = ch;
            }
        }
        for (int ax = 0; ax < 3; ++ax) acc[3 * ti + ax] = a[ax];
    }
    free(stack);
    free(inv);
}
