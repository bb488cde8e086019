"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

None of these tests retypes an oracle formula: each checks the oracle
against a worked example of the paper, a hand-worked case, a closed form,
an independent brute-force definition or an invariant, chosen so that a
dropped term, a wrong sign or index or a transposed operand fails one.
"""
import math
import os
from itertools import product

import numpy as np
import pytest

import oracle
from synth import clustered_halos, lattice, plummer, precision_stress, uniform_cube

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- minDepth

def test_min_depth_paper_example():
    """Sec. 2.3.1 worked example: 1010011... vs 1011011... -> depth 1."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "min_depth_example.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for a, b, want in rows:
        ka = int(a, 2) << (64 - len(a))
        kb = int(b, 2) << (64 - len(b))
        assert oracle.min_depth(ka, kb) == int(want)
        assert oracle.min_depth(kb, ka) == int(want)


@pytest.mark.parametrize("clz,depth", [(1, 1), (2, 1), (3, 1), (4, 2), (6, 2), (7, 3),
                                       (61, 21), (63, 21), (64, 22)])
def test_min_depth_hand_cases(clz, depth):
    a = (1 << 63) | 0x5A5A
    b = a ^ (1 << (63 - clz)) if clz < 64 else a
    assert oracle.min_depth(a, b) == depth


# ---------------------------------------------------------------- keys

def test_interleave_corners():
    assert oracle.interleave(0, 0, 0) == 1 << 63
    m = (1 << 21) - 1
    assert oracle.interleave(m, m, m) == (1 << 64) - 1
    # lowest digit: x is the most significant bit of each 3-bit group
    assert oracle.interleave(1, 0, 0) == (1 << 63) | 0b100
    assert oracle.interleave(0, 1, 0) == (1 << 63) | 0b010
    assert oracle.interleave(0, 0, 1) == (1 << 63) | 0b001
    # highest digit sits right below the leading 1
    assert oracle.interleave(1 << 20, 0, 0) == (1 << 63) | (1 << 62)
    assert oracle.interleave(0, 0, 1 << 20) == (1 << 63) | (1 << 60)
    # a hand-built pattern: q = 0b101 (x), 0b011 (y), 0b110 (z) in the low bits
    # digits (top to bottom of the three low levels): x2y2z2=1 0 1, x1y1z1=0 1 1, x0y0z0=1 1 0
    assert oracle.interleave(0b101, 0b011, 0b110) == (1 << 63) | 0b101_011_110


def test_quantise_edges():
    s = 2.0 ** 21
    assert oracle.quantise(0.0, 0.0, s) == 0
    assert oracle.quantise(1.0, 0.0, s) == (1 << 21) - 1          # clamp at the top
    assert oracle.quantise(0.5, 0.0, s) == 1 << 20                 # exact grid point
    assert oracle.quantise(float(np.float32(0.5) - np.float32(2 ** -24)), 0.0, s) == (1 << 20) - 1
    # an offset box of side 4 at 1000: q = floor((x - 1000) * 2^19); points on
    # the fp32 grid (spacing 2^-14 near 1000) that are exact multiples of 2^-19
    for k in (0, 32, 1 << 10, 12345 * 32, (1 << 21) - 32):
        x = 1000.0 + k * 2.0 ** -19
        assert float(np.float32(x)) == x
        assert oracle.quantise(x, 1000.0, 2.0 ** 21 / 4.0) == k
        # one fp32 step (2^-14 = 32 grid cells near 1000) below the grid point
        xb = float(np.nextafter(np.float32(x), np.float32(0)))
        if k:
            assert oracle.quantise(xb, 1000.0, 2.0 ** 21 / 4.0) == k - 32


def test_keys_geometry_depth1():
    """The depth-1 digit of each key is the octant of the root cube's centre
    (x high -> 4, y high -> 2, z high -> 1) -- closed-form geometry."""
    pos, _ = uniform_cube(4096, 11)
    k, lo, side = oracle.keys(pos)
    assert np.all(k >> np.uint64(63) == 1)
    mid = lo + side / 2
    p = pos.astype(np.float64)
    far = np.all(np.abs(p - mid) > 1e-6 * side, axis=1)
    want = ((p[:, 0] >= mid[0]).astype(int) << 2) | ((p[:, 1] >= mid[1]).astype(int) << 1) \
        | (p[:, 2] >= mid[2]).astype(int)
    got = ((k >> np.uint64(60)) & np.uint64(7)).astype(int)
    assert np.array_equal(got[far], want[far])


def test_keys_root_is_tight_box():
    pos, _ = plummer(2000, 2)
    k, lo, side = oracle.keys(pos)
    assert np.allclose(lo, pos.min(0).astype(np.float64), rtol=0, atol=0)
    ext = pos.max(0).astype(np.float64) - pos.min(0).astype(np.float64)
    assert side == ext.max()
    # the particle at the largest coordinate of the widest axis clamps to 2^21-1
    ax = int(np.argmax(ext))
    i = int(np.argmax(pos[:, ax]))
    shift = 2 - ax
    q = 0
    for b in range(21):
        q |= int((int(k[i]) >> (3 * b + shift)) & 1) << b
    assert q == (1 << 21) - 1


@pytest.mark.parametrize("ext,want", [(3.0, 4.0), (4.0, 4.0), (0.125, 0.125), (0.3, 0.5),
                                      (1e-3, 2.0 ** -9), (5000.0, 8192.0), (0.0, 1.0)])
def test_root_pow2_side(ext, want):
    """The power-of-two root (Sec. 2.2): the side is the smallest power of two
    at least the largest extent (1 for a single point); the corner stays at
    the per-axis minimum, and the tight root keeps the extent itself."""
    e32 = float(np.float32(ext))
    pos = np.array([[0.0, 0.0, 0.0], [e32, e32 / 2, 0.0], [e32 / 4, e32, e32 / 8]], np.float32)
    lo, side = oracle.root(pos, "pow2")
    assert np.array_equal(lo, [0.0, 0.0, 0.0])
    assert side == want
    lo_t, side_t = oracle.root(pos, "tight")
    assert side_t == (e32 if e32 > 0 else 1.0)


def test_keys_pow2_root_hand_point():
    """With extent 3 the power-of-two side is 4 and the scale 2^19 exactly:
    (3, 1.5, 0.75) quantises to (3, 1.5, 0.75) * 2^19, and its key, built here
    bit by bit, has the octant digits 4, 6, 3, 1, 0, ... (the tight root, side
    3, starts with 6 instead)."""
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 1.5, 0.75]], np.float32)
    q = (3 * 2 ** 19, 3 * 2 ** 18, 3 * 2 ** 17)
    want = 1
    for b in range(20, -1, -1):
        want = (want << 3) | (((q[0] >> b) & 1) << 2) | (((q[1] >> b) & 1) << 1) | ((q[2] >> b) & 1)
    k, lo, side = oracle.keys(pos, root_mode="pow2")
    assert side == 4.0 and int(k[1]) == want and int(k[0]) == 1 << 63
    assert [(want >> (60 - 3 * j)) & 7 for j in range(5)] == [4, 6, 3, 1, 0]
    kt, _, side_t = oracle.keys(pos)
    assert side_t == 3.0 and (int(kt[1]) >> 60) & 7 == 6


@pytest.mark.parametrize("root_mode", ["pow2", "tight"])
def test_tree_cell_boxes(root_mode):
    """Every cell of level d is the cube of side side / 2^d at the integer
    corner its key spells out (x, y, z bits of each octant digit), and each
    of its members lies in it -- under the power-of-two root and the tight
    one alike."""
    pos, _ = clustered_halos(6000, 9, n_halo=40)
    t = oracle.build_tree(pos, 8, root_mode=root_mode)
    _check_invariants(t)
    if root_mode == "pow2":
        assert math.log2(t.side) == int(math.log2(t.side))
    p = pos.astype(np.float64)[t.perm]
    for c in range(t.n_cells):
        d = int(t.level[c])
        key = int(t.ckey[c])
        ijk = [0, 0, 0]
        for j in range(d):
            dig = (key >> (3 * (d - 1 - j))) & 7
            for a in range(3):
                ijk[a] = (ijk[a] << 1) | ((dig >> (2 - a)) & 1)
        h = t.side / 2 ** d
        mem = p[t.pfirst[c]:t.pend[c]]
        for a in range(3):
            lo_c = t.lo[a] + ijk[a] * h
            assert np.all(mem[:, a] >= lo_c - 1e-12 * t.side)
            assert np.all(mem[:, a] <= lo_c + h + 1e-12 * t.side)


def test_keys_monotone_per_axis():
    """Moving one coordinate up never lowers that axis's quantised value
    (read back from the key by de-interleaving)."""
    rng = np.random.default_rng(5)
    base = rng.random((200, 3)).astype(np.float32)
    pts = np.concatenate([base, np.array([[0, 0, 0], [1, 1, 1]], np.float32)])
    k0, lo, side = oracle.keys(pts)
    up = pts.copy()
    up[:-2, 1] = np.minimum(up[:-2, 1] + np.float32(0.01), np.float32(1.0))
    k1, lo1, side1 = oracle.keys(up)
    assert side1 == side and np.array_equal(lo1, lo)

    def qy(k):
        out = np.zeros(k.shape, np.int64)
        for b in range(21):
            out |= (((k >> np.uint64(3 * b + 1)) & np.uint64(1)).astype(np.int64) << b)
        return out

    assert np.all(qy(k1[:-2]) >= qy(k0[:-2]))


# ---------------------------------------------------------------- sort

def test_sort_brute_force_with_duplicates():
    rng = np.random.default_rng(7)
    keys = (rng.integers(0, 40, 3000).astype(np.uint64) | np.uint64(1 << 63))
    sk, perm = oracle.sort(keys)
    want = sorted(range(len(keys)), key=lambda i: (int(keys[i]), i))
    assert perm.tolist() == want
    assert np.array_equal(sk, keys[perm])


# ---------------------------------------------------------------- tree

def _brute_cells(pos, n_crit):
    """Cells by the set definition of the Barnes-Hut tree: the root exists if
    n > 0; a depth-d prefix with at least one particle is a cell when its parent
    prefix is a cell holding more than n_crit particles at depth < 21."""
    k, lo, side = oracle.keys(pos)
    keys = [int(x) for x in k]
    cells = {}
    if not keys:
        return cells
    cells[(0, 1)] = len(keys)
    for d in range(1, 22):
        counts = {}
        for key in keys:
            p = key >> (63 - 3 * d)
            counts[p] = counts.get(p, 0) + 1
        for p, c in counts.items():
            par = (d - 1, p >> 3)
            if par in cells and cells[par] > n_crit:
                cells[(d, p)] = c
    return cells


@pytest.mark.parametrize("seed", range(40))
def test_tree_matches_brute_force_tiny(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 65))
    n_crit = int(rng.integers(1, 6))
    if seed % 3 == 0:  # duplicate-heavy
        pos = rng.integers(0, 3, (n, 3)).astype(np.float32)
    else:
        pos = rng.random((n, 3)).astype(np.float32)
    t = oracle.build_tree(pos, n_crit)
    want = _brute_cells(pos, n_crit)
    got = {(int(l), int(k)): int(e - f) for l, k, f, e in zip(t.level, t.ckey, t.pfirst, t.pend)}
    assert got == want
    # canonical order
    order = sorted(got)
    assert [(int(l), int(k)) for l, k in zip(t.level, t.ckey)] == order


def test_hand_tree_golden():
    pts, cells = [], []
    for line in open(os.path.join(GOLDEN, "hand_tree_8.txt")):
        if line.startswith("p "):
            pts.append([float(v) for v in line.split()[1:]])
        elif line.startswith("c "):
            _, lv, key, cnt, leaf = line.split()
            cells.append((int(lv), int(key, 2), int(cnt), int(leaf)))
    pos = np.array(pts, np.float32)
    t = oracle.build_tree(pos, 2)
    got = [(int(l), int(k), int(e - f), int(c < 0))
           for l, k, f, e, c in zip(t.level, t.ckey, t.pfirst, t.pend, t.child_first)]
    assert got == cells


@pytest.mark.parametrize("k", [1, 2, 3])
def test_complete_octree_lattice(k):
    """8^k lattice points, n_crit = 1: every cell splits down to depth k, so
    there are sum_{d<=k} 8^d cells and every leaf sits at depth k."""
    pos, _ = lattice(k)
    t = oracle.build_tree(pos, 1)
    assert t.n_cells == sum(8 ** d for d in range(k + 1))
    leaves = t.child_first < 0
    assert np.all(t.level[leaves] == k)
    assert np.all(t.pend[leaves] - t.pfirst[leaves] == 1)
    for d in range(k + 1):
        assert t.level_offset[d + 1] - t.level_offset[d] == 8 ** d


def _check_invariants(t):
    n, C = t.n, t.n_cells
    leaf = t.child_first < 0
    cnt = (t.pend - t.pfirst).astype(np.int64)
    # each particle in exactly one leaf
    cover = np.zeros(n, np.int64)
    for f, e in zip(t.pfirst[leaf], t.pend[leaf]):
        cover[f:e] += 1
    assert np.all(cover == 1)
    assert cnt[leaf].sum() == n
    # leaves hold <= n_crit, except depth-21 leaves whose keys are all equal
    big = leaf & (cnt > t.n_crit)
    for c in np.nonzero(big)[0]:
        assert t.level[c] == 21
        assert np.all(t.skeys[t.pfirst[c]:t.pend[c]] == t.skeys[t.pfirst[c]])
    # non-leaves hold more than n_crit
    assert np.all(cnt[~leaf] > t.n_crit)
    # child ranges tile the parent's range; parent links agree; keys are prefixes
    for c in np.nonzero(~leaf)[0]:
        ch = np.arange(t.child_first[c], t.child_end[c])
        assert 1 <= len(ch) <= 8
        assert np.all(t.parent[ch] == c)
        assert np.all(t.level[ch] == t.level[c] + 1)
        assert t.pfirst[ch[0]] == t.pfirst[c] and t.pend[ch[-1]] == t.pend[c]
        assert np.all(t.pfirst[ch[1:]] == t.pend[ch[:-1]])
        assert np.all(t.ckey[ch] >> np.uint64(3) == t.ckey[c])
    assert t.parent[0] == -1 and t.level[0] == 0 and t.ckey[0] == 1
    # each cell key is the prefix of its member particles' keys
    sh = (63 - 3 * t.level.astype(np.int64)).astype(np.uint64)
    assert np.all(t.skeys[t.pfirst] >> sh == t.ckey)
    assert np.all(t.skeys[t.pend - 1] >> sh == t.ckey)
    # level offsets
    lv = np.searchsorted(t.level, np.arange(23), side="left")
    assert np.array_equal(lv, t.level_offset)


@pytest.mark.parametrize("gen,n,n_crit", [("uniform", 20000, 16), ("plummer", 20000, 8),
                                          ("clustered", 30000, 16), ("stress", 30000, 16),
                                          ("uniform", 5, 16), ("uniform", 16, 16),
                                          ("uniform", 17, 16)])
def test_tree_invariants(gen, n, n_crit):
    pos = {"uniform": lambda: uniform_cube(n, 3)[0], "plummer": lambda: plummer(n, 4)[0],
           "clustered": lambda: clustered_halos(n, 5, n_halo=300)[0],
           "stress": lambda: precision_stress(n, 6, n_halo=300)[0]}[gen]()
    t = oracle.build_tree(pos, n_crit)
    _check_invariants(t)
    if n <= n_crit:
        assert t.n_cells == 1 and t.child_first[0] == -1


def test_all_identical_positions():
    pos = np.full((100, 3), 0.25, np.float32)
    t = oracle.build_tree(pos, 4)
    # side falls back to 1; every key is 2^63; the chain runs to depth 21
    assert t.n_cells == 22
    assert t.level.tolist() == list(range(22))
    assert t.pend[-1] - t.pfirst[-1] == 100
    _check_invariants(t)


def test_empty_input():
    t = oracle.build_tree(np.zeros((0, 3), np.float32), 16)
    assert t.n_cells == 0


# ------------------------------------------- Algorithms 1 and 2 (App. A)

@pytest.mark.parametrize("seed", range(60))
def test_paper_algorithms_equal_top_down(seed):
    """App. A: the leaves of Alg. 1 and the parents of Alg. 2 are exactly the
    cells of the top-down Barnes-Hut build (random and duplicate-heavy)."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 3000))
    n_crit = int(rng.integers(1, 40))
    kind = seed % 4
    if kind == 0:
        pos = rng.random((n, 3)).astype(np.float32)
    elif kind == 1:
        pos = rng.integers(0, 4, (n, 3)).astype(np.float32)   # many identical keys
    elif kind == 2:
        pos = (1000 + rng.normal(0, 1e-3, (n, 3))).astype(np.float32)  # fp32 grid at 1000
    else:
        pos = plummer(n, seed)[0]
    t = oracle.build_tree(pos, n_crit)
    lv, k, c = oracle.paper_build(t.skeys, n_crit)
    assert np.array_equal(lv, t.level)
    assert np.array_equal(k, t.ckey)
    assert np.array_equal(c, (t.pend - t.pfirst).astype(np.int64))


# ---------------------------------------------------------------- moments

def test_moments_single_particle_cells():
    pos, _ = lattice(2)
    rng = np.random.default_rng(3)
    mass = rng.random(pos.shape[0]).astype(np.float32) + np.float32(0.5)
    t = oracle.build_tree(pos, 1)
    M, com, q, bb = oracle.moments(t, pos, mass)
    leaf = t.child_first < 0
    i = t.perm[t.pfirst[leaf]]
    assert np.array_equal(M[leaf], mass[i].astype(np.float64))
    assert np.array_equal(com[leaf], pos[i].astype(np.float64))
    assert np.all(q[leaf] == 0)
    assert np.array_equal(bb[leaf][:, :3], pos[i]) and np.array_equal(bb[leaf][:, 3:], pos[i])


def test_moments_two_particle_closed_form():
    """Two masses: COM on the segment, Q = (m1 m2 / M) (x1 - x2)(x1 - x2)^T."""
    x1 = np.array([0.25, 0.5, 0.125], np.float32)
    x2 = np.array([0.75, 0.0625, 0.875], np.float32)
    m = np.array([3.0, 1.0], np.float32)
    t = oracle.build_tree(np.stack([x1, x2]), 4)
    M, com, q, bb = oracle.moments(t, np.stack([x1, x2]), m)
    Mt = 4.0
    d = (x1 - x2).astype(np.float64)
    want_q = (3.0 * 1.0 / Mt) * np.outer(d, d)
    assert M[0] == Mt
    assert np.allclose(com[0], (3 * x1.astype(np.float64) + x2) / Mt, rtol=0, atol=1e-15)
    got = np.array([[q[0, 0], q[0, 1], q[0, 2]], [q[0, 1], q[0, 3], q[0, 4]],
                    [q[0, 2], q[0, 4], q[0, 5]]])
    assert np.allclose(got, want_q, rtol=1e-14, atol=1e-16)
    assert np.array_equal(bb[0], np.concatenate([np.minimum(x1, x2), np.maximum(x1, x2)]))


def _qmat(q):
    return np.array([[q[0], q[1], q[2]], [q[1], q[3], q[4]], [q[2], q[4], q[5]]])


def test_moments_raw_moment_identity_and_bottom_up():
    """Q equals sum m x x^T - M c c^T (the raw-moment form), and every parent
    equals the parallel-axis combination of its children."""
    pos, _ = plummer(6000, 9)
    rng = np.random.default_rng(9)
    mass = np.exp(rng.normal(0, 1, pos.shape[0])).astype(np.float32)
    t = oracle.build_tree(pos, 8)
    M, com, q, bb = oracle.moments(t, pos, mass)
    p64 = pos.astype(np.float64)
    m64 = mass.astype(np.float64)
    for c in [0, 1, 5, t.n_cells // 2, t.n_cells - 1]:
        idx = t.perm[t.pfirst[c]:t.pend[c]]
        raw = (m64[idx, None, None] * p64[idx, :, None] * p64[idx, None, :]).sum(0)
        want = raw - M[c] * np.outer(com[c], com[c])
        scale = M[c] * (t.side / 2.0 ** int(t.level[c])) ** 2
        assert np.abs(_qmat(q[c]) - want).max() <= 1e-9 * scale
    for c in np.nonzero(t.child_first >= 0)[0]:
        ch = np.arange(t.child_first[c], t.child_end[c])
        Mp = M[ch].sum()
        cp = (M[ch, None] * com[ch]).sum(0) / Mp
        Qp = sum(_qmat(q[j]) + M[j] * np.outer(com[j] - cp, com[j] - cp) for j in ch)
        s = t.side / 2.0 ** int(t.level[c])
        assert abs(Mp / M[c] - 1) < 1e-13
        assert np.abs(cp - com[c]).max() < 1e-12 * s
        assert np.abs(Qp - _qmat(q[c])).max() < 1e-11 * M[c] * s * s
        assert np.array_equal(bb[c][:3], bb[ch][:, :3].min(0))
        assert np.array_equal(bb[c][3:], bb[ch][:, 3:].max(0))


def test_moments_translation_and_axis_permutation():
    """Shifting every particle by an exact power of two shifts the COM and
    leaves Q unchanged; cycling the axes cycles Q's components."""
    pos, _ = uniform_cube(3000, 21)
    # on a 2^-20 grid, so that adding 4 is exact in FP32
    pos = (np.floor(pos.astype(np.float64) * 2 ** 20) / 2 ** 20).astype(np.float32)
    rng = np.random.default_rng(21)
    mass = rng.random(3000).astype(np.float32) + np.float32(0.1)
    t = oracle.build_tree(pos, 8)
    M, com, q, bb = oracle.moments(t, pos, mass)
    shifted = pos + np.float32(4.0)
    t2 = oracle.build_tree(shifted, 8)
    assert np.array_equal(t2.ckey, t.ckey)
    M2, com2, q2, bb2 = oracle.moments(t2, shifted, mass)
    assert np.allclose(M2, M, rtol=1e-15, atol=0)
    assert np.abs(com2 - 4.0 - com).max() < 1e-14
    assert np.abs(q2 - q).max() < 1e-9 * M.max()
    # axis cycle (x,y,z) -> (y,z,x): the root's Q permutes accordingly
    cyc = pos[:, [1, 2, 0]].copy()
    t3 = oracle.build_tree(cyc, 8)
    M3, com3, q3, bb3 = oracle.moments(t3, cyc, mass)
    Q = _qmat(q[0])
    Q3 = _qmat(q3[0])
    P = np.eye(3)[[1, 2, 0]]
    assert np.allclose(Q3, P @ Q @ P.T, rtol=1e-12, atol=1e-15)
    assert np.allclose(com3[0], com[0][[1, 2, 0]], rtol=1e-14, atol=0)


def test_moments_equal_masses_default():
    pos, _ = uniform_cube(1000, 2)
    t = oracle.build_tree(pos, 16)
    M0, c0, q0, b0 = oracle.moments(t, pos, None)
    M1, c1, q1, b1 = oracle.moments(t, pos, np.full(1000, np.float32(1.0 / 1000)))
    assert np.array_equal(M0, M1) and np.array_equal(c0, c1) and np.array_equal(q0, q1)


# ---------------------------------------------------------------- tree walk

def _forces(n, theta, use_quad=True, seed=31):
    pos, mass = plummer(n, seed, a=0.1)
    t = oracle.build_tree(pos, 8)
    M, com, q, _ = oracle.moments(t, pos, mass)
    targets = np.arange(0, n, max(1, n // 512))
    eps = 1e-3 * t.side
    acc_t = oracle.tree_walk(t, pos, mass, M, com, q, targets, theta, eps, use_quad)
    acc_d = oracle.direct_acc(pos, mass, targets, eps)
    err = np.linalg.norm(acc_t - acc_d, axis=1) / np.linalg.norm(acc_d, axis=1)
    return err


def test_tree_walk_theta_zero_is_direct_sum():
    err = _forces(2048, 0.0)
    assert err.max() < 1e-12


def test_tree_walk_theta_half_against_direct():
    """Opening angle 0.5 against O(N^2) summation at N = 4096."""
    err = _forces(4096, 0.5)
    assert np.median(err) <= 1e-3
    assert np.quantile(err, 0.99) <= 1e-2


def test_tree_walk_quadrupole_helps_and_error_grows_with_theta():
    e_mono = _forces(4096, 0.7, use_quad=False)
    e_quad = _forces(4096, 0.7, use_quad=True)
    assert np.median(e_quad) < 0.5 * np.median(e_mono)
    meds = [np.median(_forces(4096, th)) for th in (0.3, 0.6, 0.9)]
    assert meds[0] < meds[1] < meds[2]


def test_prefix_index_moments_equal_tree_moments():
    """The prefix-located direct sums agree with the top-down tree's direct
    sums cell by cell (member sets and FP64 values)."""
    pos, _ = clustered_halos(20_000, 17, n_halo=100)
    rng = np.random.default_rng(17)
    mass = (rng.random(20_000) + 0.1).astype(np.float32)
    t = oracle.build_tree(pos, 8)
    idx = oracle.PrefixIndex(pos)
    assert np.array_equal(idx.skeys, t.skeys) and np.array_equal(idx.order, t.perm)
    cells = np.arange(0, t.n_cells, max(1, t.n_cells // 300))
    M, com, quad, aabb, cnt = idx.moments(mass, t.level[cells], t.ckey[cells])
    M2, com2, quad2, aabb2 = oracle.moments(t, pos, mass, cells)
    assert np.array_equal(cnt, (t.pend - t.pfirst)[cells])
    assert np.allclose(M, M2, rtol=1e-13, atol=0)
    s = t.side / np.exp2(t.level[cells].astype(np.int64))
    assert (np.abs(com - com2).max(1) / s).max() < 1e-10
    assert (np.abs(quad - quad2).max(1) / (M * s * s)).max() < 1e-9
    assert np.array_equal(aabb, aabb2)
