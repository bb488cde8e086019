"""Pins of the oracle's Peano-Hilbert keys (the alternative key order of the
footnote in Sec. 2.2): the hand-derived depth-1 order, bijection and face
adjacency along the curve on small grids, cubes as contiguous key ranges,
and the same Barnes-Hut cells as with Morton keys."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(__file__)


def _h(q):
    return np.array([oracle.hilbert(int(a), int(b), int(c)) for a, b, c in q], dtype=np.uint64)


def test_depth1_octant_order_golden():
    rows = np.loadtxt(os.path.join(HERE, "golden", "hilbert_level1.txt"), dtype=np.int64)
    for x, y, z, idx in rows:
        k = oracle.hilbert(int(x) << 20, int(y) << 20, int(z) << 20)
        assert k >> 63 == 1
        assert (k >> 60) & 7 == idx


@pytest.mark.parametrize("k", [1, 2, 3])
def test_grid_bijection_and_face_adjacency(k):
    g = np.arange(1 << k)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    keys = _h(pts << (21 - k))
    top = keys >> np.uint64(63 - 3 * k)
    idx = top - (np.uint64(1) << np.uint64(3 * k))
    assert np.array_equal(np.sort(idx), np.arange(8 ** k, dtype=np.uint64))
    walk = pts[np.argsort(keys)]
    step = np.abs(np.diff(walk, axis=0)).sum(1)
    assert np.all(step == 1)


def test_finest_level_adjacency_inside_random_cells():
    rng = np.random.default_rng(5)
    g = np.arange(4)
    cube = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    for _ in range(20):
        base = rng.integers(0, (1 << 21) // 4, 3) * 4
        pts = base + cube
        keys = _h(pts)
        # one depth-19 cube: a contiguous run of 64 keys sharing 3*19+1 bits
        assert len(set((keys >> np.uint64(6)).tolist())) == 1
        assert np.array_equal(np.sort(keys & np.uint64(63)), np.arange(64, dtype=np.uint64))
        walk = pts[np.argsort(keys)]
        assert np.all(np.abs(np.diff(walk, axis=0)).sum(1) == 1)


def test_cubes_are_key_prefixes():
    rng = np.random.default_rng(6)
    a = rng.integers(0, 1 << 21, (3000, 3))
    # partners in the same cube at some depth, and random partners
    d = rng.integers(1, 22, 3000)
    b = a.copy()
    for i in range(3000):
        mask = (1 << (21 - d[i])) - 1
        b[i] = (a[i] & ~mask) | rng.integers(0, mask + 1, 3)
    c = rng.integers(0, 1 << 21, (3000, 3))
    ka, kb, kc = _h(a), _h(b), _h(c)
    for i in range(3000):
        sh = np.uint64(63 - 3 * int(d[i]))
        assert ka[i] >> sh == kb[i] >> sh
        same = np.all((a[i] >> (21 - d[i])) == (c[i] >> (21 - d[i])))
        assert (ka[i] >> sh == kc[i] >> sh) == same


@pytest.mark.parametrize("seed", range(6))
def test_hilbert_tree_has_the_morton_cells(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(50, 3000))
    pos = rng.random((n, 3)).astype(np.float32)
    if seed % 2:
        pos[: n // 3] = pos[0]                     # duplicates
    n_crit = int(rng.integers(1, 20))
    tm = oracle.build_tree(pos, n_crit, "morton")
    th = oracle.build_tree(pos, n_crit, "hilbert")

    def cells(t):
        out = set()
        for c in range(t.n_cells):
            members = frozenset(t.perm[t.pfirst[c]:t.pend[c]].tolist())
            out.add((int(t.level[c]), members))
        return out

    assert th.n_cells == tm.n_cells
    assert cells(th) == cells(tm)
    # canonical order: level, then Hilbert key
    lv = th.level.astype(np.int64)
    same = lv[1:] == lv[:-1]
    assert np.all(np.diff(lv) >= 0) and np.all(th.ckey[1:][same] > th.ckey[:-1][same])
