"""Parity at the benchmark sizes, in the launch configuration bench.py times.

At these sizes the oracle's full top-down build is too slow for a test, so:
  * keys are compared bit for bit with the oracle's FP64 keys;
  * the permutation is checked to be the unique stable sort of those keys;
  * the cells are checked against properties that determine the Barnes-Hut
    tree uniquely (leaves hold at most n_crit particles unless they are
    depth-21 cells of identical keys, every other cell holds more and has as
    children its non-empty octants, tiling its particle range, keys are the
    members' prefixes, canonical order) -- equivalent to equality;
  * moments are compared on sampled cells with direct FP64 sums over the
    members the oracle finds by key prefix in its own sorted keys.
The 2^24 Plummer workload is compared with the full oracle tree.
"""
import numpy as np
import pytest

import oracle
from synth import WORKLOADS, batched_plummer, jitter_offsets, workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from gpu_util import (TOL_COM, TOL_MASS, TOL_QUAD, assert_structure_equal, moment_errors,  # noqa: E402
                      tb, to_np, torch)

_CACHE = {}


def _data(name):
    if name not in _CACHE:
        spec = WORKLOADS[name]
        pos, mass = workload(spec["kind"], spec["n"], spec["seed"])
        _CACHE[name] = (pos, mass, oracle.PrefixIndex(pos))
    return _CACHE[name]


def _bench_cfg(n):
    """The sort variant bench.py would time: the autotuner's cached choice,
    else the library default."""
    from paper_2312_06102_gb300 import autotune
    return autotune.cached(n)


def check_tree_properties(g, n, n_crit, okeys):
    """g: dict of numpy arrays from the GPU tree."""
    pkey, perm = g["pkey"], g["perm"].astype(np.int64)
    # permutation: a bijection, the stable sort of the oracle's keys
    seen = np.zeros(n, bool)
    seen[perm] = True
    assert seen.all()
    assert np.array_equal(pkey, okeys[perm])
    eq = pkey[1:] == pkey[:-1]
    assert np.all(pkey[1:] >= pkey[:-1])
    assert np.all(perm[1:][eq] > perm[:-1][eq])
    lv = g["level"].astype(np.int64)
    ck = g["ckey"]
    pf, pe = g["pfirst"].astype(np.int64), g["pend"].astype(np.int64)
    cf, ce = g["child_first"].astype(np.int64), g["child_end"].astype(np.int64)
    par = g["parent"].astype(np.int64)
    C = len(lv)
    # canonical order: level, then key, strictly
    assert np.all(np.diff(lv) >= 0)
    same = lv[1:] == lv[:-1]
    assert np.all(ck[1:][same] > ck[:-1][same])
    # root
    assert lv[0] == 0 and ck[0] == 1 and pf[0] == 0 and pe[0] == n and par[0] == -1
    # key prefixes of the first and last member
    sh = (63 - 3 * lv).astype(np.uint64)
    assert np.all(pkey[pf] >> sh == ck) and np.all(pkey[pe - 1] >> sh == ck)
    cnt = pe - pf
    assert np.all(cnt >= 1)
    leaf = cf < 0
    assert np.all(ce[leaf] == -1)
    # leaves: <= n_crit, or depth-21 cells of identical keys
    big = leaf & (cnt > n_crit)
    assert np.all(lv[big] == 21)
    assert np.all(pkey[pf[big]] == pkey[pe[big] - 1])
    # other cells: > n_crit, shallower than 21, 1..8 children
    inner = ~leaf
    assert np.all(cnt[inner] > n_crit) and np.all(lv[inner] < 21)
    nch = ce - cf
    assert np.all((nch[inner] >= 1) & (nch[inner] <= 8))
    # every non-root cell: parent links agree, one level up, key >> 3
    c = np.arange(1, C)
    p = par[1:]
    assert np.all((p >= 0) & (p < C))
    assert np.all((cf[p] <= c) & (c < ce[p]))
    assert np.all(lv[c] == lv[p] + 1)
    assert np.all(ck[c] >> np.uint64(3) == ck[p])
    assert np.array_equal(np.bincount(p, minlength=C)[inner], nch[inner])
    # children tile their parent's particles
    assert np.all(pf[cf[inner]] == pf[inner]) and np.all(pe[ce[inner] - 1] == pe[inner])
    sib = par[1:] == par[:-1]
    assert np.all(pf[1:][sib] == pe[:-1][sib])
    # leaves partition the particles
    lpf = np.sort(pf[leaf])
    lpe = pe[leaf][np.argsort(pf[leaf])]
    assert lpf[0] == 0 and lpe[-1] == n and np.all(lpf[1:] == lpe[:-1])
    # level offsets
    return leaf


def _gpu_arrays(t):
    return {k: to_np(getattr(t, k)) for k in ("pkey", "perm", "ckey", "level", "parent",
                                             "child_first", "child_end", "pfirst", "pend")}


def _sample_cells(lv, leaf, rng, per_level=60, extra_leaves=300):
    """The root, a few cells of each shallow level (each holds a large share
    of the particles, so its direct sum is costly), per_level random cells of
    every deeper level, and random leaves."""
    cells = [np.array([0])]
    for d in range(1, 22):
        idx = np.nonzero(lv == d)[0]
        if len(idx) == 0:
            continue
        k = 2 if d <= 2 else (per_level if d > 4 else per_level // 4)
        cells.append(rng.choice(idx, min(k, len(idx)), replace=False))
    extra = rng.choice(np.nonzero(leaf)[0], extra_leaves, replace=False)
    return np.unique(np.concatenate(cells + [extra]))


def _check_moments(t, g, idx, mass, cells, mode=0):
    M, com, quad, aabb, cnt = idx.moments(mass, g["level"][cells], g["ckey"][cells])
    assert np.array_equal(cnt, (g["pend"] - g["pfirst"])[cells].astype(np.int64))
    em, ec, eq, bb_ok = moment_errors(t, None, M, com, quad, aabb, cells=cells, mode=mode)
    assert bb_ok
    return em, ec, eq


def _build(pos, mass, n_crit, mode=0, cfg=None):
    m = tb()
    p = torch.from_numpy(pos).cuda()
    w = torch.from_numpy(mass).cuda()
    t = m.build(p, w, n_crit=n_crit, mom_mode=mode, sort_cfg=cfg)
    m.moments(t, p, w)
    torch.cuda.synchronize()
    assert t.sync() == 0
    return t


def test_plummer_2p24_full_oracle():
    spec = WORKLOADS["plummer_2p24"]
    pos, mass = workload(spec["kind"], spec["n"], spec["seed"])
    t = _build(pos, mass, 16, cfg=_bench_cfg(spec["n"]))
    o = oracle.build_tree(pos, 16)
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
    assert bb_ok
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


def test_disk_2p24_full_oracle():
    spec = WORKLOADS["disk_2p24"]
    pos, mass = workload(spec["kind"], spec["n"], spec["seed"])
    t = _build(pos, mass, 16, cfg=_bench_cfg(spec["n"]))
    o = oracle.build_tree(pos, 16)
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
    assert bb_ok
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


@pytest.mark.parametrize("n_crit", [16, 8, 32])
def test_clustered_2p27(n_crit):
    pos, mass, idx = _data("clustered_2p27")
    n = pos.shape[0]
    t = _build(pos, mass, n_crit, cfg=_bench_cfg(n))
    g = _gpu_arrays(t)
    leaf = check_tree_properties(g, n, n_crit, idx.keys)
    assert np.allclose(t.lo, idx.lo, rtol=0, atol=0) and t.side == idx.side
    rng = np.random.default_rng(n_crit)
    cells = _sample_cells(g["level"], leaf, rng, per_level=40 if n_crit != 16 else 80,
                          extra_leaves=100 if n_crit != 16 else 300)
    em, ec, eq = _check_moments(t, g, idx, mass, cells)
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


@pytest.mark.parametrize("mode", [0, 2])
def test_precision_stress_2p26(mode):
    pos, mass, idx = _data("stress_2p26")
    n = pos.shape[0]
    t = _build(pos, mass, 16, mode=mode, cfg=_bench_cfg(n))
    g = _gpu_arrays(t)
    leaf = check_tree_properties(g, n, 16, idx.keys)
    assert t.max_depth >= 18
    cells = _sample_cells(g["level"], leaf, np.random.default_rng(5))
    em, ec, eq = _check_moments(t, g, idx, mass, cells, mode=mode)
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


def test_batched_4096_sampled_sets():
    """The full batched workload at replay steps 0, 1 and 99: the build is
    captured in a CUDA graph with a fixed cell capacity (as timed) and replayed
    on the jittered positions of each step.  At step 0 the largest, the
    smallest and 30 other sets are checked whole, at steps 1 and 99 the
    largest and 10 others."""
    from test_gpu_batched import _check_sets, _run
    m = tb()
    b = batched_plummer(n_sets=4096, seed=4)
    t, p, w, off = _run(b.pos, b.mass, b.offsets)
    sizes = np.diff(b.offsets)
    rng = np.random.default_rng(44)
    sets = sorted(set([int(np.argmax(sizes)), int(np.argmin(sizes))] +
                      list(rng.choice(4096, 30, replace=False))))
    _check_sets(t, b.pos, b.mass, b.offsets, 16, sets=sets)

    cap = int(t.n_cells * 1.05) + 4096
    m.build_batched(p, w, off, cell_capacity=cap, tree=t)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m.build_batched(p, w, off, cell_capacity=cap, tree=t, stream=s)
    for step in (1, 99):
        pj = (b.pos + jitter_offsets(4, step, b.offsets, b.scale)).astype(np.float32)
        p.copy_(torch.from_numpy(pj))
        g.replay()
        torch.cuda.synchronize()
        assert t.sync() == 0
        few = sorted(set([int(np.argmax(sizes))] + list(rng.choice(4096, 10, replace=False))))
        _check_sets(t, pj, b.mass, b.offsets, 16, sets=few)
