"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Structure -- keys, permutation, cells, levels, links, ranges -- must be
bit-exact; moments must meet the tolerances in gpu_util.  Sizes span several
sort tiles (4096) and level tiles (4096) with ragged tails.
"""
import numpy as np
import pytest

import oracle
from synth import clustered_halos, exponential_disk, lattice, plummer, precision_stress, uniform_cube

pytestmark = pytest.mark.gpu

from gpu_util import (TOL_COM, TOL_MASS, TOL_QUAD, assert_structure_equal, gpu_tree,  # noqa: E402
                      moment_errors, tb, to_np, torch)


def _check(pos, mass, n_crit, mode=0, radix_bits=0, cell_capacity=0, tol_scale=1.0):
    o = oracle.build_tree(pos, n_crit)
    t, p, w = gpu_tree(pos, mass, n_crit, mode=mode, radix_bits=radix_bits,
                       cell_capacity=cell_capacity)
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb, mode=mode)
    assert bb_ok
    assert em.max() <= TOL_MASS * tol_scale, em.max()
    assert ec.max() <= TOL_COM * tol_scale, ec.max()
    assert eq.max() <= TOL_QUAD * tol_scale, eq.max()
    return t, o


def test_uniform_65536():
    """Plain single build, N = 65,536 uniform, n_crit = 16 (the small workload)."""
    pos, mass = uniform_cube(65536, 1)
    _check(pos, mass, 16)


@pytest.mark.parametrize("n", [1, 2, 3, 15, 16, 17, 33, 4095, 4096, 4097, 3 * 4096 + 77,
                               50_001])
def test_ragged_sizes(n):
    pos, mass = uniform_cube(n, 1000 + n)
    _check(pos, mass, 16)


@pytest.mark.parametrize("radix_bits", [8, 9, 10, 11])
def test_radix_widths(radix_bits):
    pos, mass = plummer(70_000, 7)
    _check(pos, mass, 8, radix_bits=radix_bits)


def test_every_sort_variant():
    """Every compiled radix-sort shape (digit bits, threads, keys per thread)
    gives the same keys, permutation and cells: the autotuner may pick any.
    The size spans many tiles of the smallest shape and ends in a ragged
    tile of every shape; the clusters leave long runs of equal upper bits."""
    pos, mass = clustered_halos(70_001, 9, n_halo=150)
    o = oracle.build_tree(pos, 16)
    m = tb()
    p = torch.from_numpy(pos).cuda()
    w = torch.from_numpy(mass).cuda()
    variants = m.sort_variants()
    assert len(variants) >= 11
    for cfg in variants:
        t = m.build(p, w, n_crit=16, sort_cfg=cfg)
        torch.cuda.synchronize()
        assert t.sync() == 0, cfg
        assert_structure_equal(t, o)


@pytest.mark.parametrize("n_crit", [1, 2, 8, 32, 100, 1024])
def test_n_crit_values(n_crit):
    pos, mass = clustered_halos(60_000, 8, n_halo=200)
    _check(pos, mass, n_crit)


@pytest.mark.parametrize("n_crit", [8, 16])
def test_exponential_disc(n_crit):
    """Thin disc (height 0.1 of the scale length): flat, anisotropic cells."""
    pos, mass = exponential_disk(1 << 18, 16)
    t, o = _check(pos, mass, n_crit)
    assert t.max_depth >= 8


def test_plummer_deep():
    pos, mass = plummer(1 << 18, 2)
    t, o = _check(pos, mass, 16)
    assert t.max_depth >= 8


def test_clustered():
    pos, mass = clustered_halos(1 << 18, 3, n_halo=500)
    _check(pos, mass, 16)


@pytest.mark.parametrize("mode", [0, 2])
def test_precision_stress_offset_box(mode):
    """[1000,1001)^3 FP32 positions (many identical keys), log-normal masses."""
    pos, mass = precision_stress(1 << 17, 5, n_halo=300)
    t, o = _check(pos, mass, 16, mode=mode)
    assert t.max_depth >= 10


def test_null_mass_means_equal_masses():
    pos, _ = uniform_cube(20_000, 4)
    _check(pos, None, 16)


def test_duplicates_and_identical():
    rng = np.random.default_rng(3)
    pos = rng.integers(0, 3, (30_000, 3)).astype(np.float32)
    _check(pos, None, 4)
    same = np.full((10_000, 3), 0.5, np.float32)
    t, o = _check(same, None, 16)
    assert t.n_cells == 22


@pytest.mark.parametrize("radix_bits", [8, 11])
def test_long_sort_runs(radix_bits):
    """Dense clusters inside single depth-13 cells: the keys share their upper
    bits over runs of hundreds to thousands of particles (runs longer than the
    run step's window go to the block sort), spread over tile boundaries."""
    rng = np.random.default_rng(21)
    parts = [rng.random((40_000, 3)), np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]])]
    cell = 2.0 ** -13
    for j, m in enumerate([300, 900, 1023, 1024, 1025, 1500, 2047, 2049, 5000, 12_000]):
        corner = (np.array([3 + 7 * j, 5 + 11 * j, 2 + 13 * j]) + 0.2) * cell
        parts.append(corner + rng.random((m, 3)) * (cell / 16))
    pos = np.concatenate(parts).astype(np.float32)
    pos = pos[rng.permutation(len(pos))]
    mass = (rng.random(len(pos)) + 0.5).astype(np.float32)
    t, o = _check(pos, mass, 16, radix_bits=radix_bits)
    top = o.skeys >> np.uint64(63 - 40)
    _, counts = np.unique(top, return_counts=True)
    assert counts.max() > 4096


def _runs_at_tile_ends():
    """Lattice points (every one alone in its depth-13 cell) plus, for each of
    several run-step tiles (2048 keys), two more points in the cell of the
    key that sorts last in the tile: a run of three equal upper-bit keys that
    starts at the tile's last position and whose order needs the low bits."""
    g = np.arange(20)
    pts = (np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.5) / 20.0
    pts = np.concatenate([pts, [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])
    for end in (2047, 4095, 6143):
        k, _, _ = oracle.keys(pts.astype(np.float32))
        i = np.argsort(k, kind="stable")[end]
        pts = np.concatenate([pts, pts[i] + np.array([[2e-6, 1e-6, 3e-6], [1e-6, 3e-6, 1e-6]])])
    pos = pts.astype(np.float32)
    sk = np.sort(oracle.keys(pos)[0])
    top = sk >> np.uint64(23)
    starts = np.flatnonzero(np.concatenate([[True], top[1:] != top[:-1]]))
    lens = np.diff(np.concatenate([starts, [len(sk)]]))
    assert set(starts[lens > 1].tolist()) == {2047, 4095, 6143}
    return pos


@pytest.mark.parametrize("order", [0, 1])
def test_sort_runs_from_tile_end(order):
    pos = _runs_at_tile_ends()
    if order:
        pos = pos[::-1].copy()
    _check(pos, None, 4)


def test_lattice_complete_octree():
    pos, mass = lattice(5)
    t, o = _check(pos, mass, 1)
    assert t.n_cells == sum(8 ** d for d in range(6))


def test_fixed_capacity_and_rebuild_in_place():
    m = tb()
    pos, mass = uniform_cube(40_000, 9)
    o = oracle.build_tree(pos, 16)
    t, p, w = gpu_tree(pos, mass, 16, cell_capacity=o.n_cells + 10)
    assert t.sync() == 0
    assert_structure_equal(t, o)
    # rebuild the same tree object with other particles
    pos2, mass2 = plummer(30_000, 10)
    o2 = oracle.build_tree(pos2, 16)
    p2 = torch.from_numpy(pos2).cuda()
    m.build(p2, None, n_crit=16, tree=t)
    assert_structure_equal(t, o2)


def test_graph_captured_build_and_moments():
    """A rebuild with a fixed cell capacity into buffers that are large
    enough never waits on the host, so tb_build + tb_moments can be captured
    in a CUDA graph once and replayed on new positions of the same count:
    each replay matches the oracle in structure and moments."""
    m = tb()
    n = 50_000
    sets = [plummer(n, 31), uniform_cube(n, 32), clustered_halos(n, 33, n_halo=60)]
    trees = [oracle.build_tree(pos, 16) for pos, _ in sets]
    cap = max(o.n_cells for o in trees) + 64
    pos0, mass0 = sets[0]
    p = torch.from_numpy(pos0).cuda()
    w = torch.from_numpy(mass0).cuda()
    t = m.build(p, w, n_crit=16, cell_capacity=cap)
    m.moments(t, p, w)
    torch.cuda.synchronize()
    assert t.sync() == 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m.build(p, w, n_crit=16, cell_capacity=cap, tree=t, stream=s)
            m.moments(t, p, w, stream=s)
    for (pos, mass), o in zip(sets[1:] + sets[:1], trees[1:] + trees[:1]):
        p.copy_(torch.from_numpy(pos))
        w.copy_(torch.from_numpy(mass))
        g.replay()
        torch.cuda.synchronize()
        assert t.sync() == 0
        assert_structure_equal(t, o)
        M, com, quad, aabb = oracle.moments(o, pos, mass)
        em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
        assert bb_ok
        assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


def test_capacity_overflow_reported():
    m = tb()
    pos, mass = uniform_cube(40_000, 9)
    p = torch.from_numpy(pos).cuda()
    t = m.build(p, None, n_crit=16, cell_capacity=100)
    assert m.STATUS[t.sync()] == "TB_EOVERFLOW"
    # the tree stays usable
    m.build(p, None, n_crit=16, tree=t, cell_capacity=0)
    assert t.sync() == 0


def test_nonfinite_rejected():
    m = tb()
    pos, _ = uniform_cube(5000, 9)
    pos[123, 1] = np.nan
    with pytest.raises(m.TbError) as ei:
        m.build(torch.from_numpy(pos).cuda(), None)
    assert ei.value.name == "TB_ENONFINITE"
    pos[123, 1] = np.inf
    with pytest.raises(m.TbError):
        m.build(torch.from_numpy(pos).cuda(), None)


def test_argument_errors():
    m = tb()
    p = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    for kw in (dict(n_crit=0), dict(n_crit=2000), dict(mom_mode=7), dict(radix_bits=5)):
        with pytest.raises(m.TbError) as ei:
            m.build(p, None, **kw)
        assert ei.value.name == "TB_EINVAL"


def test_empty_input():
    m = tb()
    t = m.build(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), None)
    assert t.n_cells == 0
    m.moments(t, torch.zeros((0, 3), dtype=torch.float32, device="cuda"))


def test_plain_mode_structure_and_report():
    """FP32-plain moments: same structure; errors reported, not bounded."""
    pos, mass = plummer(1 << 16, 12)
    o = oracle.build_tree(pos, 16)
    t, p, w = gpu_tree(pos, mass, 16, mode=1)
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
    assert bb_ok and em.max() < 1e-4


def test_reorder_output():
    pos, mass = uniform_cube(30_000, 13)
    o = oracle.build_tree(pos, 16)
    t, p, w = gpu_tree(pos, mass, 16, reorder=True)
    xs = to_np(t.pos_sorted)
    assert np.array_equal(xs[:, :3], pos[o.perm])
    assert np.array_equal(xs[:, 3], mass[o.perm])


def test_moments_with_other_arrays_than_the_build():
    """New masses through other pointers are read afresh (no stale snapshot)."""
    m = tb()
    pos, mass = plummer(30_000, 15)
    o = oracle.build_tree(pos, 16)
    t, p, w = gpu_tree(pos, mass, 16)
    mass2 = (mass * np.float32(3.0)).astype(np.float32)
    w2 = torch.from_numpy(mass2).cuda()
    m.moments(t, p, w2)
    torch.cuda.synchronize()
    M, com, quad, aabb = oracle.moments(o, pos, mass2)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


def test_inputs_not_16_byte_aligned():
    """Positions and masses that start 4 bytes into their buffers (aligned to
    4 bytes only) take the scalar load path of the root and key kernels; the
    tree and moments are the same."""
    m = tb()
    pos, mass = clustered_halos(30_001, 17, n_halo=80)
    n = pos.shape[0]
    o = oracle.build_tree(pos, 16)
    pbuf = torch.zeros(3 * n + 1, dtype=torch.float32, device="cuda")
    wbuf = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    p = pbuf[1:].view(n, 3)
    w = wbuf[1:]
    p.copy_(torch.from_numpy(pos))
    w.copy_(torch.from_numpy(mass))
    assert p.data_ptr() % 16 == 4 and w.data_ptr() % 16 == 4
    t = m.build(p, w, n_crit=16)
    m.moments(t, p, w)
    torch.cuda.synchronize()
    assert t.sync() == 0
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
    assert bb_ok
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


def test_deterministic_repeat():
    pos, mass = clustered_halos(1 << 17, 14, n_halo=300)
    t1, p, w = gpu_tree(pos, mass, 16)
    a = {k: to_np(getattr(t1, k)).copy() for k in ("mass", "com", "com_lo", "quad", "aabb")}
    m = tb()
    for _ in range(3):
        m.build(p, w, n_crit=16, tree=t1)
        m.moments(t1, p, w)
        torch.cuda.synchronize()
        for k, v in a.items():
            assert np.array_equal(to_np(getattr(t1, k)), v), k


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_moments_repeat_on_one_build(mode):
    """Parents are combined by the last of their children to finish, which
    counts arrivals per cell and clears the count as it combines: calling
    tb_moments again on the same build gives the same moments bit for bit.
    Identical particles add a leaf of 3,000 (block-summed) and one of 300
    (past the leaf tile's halo, summed from the queue), whose ancestors are
    combined from those launches."""
    pos, mass = clustered_halos(1 << 16, 21, n_halo=40)
    pos = np.concatenate([pos, np.full((3000, 3), pos[5], np.float32),
                          np.full((300, 3), pos[7], np.float32)])
    mass = np.concatenate([mass, np.full(3300, mass[3], np.float32)])
    if mode == 1:
        # plain FP32: errors are reported, not bounded (as for the other plain-mode test)
        o = oracle.build_tree(pos, 8)
        t, p, w = gpu_tree(pos, mass, 8, mode=1)
        assert_structure_equal(t, o)
        M, com, quad, aabb = oracle.moments(o, pos, mass)
        em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
        assert bb_ok and em.max() < 1e-4
    else:
        t, o = _check(pos, mass, 8, mode=mode)
    m = tb()
    p = torch.from_numpy(pos).cuda()
    w = torch.from_numpy(mass).cuda()
    keys = ("mass", "com", "com_lo", "quad", "aabb") + (("mass64", "com64", "quad64") if mode == 2 else ())
    m.moments(t, p, w)
    torch.cuda.synchronize()
    a = {k: to_np(getattr(t, k)).copy() for k in keys}
    for _ in range(2):
        m.moments(t, p, w)
        torch.cuda.synchronize()
        assert t.sync() == 0
        for k, v in a.items():
            assert np.array_equal(to_np(getattr(t, k)), v), k


@pytest.mark.parametrize("gen,n_crit", [("plummer", 16), ("clustered", 8), ("stress", 16),
                                         ("uniform", 1)])
def test_root_pow2(gen, n_crit):
    """The power-of-two root cube (Sec. 2.2): side forced to the smallest
    power of two at least the extent; keys, cells and moments equal the
    oracle's under the same root.  The scale is then a power of two, so
    every ambiguous quantisation takes the exact FP32 route."""
    pos, mass = {"plummer": lambda: plummer(1 << 16, 41),
                 "clustered": lambda: clustered_halos(1 << 16, 42, n_halo=60),
                 "stress": lambda: precision_stress(1 << 16, 43, n_halo=60),
                 "uniform": lambda: uniform_cube(5000, 44)}[gen]()
    o = oracle.build_tree(pos, n_crit, root_mode="pow2")
    assert o.side == 2.0 ** np.ceil(np.log2(o.side))
    t, p, w = gpu_tree(pos, mass, n_crit, root_pow2=True)
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb)
    assert bb_ok
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD


def test_bounded_wait_times_out():
    m = tb()
    assert m.STATUS[m.selftest_wait(1000)] == "TB_ETIMEOUT"
    # context still usable
    pos, mass = uniform_cube(1000, 1)
    _check(pos, mass, 16)
