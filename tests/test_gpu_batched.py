"""tb_build_batched: every set is its own tree, identical to the oracle's tree
of that set alone (structure bit-exact, moments within tolerance); indices
in the batched output are global."""
import numpy as np
import pytest

import oracle
from synth import batched_plummer, jitter_offsets, plummer, uniform_cube

pytestmark = pytest.mark.gpu

from gpu_util import TOL_COM, TOL_MASS, TOL_QUAD, tb, to_np, torch  # noqa: E402


def _run(pos, mass, offsets, n_crit=16, cap=0, mode=0, tree=None, threads=512, root_pow2=False):
    m = tb()
    p = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).cuda()
    w = None if mass is None else torch.from_numpy(np.ascontiguousarray(mass, np.float32)).cuda()
    off = torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    t = m.build_batched(p, w, off, n_crit=n_crit, cell_capacity=cap, mom_mode=mode, tree=tree,
                        batch_threads=threads, root_pow2=root_pow2)
    torch.cuda.synchronize()
    assert t.sync() == 0
    return t, p, w, off


def _check_sets(t, pos, mass, offsets, n_crit, sets=None, mode=0, root_mode="tight"):
    offsets = np.asarray(offsets, np.int64)
    S = len(offsets) - 1
    g = {k: to_np(getattr(t, k)) for k in ("pkey", "perm", "ckey", "level", "parent",
                                          "child_first", "child_end", "pfirst", "pend",
                                          "mass", "com", "com_lo", "quad", "aabb")}
    coff = to_np(t.set_cell_offset)
    root = to_np(t.set_root)
    assert coff[0] == 0 and coff[-1] == t.n_cells
    for s in (range(S) if sets is None else sets):
        a, b = int(offsets[s]), int(offsets[s + 1])
        c0, c1 = int(coff[s]), int(coff[s + 1])
        if b == a:
            assert c1 == c0
            continue
        sp = pos[a:b]
        sm = None if mass is None else mass[a:b]
        o = oracle.build_tree(sp, n_crit, root_mode=root_mode)
        assert c1 - c0 == o.n_cells, (s, c1 - c0, o.n_cells)
        assert np.array_equal(g["pkey"][a:b], o.skeys), s
        assert np.array_equal(g["perm"][a:b] - a, o.perm), s
        sl = slice(c0, c1)
        assert np.array_equal(g["ckey"][sl], o.ckey)
        assert np.array_equal(g["level"][sl], o.level)
        for k in ("pfirst", "pend"):
            assert np.array_equal(g[k][sl] - a, getattr(o, k)), (s, k)
        for k in ("parent", "child_first", "child_end"):
            want = getattr(o, k).astype(np.int64)
            want = np.where(want >= 0, want + c0, -1)
            assert np.array_equal(g[k][sl].astype(np.int64), want), (s, k)
        assert np.array_equal(root[s, :3], o.lo) and root[s, 3] == o.side
        M, com, quad, aabb = oracle.moments(o, sp, sm)
        side = o.side / np.exp2(o.level.astype(np.int64))
        gc = g["com"][sl].astype(np.float64) + g["com_lo"][sl].astype(np.float64)
        assert np.abs(g["mass"][sl] / M - 1).max() <= TOL_MASS
        assert (np.abs(gc - com).max(1) / side).max() <= TOL_COM
        assert (np.abs(g["quad"][sl] - quad).max(1) / (M * side * side)).max() <= TOL_QUAD
        assert np.array_equal(g["aabb"][sl], aabb)


def _sets(sizes, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for i, n in enumerate(sizes):
        kind = i % 3
        if kind == 0:
            parts.append(uniform_cube(n, seed + i)[0] if n else np.zeros((0, 3), np.float32))
        elif kind == 1:
            parts.append(plummer(n, seed + i, a=0.02 + 0.01 * (i % 5))[0] if n else np.zeros((0, 3), np.float32))
        else:
            parts.append(rng.integers(0, 4, (n, 3)).astype(np.float32))   # duplicates
    pos = np.concatenate(parts) if parts else np.zeros((0, 3), np.float32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    mass = (rng.random(pos.shape[0]) + 0.5).astype(np.float32)
    return pos, mass, offsets


@pytest.mark.parametrize("threads", [512, 1024])
@pytest.mark.parametrize("n_crit", [1, 8, 16, 100])
def test_batched_mixed_sizes(n_crit, threads):
    """Both block sizes per set: tiles of 512 or 1024 particles, sort tiles of
    2048 or 4096 keys; sizes around every tile boundary."""
    sizes = [0, 1, 2, 16, 17, 100, 511, 512, 513, 1023, 1024, 1025, 2047, 2048, 2049, 4095,
             4096, 4097, 9000, 0, 3, 20_000, 65_536, 5]
    pos, mass, offsets = _sets(sizes, 10 + n_crit)
    t, *_ = _run(pos, mass, offsets, n_crit=n_crit, threads=threads)
    _check_sets(t, pos, mass, offsets, n_crit)


@pytest.mark.parametrize("threads", [512, 1024])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batched_one_launch_equals_separate_launches(threads, mode):
    """The cooperative one-launch build gives the same arrays as the separate
    launches, for both block sizes and every moment mode."""
    m = tb()
    sizes = [700, 3000, 50_000, 1, 0, 9999, 4096, 65_536]
    pos, mass, offsets = _sets(sizes, 9)
    a, p, w, off = _run(pos, mass, offsets, mode=mode, threads=threads)
    cap = a.n_cells + 16
    b = m.build_batched(p, w, off, cell_capacity=cap, mom_mode=mode, batch_threads=threads,
                        one_launch=True)
    torch.cuda.synchronize()
    assert b.sync() == 0 and b.n_cells == a.n_cells
    keys = ["pkey", "perm", "ckey", "level", "parent", "child_first", "child_end", "pfirst",
            "pend", "mass", "com", "com_lo", "quad", "aabb"] + (["mass64", "com64", "quad64"]
                                                                if mode == 2 else [])
    for k in keys:
        assert np.array_equal(to_np(getattr(a, k)), to_np(getattr(b, k))), k
    if mode != 1:   # plain FP32 is reported, not held to the tolerances
        _check_sets(b, pos, mass, offsets, 16, mode=mode)


def test_batched_block_sizes_agree():
    """512- and 1024-thread builds of the same sets give identical arrays."""
    sizes = [700, 3000, 50_000, 1, 9999]
    pos, mass, offsets = _sets(sizes, 5)
    a, *_ = _run(pos, mass, offsets, threads=512)
    b, *_ = _run(pos, mass, offsets, threads=1024)
    for k in ("pkey", "perm", "ckey", "level", "parent", "child_first", "child_end", "pfirst",
              "pend", "mass", "com", "com_lo", "quad", "aabb"):
        assert np.array_equal(to_np(getattr(a, k)), to_np(getattr(b, k))), k


def test_batched_null_mass_and_fp64_mode():
    sizes = [300, 5000, 1, 12_345]
    pos, _, offsets = _sets(sizes, 77)
    t, *_ = _run(pos, None, offsets, mode=2)
    _check_sets(t, pos, None, offsets, 16)


def test_batched_plummer_sets_sampled():
    """The batched workload's recipe with 512 sets; 40 sets checked in full."""
    b = batched_plummer(n_sets=512, seed=4)
    t, *_ = _run(b.pos, b.mass, b.offsets)
    rng = np.random.default_rng(1)
    _check_sets(t, b.pos, b.mass, b.offsets, 16, sets=sorted(rng.choice(512, 40, replace=False)))


@pytest.mark.parametrize("one_launch", [False, True])
def test_batched_graph_replay_with_jitter(one_launch):
    """Capacity mode needs no host sync; captured in a CUDA graph and replayed
    on jittered positions (steps 1 and 3), each matching the oracle -- as
    separate launches, or as one cooperative launch."""
    m = tb()
    b = batched_plummer(n_sets=64, seed=4)
    t, p, w, off = _run(b.pos, b.mass, b.offsets)
    cap = int(t.n_cells * 1.2) + 64
    m.build_batched(p, w, off, cell_capacity=cap, tree=t, one_launch=one_launch)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        n0 = m.kernel_launches()
        with torch.cuda.graph(g, stream=s):
            m.build_batched(p, w, off, cell_capacity=cap, tree=t, stream=s, one_launch=one_launch)
        if one_launch:
            assert m.kernel_launches() - n0 == 1
    for step in (1, 3):
        jit = jitter_offsets(4, step, b.offsets, b.scale)
        pj = (b.pos + jit).astype(np.float32)
        p.copy_(torch.from_numpy(pj))
        g.replay()
        torch.cuda.synchronize()
        assert t.sync() == 0
        _check_sets(t, pj, b.mass, b.offsets, 16, sets=[0, 1, 17, 40, 63])


def test_batched_root_pow2():
    """Every set's root cube with its side forced to a power of two (Sec. 2.2)
    equals the oracle's tree of that set under the same root."""
    pos, mass, offsets = _sets([1, 7, 300, 4096, 0, 9000, 33], 61)
    t, p, w, off = _run(pos, mass, offsets, root_pow2=True)
    _check_sets(t, pos, mass, offsets, 16, root_mode="pow2")


def test_batched_invalid_offsets_rejected():
    m = tb()
    pos, mass, offsets = _sets([10, 20, 30], 5)
    bad = offsets.copy()
    bad[2] = 5          # not non-decreasing
    p = torch.from_numpy(pos).cuda()
    with pytest.raises(m.TbError) as ei:
        m.build_batched(p, None, torch.from_numpy(bad).cuda())
    assert ei.value.name == "TB_EINVAL"


def test_batched_empty():
    m = tb()
    t = m.build_batched(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), None,
                        torch.zeros(4, dtype=torch.int64, device="cuda"))
    assert t.n_cells == 0
