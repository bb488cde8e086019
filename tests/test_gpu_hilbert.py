"""Peano-Hilbert keys through the whole GPU path (key_order = KEYS_HILBERT):
keys, stable sort, cells, links and moments against the oracle's build in
the same order; the cells as sets equal those of the Morton build."""
import numpy as np
import pytest

import oracle
from synth import clustered_halos, exponential_disk, plummer, precision_stress, uniform_cube

pytestmark = pytest.mark.gpu

from gpu_util import (TOL_COM, TOL_MASS, TOL_QUAD, assert_structure_equal, gpu_tree,  # noqa: E402
                      moment_errors, tb, to_np, torch)


def _check(pos, mass, n_crit, mode=0, radix_bits=0):
    o = oracle.build_tree(pos, n_crit, "hilbert")
    t, p, w = gpu_tree(pos, mass, n_crit, mode=mode, radix_bits=radix_bits, key_order=1)
    assert_structure_equal(t, o)
    M, com, quad, aabb = oracle.moments(o, pos, mass)
    em, ec, eq, bb_ok = moment_errors(t, o, M, com, quad, aabb, mode=mode)
    assert bb_ok
    assert em.max() <= TOL_MASS and ec.max() <= TOL_COM and eq.max() <= TOL_QUAD
    return t, o


@pytest.mark.parametrize("n", [1, 2, 17, 4097, 50_001])
def test_ragged_sizes(n):
    pos, mass = uniform_cube(n, 2000 + n)
    _check(pos, mass, 16)


@pytest.mark.parametrize("radix_bits", [8, 11])
def test_plummer(radix_bits):
    pos, mass = plummer(1 << 18, 21)
    _check(pos, mass, 16, radix_bits=radix_bits)


@pytest.mark.parametrize("n_crit", [1, 8, 100])
def test_clustered(n_crit):
    pos, mass = clustered_halos(1 << 17, 22, n_halo=200)
    _check(pos, mass, n_crit)


def test_disc_and_stress():
    pos, mass = exponential_disk(1 << 17, 23)
    _check(pos, mass, 16)
    pos, mass = precision_stress(1 << 16, 24, n_halo=100)
    _check(pos, mass, 16, mode=2)


def test_duplicates():
    rng = np.random.default_rng(25)
    pos = rng.integers(0, 3, (20_000, 3)).astype(np.float32)
    _check(pos, None, 4)


def test_same_cells_as_morton():
    pos, mass = clustered_halos(1 << 16, 26, n_halo=100)
    th, *_ = gpu_tree(pos, mass, 16, key_order=1)
    tm, *_ = gpu_tree(pos, mass, 16, key_order=0)
    assert th.n_cells == tm.n_cells and th.level_offset == tm.level_offset

    def cells(t):
        perm = to_np(t.perm)
        lv, pf, pe = to_np(t.level), to_np(t.pfirst), to_np(t.pend)
        return {(int(lv[c]), frozenset(perm[pf[c]:pe[c]].tolist())) for c in range(t.n_cells)}

    assert cells(th) == cells(tm)
    assert np.allclose(np.sort(to_np(th.mass)), np.sort(to_np(tm.mass)), rtol=1e-6, atol=0)


def test_batched_takes_morton_keys_only():
    m = tb()
    pos, _ = uniform_cube(1000, 27)
    p = torch.from_numpy(pos).cuda()
    off = torch.tensor([0, 400, 1000], dtype=torch.int64, device="cuda")
    with pytest.raises(m.TbError) as ei:
        m.build_batched(p, None, off, key_order=1)
    assert ei.value.name == "TB_EINVAL"
