"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

# Tolerances of the moments (floating point; structure is bit-exact):
# |M_gpu / M_ora - 1| <= 2e-6; |COM_gpu - COM_ora|_inf <= 2e-6 s;
# |Q_gpu - Q_ora|_max <= 1e-5 M s^2, with s = L / 2^level the cell side.
TOL_MASS = 2e-6
TOL_COM = 2e-6
TOL_QUAD = 1e-5


def tb():
    import paper_2312_06102_gb300 as m
    m.lib()
    return m


def to_np(t):
    return t.detach().cpu().numpy()


def gpu_tree(pos, mass, n_crit, mode=0, radix_bits=0, cell_capacity=0, moments=True,
             reorder=False, key_order=0, root_pow2=False):
    m = tb()
    p = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).cuda()
    w = None if mass is None else torch.from_numpy(np.ascontiguousarray(mass, np.float32)).cuda()
    t = m.build(p, w, n_crit=n_crit, mom_mode=mode, radix_bits=radix_bits,
                cell_capacity=cell_capacity, reorder=reorder, key_order=key_order,
                root_pow2=root_pow2)
    if cell_capacity:
        st = t.sync()
        assert st == 0, m.STATUS[st]
    if moments:
        m.moments(t, p, w)
    torch.cuda.synchronize()
    assert t.sync() == 0
    return t, p, w


def structure(t):
    return {k: to_np(getattr(t, k)) for k in
            ("pkey", "perm", "ckey", "level", "parent", "child_first", "child_end", "pfirst",
             "pend")}


def assert_structure_equal(t, o):
    g = structure(t)
    assert t.n_cells == o.n_cells
    assert np.array_equal(g["pkey"], o.skeys)
    assert np.array_equal(g["perm"], o.perm)
    for k in ("ckey", "level", "parent", "child_first", "child_end", "pfirst", "pend"):
        assert np.array_equal(g[k], getattr(o, k)), k
    assert t.level_offset == [int(v) for v in o.level_offset]
    assert t.max_depth == o.max_depth
    assert t.n_leaves == int((o.child_first < 0).sum())
    assert np.allclose(t.lo, o.lo, rtol=0, atol=0) and t.side == o.side


def moment_errors(t, o_tree, M, com, quad, aabb, cells=None, mode=0):
    """Max normalised errors (mass rel, COM / s, Q / (M s^2)) and AABB equality."""
    sel = slice(None) if cells is None else cells
    gm = to_np(t.mass)[sel].astype(np.float64)
    gc = to_np(t.com)[sel].astype(np.float64) + to_np(t.com_lo)[sel].astype(np.float64)
    gq = to_np(t.quad)[sel].astype(np.float64)
    if mode == 2:
        gm = to_np(t.mass64)[sel]
        gc = to_np(t.com64)[sel]
        gq = to_np(t.quad64)[sel]
    gb = to_np(t.aabb)[sel]
    lv = to_np(t.level)[sel].astype(np.int64)
    s = t.side / np.exp2(lv)
    em = np.abs(gm / M - 1.0)
    ec = np.abs(gc - com).max(1) / s
    eq = np.abs(gq - quad).max(1) / (M * s * s)
    return em, ec, eq, np.array_equal(gb, aabb)
