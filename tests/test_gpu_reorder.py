"""tb_reorder: per-particle arrays into key order (Sec. 2.3 step 3).

The reordered rows must equal the rows taken in the oracle's stable key order,
bit for bit, for any row width; a build on reordered positions must give the
same tree, with the identity permutation and identical moments."""
import numpy as np
import pytest

import oracle
from synth import clustered_halos, plummer

pytestmark = pytest.mark.gpu

from gpu_util import tb, to_np, torch  # noqa: E402


def _tree(pos, mass=None, n_crit=16):
    m = tb()
    p = torch.from_numpy(pos).cuda()
    w = None if mass is None else torch.from_numpy(mass).cuda()
    t = m.build(p, w, n_crit=n_crit)
    m.moments(t, p, w)
    torch.cuda.synchronize()
    assert t.sync() == 0
    return t, p, w


@pytest.mark.parametrize("n", [1, 1000, 4097, 70_001])
def test_reorder_rows_match_oracle_order(n):
    m = tb()
    pos, mass = plummer(n, 30 + n)
    t, p, w = _tree(pos, mass)
    keys, _, _ = oracle.keys(pos)
    _, operm = oracle.sort(keys)
    rng = np.random.default_rng(n)
    cases = [
        pos,                                                  # 12-byte rows
        mass,                                                 # 4-byte rows
        rng.standard_normal((n, 4)).astype(np.float32),       # 16-byte rows
        rng.integers(-2**31, 2**31, (n, 2), dtype=np.int64).astype(np.int32),   # 8-byte rows
        rng.integers(0, 256, (n, 28), dtype=np.uint8),        # 28-byte rows
        rng.standard_normal((n, 6)),                          # 48-byte rows (FP64)
    ]
    for src in cases:
        out = m.reorder(t, torch.from_numpy(np.ascontiguousarray(src)).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(to_np(out), src[operm]), src.dtype


def test_reorder_arguments_rejected():
    m = tb()
    pos, _ = plummer(5000, 3)
    t, p, _ = _tree(pos)
    with pytest.raises(m.TbError) as ei:
        m.reorder(t, p, p)                                    # overlapping
    assert ei.value.name == "TB_EINVAL"
    odd = torch.zeros((5000, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(m.TbError):
        m.reorder(t, odd)                                     # 3-byte rows
    off = torch.tensor([0, 2500, 5000], dtype=torch.int64, device="cuda")
    bt = m.build_batched(p, None, off)
    with pytest.raises(m.TbError):
        m.reorder(bt, p)                                      # batched tree


def test_build_on_reordered_input_is_the_same_tree():
    """Reorder positions and masses into key order, build again: identical
    keys, cells, links and moments, and the identity permutation."""
    m = tb()
    pos, mass = clustered_halos(200_000, 12, n_halo=300)
    mass = (np.random.default_rng(1).random(len(pos)) + 0.5).astype(np.float32)
    t, p, w = _tree(pos, mass)
    pr = m.reorder(t, p)
    wr = m.reorder(t, w)
    t2, _, _ = _tree(to_np(pr), to_np(wr))
    assert t2.n_cells == t.n_cells
    assert np.array_equal(to_np(t2.perm), np.arange(len(pos), dtype=np.int32))
    for k in ("pkey", "ckey", "level", "parent", "child_first", "child_end", "pfirst", "pend",
              "leaf_cell", "mass", "com", "com_lo", "quad", "aabb"):
        assert np.array_equal(to_np(getattr(t2, k)), to_np(getattr(t, k))), k
