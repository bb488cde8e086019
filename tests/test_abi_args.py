"""Argument errors of the C ABI, checked on a machine without a GPU.

Every entry point validates its arguments before it allocates, synchronises
or launches anything, and returns TB_EINVAL at once.  These calls pass NULL,
misaligned or out-of-range values (the "device pointers" are small integers
that are never dereferenced), so the whole file is skipped where CUDA is
available: there a missing check could reach a launch on those pointers.
"""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host-only argument checks; fake device pointers")

EINVAL = 1


@pytest.fixture(scope="module")
def tb():
    from paper_2312_06102_gb300 import _lib, compile_lib
    compile_lib.build()
    return _lib


def _params(tb, **kw):
    p = tb.lib().tb_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _build(tb, pos, mass, n, p):
    out = C.POINTER(tb.TreeC)()
    code = tb.lib().tb_build(pos, mass, n, None if p is None else C.byref(p), None, C.byref(out))
    assert not out, "no tree may be created for a rejected call"
    return code


def test_defaults_are_valid_values(tb):
    p = _params(tb)
    assert (p.n_crit, p.mom_mode, p.cell_capacity, p.reorder, p.radix_bits, p.key_order,
            p.root_pow2) == (16, 0, 0, 0, 0, 0, 0)


def test_build_rejects_null_tree_and_params(tb):
    p = _params(tb)
    assert tb.lib().tb_build(16, None, 10, C.byref(p), None, None) == EINVAL
    assert _build(tb, 16, None, 10, None) == EINVAL


@pytest.mark.parametrize("n", [-1, 1 << 31, 1 << 40])
def test_build_rejects_particle_counts(tb, n):
    assert _build(tb, 16, None, n, _params(tb)) == EINVAL


@pytest.mark.parametrize("field,value", [
    ("n_crit", 0), ("n_crit", -3), ("n_crit", 1025),
    ("mom_mode", -1), ("mom_mode", 3),
    ("cell_capacity", -1), ("cell_capacity", 1 << 31),   # cell indices are int32
    ("radix_bits", 7), ("radix_bits", 12),
    ("key_order", 2), ("key_order", -1),
    ("root_pow2", 2), ("root_pow2", -1),
    ("sort_threads", 300), ("sort_items", 5),
])
def test_build_rejects_params(tb, field, value):
    assert _build(tb, 16, None, 10, _params(tb, **{field: value})) == EINVAL


def test_build_rejects_pointers(tb):
    p = _params(tb)
    assert _build(tb, None, None, 10, p) == EINVAL        # positions needed for n > 0
    assert _build(tb, 18, None, 10, p) == EINVAL          # positions not 4-byte aligned
    assert _build(tb, 16, 22, 10, p) == EINVAL            # masses not 4-byte aligned


def test_batched_rejects(tb):
    L = tb.lib()

    def call(pos, off, S, n_total, **kw):
        out = C.POINTER(tb.TreeC)()
        p = _params(tb, **kw)
        code = L.tb_build_batched(pos, None, off, S, n_total, C.byref(p), None, C.byref(out))
        assert not out
        return code

    assert call(16, 64, 4, 100, key_order=1) == EINVAL   # Morton keys only
    assert call(16, None, 4, 100) == EINVAL              # offsets needed for sets
    assert call(16, 64, -1, 100) == EINVAL
    assert call(16, 64, 4, -5) == EINVAL
    assert call(16, 64, 4, 1 << 31) == EINVAL
    assert call(None, 64, 4, 100) == EINVAL
    assert call(18, 64, 4, 100) == EINVAL
    assert call(16, 64, 4, 100, n_crit=0) == EINVAL


def test_moments_walk_reorder_status_reject_null_tree(tb):
    L = tb.lib()
    assert L.tb_moments(None, 16, None, None) == EINVAL
    assert L.tb_walk(None, 0.5, 0.0, 32, 1, 16, None) == EINVAL
    assert L.tb_reorder(None, 16, 4096, 16, None) == EINVAL
    assert L.tb_tree_status(None, None) == EINVAL
    L.tb_free(None)   # NULL-safe


@pytest.mark.parametrize("theta,eps,n_group", [
    (-0.1, 0.0, 32), (float("nan"), 0.0, 32), (float("inf"), 0.0, 32),
    (0.5, -1.0, 32), (0.5, float("nan"), 32),
    (0.5, 0.0, 0), (0.5, 0.0, (1 << 20) + 1),
])
def test_walk_rejects_parameters(tb, theta, eps, n_group):
    t = tb.TreeC()          # host struct only: the checks read n_sets and stop
    t.n_particles = 100
    assert tb.lib().tb_walk(C.byref(t), theta, eps, n_group, 1, 16, None) == EINVAL


def test_reorder_rejects(tb):
    L = tb.lib()
    t = tb.TreeC()
    t.n_particles = 100
    t.perm = 0x10           # never dereferenced: every call below stops at a check
    for row in (0, -4, 6, (1 << 20) + 4):
        assert L.tb_reorder(C.byref(t), 1 << 20, 1 << 24, row, None) == EINVAL
    assert L.tb_reorder(C.byref(t), None, 1 << 24, 16, None) == EINVAL
    assert L.tb_reorder(C.byref(t), 1 << 20, None, 16, None) == EINVAL
    assert L.tb_reorder(C.byref(t), (1 << 20) + 2, 1 << 24, 16, None) == EINVAL   # misaligned
    # the destination starts inside the source's 1600 bytes
    assert L.tb_reorder(C.byref(t), 1 << 20, (1 << 20) + 800, 16, None) == EINVAL
    t.n_sets = 3            # a batched tree
    assert L.tb_reorder(C.byref(t), 1 << 20, 1 << 24, 16, None) == EINVAL
    t.n_sets = 0            # valid arguments, but no completed build behind the tree
    assert L.tb_reorder(C.byref(t), 1 << 20, 1 << 24, 16, None) == EINVAL
    t.n_particles = 0
    assert L.tb_reorder(C.byref(t), None, None, 16, None) == 0   # empty tree: nothing to do


def test_keys_noalloc_rejects(tb):
    L = tb.lib()
    root = (C.c_double * 4)()
    n_max = tb.NOALLOC_MAX_N
    assert L.tb_keys_sorted_noalloc(16, -1, 64, 32, root, None) == EINVAL
    assert L.tb_keys_sorted_noalloc(16, n_max + 1, 64, 32, root, None) == EINVAL
    assert L.tb_keys_sorted_noalloc(None, 10, 64, 32, root, None) == EINVAL
    assert L.tb_keys_sorted_noalloc(16, 10, None, 32, root, None) == EINVAL
    assert L.tb_keys_sorted_noalloc(16, 10, 64, None, root, None) == EINVAL
    assert L.tb_keys_sorted_noalloc(18, 10, 64, 32, root, None) == EINVAL   # positions
    assert L.tb_keys_sorted_noalloc(16, 10, 68, 32, root, None) == EINVAL   # keys need 8 B
    assert L.tb_keys_sorted_noalloc(16, 10, 64, 34, root, None) == EINVAL   # permutation


def test_wait_limit_setter(tb):
    assert tb.lib().tb_set_wait_limit(-1) == EINVAL
    assert tb.lib().tb_set_wait_limit(5) == 0
    assert tb.lib().tb_set_wait_limit(0) == 0      # back to the default


@pytest.mark.parametrize("threads", [-1, 1, 256, 768, 2048])
def test_batched_rejects_block_sizes(tb, threads):
    p = _params(tb, batch_threads=threads)
    out = C.POINTER(tb.TreeC)()
    code = tb.lib().tb_build_batched(16, None, 16, 1, 10, C.byref(p), None, C.byref(out))
    assert code == EINVAL and not out
