"""The allocation-free entry point (tb_keys_sorted_noalloc).

It serves callers of this library that cannot allocate device memory at
call time (for instance while another component's caching allocator holds
the device's free memory, or inside a loop that must not pay cudaMalloc's
implicit synchronisation).  Its scratch is a fixed device array shared by
all calls and keeping the last call's contents, so this file makes three
calls in a row -- a mid-size one, one at the maximum size, then a smaller one
that meets everything the larger call left behind -- and checks each against
the keys and permutation that tb_build produces for the same particles and
against the oracle's keys and stable sort.  Keys and permutations are
integers: the comparisons are exact.  It also checks that, once start-up
calls have loaded the scratch array and the kernels, calls change the
device's free memory by nothing.  The
file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
from synth import clustered_halos, plummer, uniform_cube

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tb():
    import paper_2312_06102_gb300 as tb
    tb.lib()
    return tb


def _reference(tb, pos):
    p = torch.from_numpy(pos).cuda()
    t = tb.build(p, None, n_crit=16)
    torch.cuda.synchronize()
    return p, t.pkey.cpu().numpy().copy(), t.perm.cpu().numpy().copy(), t


def test_noalloc_matches_tb_build_and_oracle_on_calls_in_a_row():
    tb = _tb()
    cases = [plummer(300_000, 21)[0], clustered_halos(tb.NOALLOC_MAX_N, 22, n_halo=400)[0],
             uniform_cube(50_001, 24)[0]]
    for pos in cases:
        p, want_k, want_p, t = _reference(tb, pos)
        n = pos.shape[0]
        k = torch.empty(n, dtype=torch.uint64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        st, root = tb.keys_sorted_noalloc(p, k, perm)
        assert st == 0, tb.STATUS[st]
        got_k, got_p = k.cpu().numpy(), perm.cpu().numpy()
        # the existing entry point
        assert np.array_equal(got_k, want_k)
        assert np.array_equal(got_p, want_p)
        assert root[:3] == t.lo and root[3] == t.side
        t.free()
        # the oracle: FP64 keys of the tight root cube, then a stable sort
        ok, lo, side = oracle.keys(pos)
        sk, sp = oracle.sort(ok)
        assert np.array_equal(got_k, sk)
        assert np.array_equal(got_p, sp)
        assert root[:3] == list(lo) and root[3] == side


def test_noalloc_allocates_nothing_after_the_first_call():
    tb = _tb()
    pos = uniform_cube(200_000, 25)[0]
    p = torch.from_numpy(pos).cuda()
    k = torch.empty(pos.shape[0], dtype=torch.uint64, device="cuda")
    perm = torch.empty(pos.shape[0], dtype=torch.int32, device="cuda")
    # the start-up calls: n = 0 reserves the scratch array, n >= 2 loads the
    # kernels (CUDA loads modules lazily)
    empty = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    st, _ = tb.keys_sorted_noalloc(empty, k[:0], perm[:0])
    assert st == 0, tb.STATUS[st]
    st, _ = tb.keys_sorted_noalloc(p[:2], k[:2], perm[:2])
    assert st == 0, tb.STATUS[st]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        st, _ = tb.keys_sorted_noalloc(p, k, perm)
        assert st == 0, tb.STATUS[st]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_sizes_above_its_maximum():
    tb = _tb()
    n = tb.NOALLOC_MAX_N + 1
    p = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    k = torch.empty(n, dtype=torch.uint64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    st, _ = tb.keys_sorted_noalloc(p, k, perm)
    assert tb.STATUS[st] == "TB_EINVAL"
