"""The allocation-free entry point (tb_keys_sorted_noalloc) against tb_build.

It serves callers of this library that cannot allocate device memory at
call time (for instance while another component's caching allocator holds
the device's free memory, or inside a loop that must not pay cudaMalloc's
implicit synchronisation).  Its scratch is a fixed device array shared by
all calls, so this file checks two calls in a row, of different sizes,
against the keys and permutation that tb_build produces for the same
particles.  Keys and permutations are integers: the comparison is exact.
The file is named to be collected last.
"""
import numpy as np
import pytest

from synth import clustered_halos, plummer

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _reference(tb, pos):
    p = torch.from_numpy(pos).cuda()
    t = tb.build(p, None, n_crit=16)
    torch.cuda.synchronize()
    return p, t.pkey.cpu().numpy().copy(), t.perm.cpu().numpy().copy(), t


def test_noalloc_matches_tb_build_on_two_calls_in_a_row():
    import paper_2312_06102_gb300 as tb
    tb.lib()
    cases = [plummer(300_000, 21)[0], clustered_halos(tb.NOALLOC_MAX_N, 22, n_halo=400)[0]]
    for pos in cases:
        p, want_k, want_p, t = _reference(tb, pos)
        n = pos.shape[0]
        k = torch.empty(n, dtype=torch.uint64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        st, root = tb.keys_sorted_noalloc(p, k, perm)
        assert st == 0, tb.STATUS[st]
        assert np.array_equal(k.cpu().numpy(), want_k)
        assert np.array_equal(perm.cpu().numpy(), want_p)
        assert root[:3] == t.lo and root[3] == t.side
        t.free()


def test_noalloc_refuses_sizes_above_its_maximum():
    import paper_2312_06102_gb300 as tb
    n = tb.NOALLOC_MAX_N + 1
    p = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    k = torch.empty(n, dtype=torch.uint64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    st, _ = tb.keys_sorted_noalloc(p, k, perm)
    assert tb.STATUS[st] == "TB_EINVAL"
