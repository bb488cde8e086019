"""Failure paths of the build, made without faulting the GPU.

- A radix-pass look-back wait that runs out: the wait limit is lowered so
  that a look-back which finds a predecessor tile not yet published gives up
  at once; the build reports TB_ETIMEOUT, every access stays in bounds, and
  the next build of the same tree with the default limit is exact.
- A device allocation that fails: the library's TB_FAULT_ALLOC=k hook makes
  its k-th cudaMalloc fail in a child process; the build reports TB_ENOMEM
  and releasing the half-made tree succeeds.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from synth import uniform_cube

pytestmark = pytest.mark.gpu

from gpu_util import assert_structure_equal, tb, torch  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lookback_wait_runs_out_then_next_build_is_exact():
    m = tb()
    # 2^21 particles: 512 tiles of 4096 keys in each of the five passes, with
    # hundreds of tiles in flight at once
    pos, mass = uniform_cube(1 << 21, 23)
    p = torch.from_numpy(pos).cuda()
    w = torch.from_numpy(mass).cuda()
    t = m.Tree()
    cfg = (8, 512, 8)
    assert m.set_wait_limit(0) == 0
    m.set_wait_limit(1)
    try:
        with pytest.raises(m.TbError) as ei:
            m.build(p, w, n_crit=16, tree=t, sort_cfg=cfg)
            torch.cuda.synchronize()
            st = t.sync()
            if st != 0:
                raise m.TbError(st, "status")
        assert ei.value.name == "TB_ETIMEOUT"
    finally:
        m.set_wait_limit(0)
    assert m.set_wait_limit(-1) == 1          # TB_EINVAL
    m.build(p, w, n_crit=16, tree=t, sort_cfg=cfg)
    torch.cuda.synchronize()
    assert t.sync() == 0
    assert_structure_equal(t, oracle.build_tree(pos, 16))


_CHILD = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
import paper_2312_06102_gb300 as tb
p = torch.rand(200000, 3, device="cuda")
t = tb.Tree()
try:
    tb.build(p, None, n_crit=16, tree=t, sort_cfg=(8, 512, 8))
    print("RESULT TB_OK")
except tb.TbError as e:
    print("RESULT", e.name)
t.free()
torch.cuda.synchronize()
print("FREED")
"""


@pytest.mark.parametrize("k", [1, 4, 9])
def test_allocation_failure_reports_enomem(k):
    env = dict(os.environ, TB_FAULT_ALLOC=str(k))
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "RESULT TB_ENOMEM" in r.stdout, r.stdout
    assert "FREED" in r.stdout
