"""Host-side pieces of bench.py that need no GPU: the on-device jitter of the
batched workload follows the same counter-based definition as the seeded
generator (checked here with torch on the CPU)."""
import numpy as np
import pytest

import bench
from synth import batched_plummer, jitter_offsets

torch = pytest.importorskip("torch")


def test_torch_jitter_matches_generator():
    b = batched_plummer(n_sets=12, seed=4, nmin=50, nmax=400)
    j = bench.Jitter(torch, b, 4, dev="cpu")
    out = torch.empty((int(b.offsets[-1]), 3), dtype=torch.float32)
    for step in (0, 1, 99):
        j.fill(step, out)
        want = (b.pos + jitter_offsets(4, step, b.offsets, b.scale)).astype(np.float32)
        assert np.array_equal(out.numpy(), want), step


def _rate_worker(rank, world, port, q):
    import os
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.whole_job_rate(1000, 4, world, 10.0 * (rank + 1), device="cpu")
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_gloo():
    """world_size 2 on the CPU: both ranks report the slower rank's time and
    the rate of all ranks' particles over it."""
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rate_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 20.0
        assert value == pytest.approx(1000 * 4 * 2 / 0.020 / 1e6)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    """Under torchrun only rank 0 runs the oracle arm; the others exit 0 at once."""
    import sys
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    a = bench.args_()
    assert bench.run_reference(a) == 0
    assert capsys.readouterr().out == ""


def test_clock_samples_are_kept_inside_the_timed_region(tmp_path):
    """The nvidia-smi sampler's rows are filtered to the timed window by their
    timestamps, throttle reasons are collected, and the median SM clock kept."""
    import datetime
    import time as _time

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    now = _time.time()

    def row(dt, sm, reason=""):
        ts = datetime.datetime.fromtimestamp(now + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        flags = ["Active" if r == reason else "Not Active"
                 for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
        return ", ".join([ts, "0", str(sm), "2070", "900.0", "0x0"] + flags) + "\n"

    path = tmp_path / "clocks.csv"
    path.write_text(row(-1.0, 1000, "hw_slowdown") + row(0.05, 2070) + row(0.10, 2050, "sw_power_cap")
                    + row(2.0, 500))
    c = bench.Clocks(0)
    c.proc, c.path, c.f = _Done(), str(path), open(tmp_path / "unused", "w")
    out = c.stop((now, now + 0.15))
    assert out["samples"] == 2
    assert out["reasons"] == ["sw_power_cap"]
    assert out["sm_mhz"] == 2060.0 and out["sm_max_mhz"] == 2070.0


def _library_marks(steps):
    """Stage intervals as tb_stage_times returns them: events are recorded at
    "start" and at the end of every stage of each step, and each interval is
    named after the event that closes it, so the first "start" names none."""
    events = []
    for i, keys_ms in enumerate(steps):
        events += [("start", 0.01), ("root", 0.3), ("keys", keys_ms), ("sort_pass", 1.2),
                   ("sort_pass", 1.2), ("levels", 0.5), ("emit", 0.4), ("moments", 1.5)]
    return events[1:]


def test_per_step_times_from_stage_marks():
    # the gap before each later step's "start" belongs to that step
    r = bench.per_step_ms(_library_marks([1.0, 2.0, 1.0]), 3)
    first = 0.3 + 1.0 + 2.4 + 0.9 + 1.5             # no "start" interval
    assert r["min"] == round(first, 4)
    assert r["median"] == round(0.01 + first, 4)
    assert r["max"] == round(0.01 + first + 1.0, 4)
    assert bench.per_step_ms(_library_marks([1.0] * 20), 20)["median"] > 0
    assert bench.per_step_ms(_library_marks([1.0, 1.0]), 3) is None   # two steps, not three
    assert bench.per_step_ms([], 1) is None
