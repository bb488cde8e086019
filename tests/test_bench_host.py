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


def test_metric_names_the_baseline_metric():
    import json, os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "BASELINE.json")) as f:
        assert json.load(f)["metric"] == bench.METRIC
