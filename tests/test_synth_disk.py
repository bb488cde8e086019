"""The exponential-disc input recipe (the paper's second dataset family):
checks of the drawn distribution against its closed forms."""
import math

import numpy as np

from synth import WORKLOADS, exponential_disk, workload


def test_disc_radial_and_vertical_laws():
    rd, z0 = 0.05, 0.005
    pos, mass = exponential_disk(400_000, 6, rd=rd, z0=z0)
    R = np.hypot(pos[:, 0].astype(np.float64) - 0.5, pos[:, 1].astype(np.float64) - 0.5) / rd
    z = (pos[:, 2].astype(np.float64) - 0.5) / z0
    # R / rd ~ Gamma(2, 1) truncated at 10: mean = (2 - e^-10 (10^2 + 2*10 + 2)) / (1 - 11 e^-10)
    t = 10.0
    mean = (2.0 - math.exp(-t) * (t * t + 2 * t + 2)) / (1.0 - (1 + t) * math.exp(-t))
    assert abs(R.mean() - mean) < 0.01
    # enclosed mass fraction at R = rd: 1 - 2/e (untruncated; the cut moves it by < 1e-3)
    assert abs((R < 1.0).mean() - (1.0 - 2.0 / math.e)) < 0.005
    # sech^2 heights: median |z| = z0 atanh(1/2), symmetric, |z| <= 10 z0
    assert abs(np.median(np.abs(z)) - math.atanh(0.5)) < 0.01
    assert abs(z.mean()) < 0.02 and np.abs(z).max() <= 10.0 + 1e-3
    assert mass.dtype == np.float32 and np.all(mass == np.float32(1.0 / 400_000))


def test_disc_is_seeded_and_registered():
    a, _ = exponential_disk(1000, 9)
    b, _ = exponential_disk(1000, 9)
    c, _ = exponential_disk(1000, 10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    spec = WORKLOADS["disk_2p24"]
    assert spec["n"] == 1 << 24 and spec["kind"] == "disk"
    p, _ = workload("disk", 2000, 6)
    assert np.array_equal(p, exponential_disk(2000, 6)[0])
