"""The synthetic input recipes, checked against their closed forms.

Each workload stands in for one of the paper's datasets, so each generator
is held to the distribution it states: the truncated Plummer enclosed-mass
law, the NFW enclosed-mass law of the haloes, the exact halo counts after
largest-remainder rounding, the uniform background, the batched set sizes,
scale radii and masses, and the offset box and log-normal masses of the
precision-stress set.  Sample fractions are compared within five standard
errors."""
import math

import numpy as np

from synth import batched_plummer, clustered_halos, plummer, precision_stress
from synth import generators as g


def _within(frac, p, n, k=5.0):
    return abs(frac - p) <= k * math.sqrt(p * (1 - p) / n)


def _plummer_cdf(r_over_a, cut=20.0):
    m = lambda x: x ** 3 / (x * x + 1.0) ** 1.5   # noqa: E731
    return m(r_over_a) / m(cut)


def test_plummer_enclosed_mass_law():
    n, a = 400_000, 0.05
    pos, mass = plummer(n, 2, a=a)
    d = pos.astype(np.float64) - 0.5
    r = np.linalg.norm(d, axis=1) / a
    for x in (0.5, 1.0, 2.0, 5.0):
        assert _within((r < x).mean(), _plummer_cdf(x), n), x
    assert r.max() <= 20.0 * (1 + 1e-6)
    # isotropic directions: each axis holds a third of r^2 on average
    share = (d * d).mean(0) / (d * d).sum(1).mean()
    assert np.all(np.abs(share - 1 / 3) < 0.01)
    assert np.all(mass == np.float32(1.0 / n))


def test_nfw_radii_follow_the_enclosed_mass_law():
    n, c = 300_000, 10.0
    x = g._nfw_radii(np.random.Generator(np.random.PCG64(5)), n, c)
    assert x.min() >= 0.0 and x.max() <= c
    mu = lambda y: math.log1p(y) - y / (1.0 + y)   # noqa: E731
    for y in (0.3, 1.0, 3.0, 7.0):
        assert _within((x < y).mean(), mu(y) / mu(c), n), y


def test_halo_counts_sum_exactly_and_round_by_largest_remainder():
    rng = np.random.Generator(np.random.PCG64(3))
    total = 93_952_410          # round(0.7 * 2^27)
    counts = g._halo_counts(rng, 10_000, total, 100.0, 1e6, 1.9)
    assert counts.sum() == total and counts.min() >= 0
    # the same draw before rounding: every count within one of its share
    rng = np.random.Generator(np.random.PCG64(3))
    gexp = 1.0 - 1.9
    u = rng.random(10_000)
    raw = (100.0 ** gexp + u * (1e6 ** gexp - 100.0 ** gexp)) ** (1.0 / gexp)
    scaled = raw * (total / raw.sum())
    assert np.all(np.abs(counts - scaled) < 1.0)
    assert raw.min() >= 100.0 * (1 - 1e-12) and raw.max() <= 1e6 * (1 + 1e-12)


def test_clustered_mix_has_the_uniform_background_and_stays_in_the_box():
    n = 200_000
    pos, mass = clustered_halos(n, 3, n_halo=300, shuffle=False)
    assert pos.dtype == np.float32 and pos.min() >= 0.0 and pos.max() < 1.0
    n_h = int(round(0.7 * n))
    bg = pos[n_h:].astype(np.float64)
    assert bg.shape[0] == n - n_h
    assert np.all(np.abs(bg.mean(0) - 0.5) < 5 * math.sqrt(1 / 12 / bg.shape[0]))
    assert np.all(np.abs(bg.var(0) - 1 / 12) < 0.003)
    # the halo particles are concentrated: far more pairs of close
    # neighbours in key order than a uniform set of the same size would have
    hal = pos[:n_h].astype(np.float64)
    near_h = (np.linalg.norm(np.diff(hal, axis=0), axis=1) < 0.01).mean()
    near_b = (np.linalg.norm(np.diff(bg, axis=0), axis=1) < 0.01).mean()
    assert near_h > 10 * near_b
    same, _ = clustered_halos(n, 3, n_halo=300, shuffle=True)
    assert np.array_equal(np.sort(same, axis=0), np.sort(pos, axis=0))
    assert np.all(mass == np.float32(1.0 / n))


def test_batched_sets_sizes_scales_and_masses():
    b = batched_plummer(n_sets=256, seed=4)
    sizes = np.diff(b.offsets)
    assert b.offsets[0] == 0 and sizes.min() >= 256 and sizes.max() < 65536
    assert b.scale.min() >= 0.01 and b.scale.max() <= 0.2
    # log-uniform sizes: the median is near sqrt(256 * 65536) = 4096
    assert 2500 < np.median(sizes) < 6500
    for s in (0, 17, 255):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        r = np.linalg.norm(b.pos[lo:hi].astype(np.float64) - 0.5, axis=1)
        assert r.max() <= 20.0 * b.scale[s] * (1 + 1e-6)
        assert np.all(b.mass[lo:hi] == np.float32(1.0 / (hi - lo)))


def test_precision_stress_box_and_lognormal_masses():
    n = 200_000
    pos, mass = precision_stress(n, 5, n_halo=300)
    assert pos.min() >= 1000.0 and pos.max() <= 1001.0
    z = np.log(mass.astype(np.float64) * n) / 2.0      # Z ~ N(0, 1)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
