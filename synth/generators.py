"""Seeded synthetic particle sets standing in for the paper's N-body inputs.

The paper times its build on Plummer spheres and exponential discs drawn
with NEMO (Sec. 3).  Those files are not available here, so the
workloads below are drawn from their defining distributions:

* ``uniform_cube``   -- i.i.d. uniform positions in [0,1)^3.
* ``plummer``        -- Plummer (1911) sphere, radius from the inverse of
  the cumulative mass M(<r)/M = r^3 / (r^2 + a^2)^(3/2), truncated.
* ``clustered_halos``-- NFW haloes (Navarro, Frenk & White 1997) with a
  power-law count distribution plus a uniform background, standing in for
  a cosmological snapshot.
* ``precision_stress`` -- the clustered mix moved to [1000,1001)^3 with
  log-normal masses.
* ``batched_plummer``  -- thousands of independent Plummer sets.

All draws are FP64 from ``numpy.random.Generator(PCG64(seed))``; the
result is rounded to FP32 once.  Particle order is randomised so that the
input order carries no spatial coherence.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _equal_masses(n: int) -> np.ndarray:
    # 1/n rounded once from FP64 to FP32 (the same value the C-ABI uses
    # when the caller passes no masses).
    return np.full(n, np.float32(1.0 / n) if n > 0 else np.float32(0), dtype=np.float32)


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere (cos(theta) uniform, phi uniform)."""
    mu = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    out = np.empty((n, 3), dtype=np.float64)
    out[:, 0] = s * np.cos(phi)
    out[:, 1] = s * np.sin(phi)
    out[:, 2] = mu
    return out


def uniform_cube(n: int, seed: int):
    """i.i.d. uniform positions in [0,1)^3, equal masses 1/n."""
    rng = _rng(seed)
    pos = rng.random((n, 3)).astype(np.float32)
    return pos, _equal_masses(n)


def _plummer_radii(rng: np.random.Generator, a: np.ndarray, rmax_over_a: float) -> np.ndarray:
    """Plummer radii by inverting M(<r)/M = u: r = a / sqrt(u^(-2/3) - 1).

    ``a`` is one scale radius per requested radius.  Radii beyond
    rmax_over_a * a are redrawn (truncation), in order, until none remain.
    """
    n = a.shape[0]
    r = np.empty(n, dtype=np.float64)
    todo = np.arange(n)
    while todo.size:
        u = rng.random(todo.size)
        u = np.where(u <= 0.0, np.finfo(np.float64).tiny, u)
        rr = a[todo] / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        ok = rr <= rmax_over_a * a[todo]
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    return r


def plummer(n: int, seed: int, a: float = 0.05, centre: float = 0.5, rmax_over_a: float = 20.0):
    """Plummer sphere of scale radius ``a`` centred at (centre,)*3, truncated at
    ``rmax_over_a * a``; equal masses 1/n."""
    rng = _rng(seed)
    r = _plummer_radii(rng, np.full(n, a), rmax_over_a)
    d = _isotropic(rng, n)
    pos = (centre + r[:, None] * d).astype(np.float32)
    return pos, _equal_masses(n)


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radii(rng: np.random.Generator, n: int, conc: float) -> np.ndarray:
    """Radii in units of r_s with NFW enclosed-mass CDF mu(x)/mu(c), x in [0,c].

    Inverse by table lookup (4097 nodes, denser near the centre) followed by
    three Newton steps on mu(x) - u mu(c) = 0, mu'(x) = x / (1+x)^2.
    """
    t = np.linspace(0.0, 1.0, 4097)
    xt = conc * t * t
    mt = _nfw_mu(xt)
    target = rng.random(n) * _nfw_mu(conc)
    x = np.interp(target, mt, xt)
    for _ in range(3):
        xs = np.maximum(x, 1e-12)
        f = _nfw_mu(xs) - target
        x = xs - f * (1.0 + xs) ** 2 / xs
        x = np.clip(x, 0.0, conc)
    return x


def _halo_counts(rng, n_halo, total, mmin, mmax, slope):
    """Power-law counts dN/dM ~ M^-slope on [mmin, mmax], rescaled so that they
    sum to exactly ``total`` (largest-remainder rounding)."""
    g = 1.0 - slope
    u = rng.random(n_halo)
    raw = (mmin ** g + u * (mmax ** g - mmin ** g)) ** (1.0 / g)
    scaled = raw * (total / raw.sum())
    base = np.floor(scaled).astype(np.int64)
    rem = int(total - base.sum())
    if rem > 0:
        order = np.argsort(-(scaled - base), kind="stable")
        base[order[:rem]] += 1
    return base


def clustered_halos(n: int, seed: int, n_halo: int = 10000, conc: float = 10.0,
                    slope: float = 1.9, mmin: float = 100.0, mmax: float = 1e6,
                    halo_frac: float = 0.7, shuffle: bool = True):
    """Cosmology-like clustered particles in [0,1)^3, equal masses 1/n.

    ``halo_frac`` of the particles sit in ``n_halo`` NFW haloes (concentration
    ``conc``) whose counts follow a power law and are rescaled to sum to
    round(halo_frac * n); the rest are uniform.  A halo of M particles has
    virial radius r_vir = (3 M / (4 pi 200 n))^(1/3) (mean density 200 times
    the box mean) and r_s = r_vir / conc; positions wrap periodically.
    """
    rng = _rng(seed)
    n_h = int(round(halo_frac * n))
    counts = _halo_counts(rng, n_halo, n_h, mmin, mmax, slope)
    centres = rng.random((n_halo, 3))
    rvir = (3.0 * counts / (4.0 * math.pi * 200.0 * max(n, 1))) ** (1.0 / 3.0)
    rs = rvir / conc
    hid = np.repeat(np.arange(n_halo), counts)
    x = _nfw_radii(rng, n_h, conc)
    d = _isotropic(rng, n_h)
    hal = centres[hid] + (rs[hid] * x)[:, None] * d
    del d, x
    hal -= np.floor(hal)
    bg = rng.random((n - n_h, 3))
    pos64 = np.concatenate([hal, bg], axis=0)
    del hal, bg
    pos = pos64.astype(np.float32)
    del pos64
    # values that round up to 1.0f stay inside [0,1)
    np.minimum(pos, np.float32(np.nextafter(np.float32(1.0), np.float32(0.0))), out=pos)
    if shuffle:
        pos = pos[rng.permutation(n)]
    return pos, _equal_masses(n)


def precision_stress(n: int, seed: int, **kw):
    """The clustered mix moved to [1000,1001)^3 (x <- fp32(1000 + x), the add
    in FP64) with log-normal masses fp32((1/n) exp(2 Z)), Z ~ N(0,1)."""
    pos, _ = clustered_halos(n, seed, **kw)
    pos = (1000.0 + pos.astype(np.float64)).astype(np.float32)
    rng = _rng(seed + 1_000_003)
    z = rng.standard_normal(n)
    mass = ((1.0 / n) * np.exp(2.0 * z)).astype(np.float32)
    return pos, mass


@dataclass
class BatchedSets:
    pos: np.ndarray        # [N,3] f32, sets contiguous
    mass: np.ndarray       # [N] f32
    offsets: np.ndarray    # [S+1] int64
    scale: np.ndarray      # [S] f64 Plummer scale radius of each set
    seed: int


def batched_plummer(n_sets: int = 4096, seed: int = 4, nmin: int = 256, nmax: int = 65536,
                    amin: float = 0.01, amax: float = 0.2):
    """Independent Plummer sets: sizes floor(exp(U(ln nmin, ln nmax))), scale
    radii log-uniform in [amin, amax], centre 0.5, truncated at 20 a; masses
    1/n_s within set s."""
    rng = _rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_sets))).astype(np.int64)
    sizes = np.clip(sizes, 1, None)
    a = np.exp(rng.uniform(math.log(amin), math.log(amax), n_sets))
    offsets = np.zeros(n_sets + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    aa = np.repeat(a, sizes)
    r = _plummer_radii(rng, aa, 20.0)
    d = _isotropic(rng, total)
    pos = (0.5 + r[:, None] * d).astype(np.float32)
    mass = np.repeat((1.0 / sizes).astype(np.float32), sizes)
    return BatchedSets(pos=pos, mass=mass, offsets=offsets, scale=a, seed=seed)


def exponential_disk(n: int, seed: int, rd: float = 0.05, z0: float = 0.005,
                     rmax_over_rd: float = 10.0, zmax_over_z0: float = 10.0,
                     centre: float = 0.5):
    """Thin exponential disc in the x-y plane centred at (centre,)*3, equal
    masses 1/n.  Surface density ~ exp(-R / rd): R / rd follows a Gamma(2, 1)
    law (enclosed mass 1 - (1 + x) e^-x), redrawn beyond rmax_over_rd; azimuth
    uniform; height z with density ~ sech^2(z / z0), z = z0 atanh(2u - 1),
    redrawn beyond zmax_over_z0."""
    rng = _rng(seed)
    R = rd * rng.gamma(2.0, 1.0, n)
    bad = R > rmax_over_rd * rd
    while bad.any():
        R[bad] = rd * rng.gamma(2.0, 1.0, int(bad.sum()))
        bad = R > rmax_over_rd * rd
    phi = rng.random(n) * (2.0 * math.pi)
    z = z0 * np.arctanh(2.0 * rng.random(n) - 1.0)
    bad = np.abs(z) > zmax_over_z0 * z0
    while bad.any():
        z[bad] = z0 * np.arctanh(2.0 * rng.random(int(bad.sum())) - 1.0)
        bad = np.abs(z) > zmax_over_z0 * z0
    pos = np.empty((n, 3))
    pos[:, 0] = centre + R * np.cos(phi)
    pos[:, 1] = centre + R * np.sin(phi)
    pos[:, 2] = centre + z
    return pos.astype(np.float32), _equal_masses(n)


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
    return z ^ (z >> np.uint64(31))


def jitter_offsets(seed: int, step: int, offsets: np.ndarray, scale: np.ndarray,
                   amplitude: float = 1e-4) -> np.ndarray:
    """Per-axis jitter of batched step ``step`` for every particle.

    For particle i (local index within set s) and axis a the counter
    h = SM(SM(SM(SM(seed) ^ step) ^ s) ^ (4 i + a)) gives u = (h >> 40) 2^-24 in
    [0,1); the jitter is fp32(2u - 1) * fp32(amplitude * a_s), both factors and
    the product in FP32.  Jittered positions are fp32(x_0 + jitter) (FP32 add),
    not cumulative over steps.
    """
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = np.diff(offsets)
    n = int(offsets[-1])
    with np.errstate(over="ignore"):
        set_id = np.repeat(np.arange(len(sizes), dtype=np.uint64), sizes)
        local = (np.arange(n, dtype=np.int64) - np.repeat(offsets[:-1], sizes)).astype(np.uint64)
        h1 = splitmix64(splitmix64(np.uint64(seed)) ^ np.uint64(step))
        h2 = splitmix64(h1 ^ set_id)
        out = np.empty((n, 3), dtype=np.float32)
        amp = np.repeat((amplitude * np.asarray(scale, dtype=np.float64)).astype(np.float32), sizes)
        for ax in range(3):
            h3 = splitmix64(h2 ^ ((local << np.uint64(2)) | np.uint64(ax)))
            u = (h3 >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)
            out[:, ax] = (np.float32(2.0) * u - np.float32(1.0)) * amp
    return out


def lattice(k: int, origin: float = 0.0, spacing: float = 1.0):
    """Regular lattice of (2^k)^3 points at origin + (i + 1/2) * spacing."""
    m = 1 << k
    g = (np.arange(m, dtype=np.float64) + 0.5) * spacing + origin
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)
    return pos, _equal_masses(pos.shape[0])


# The five workloads the build is measured and checked on.
WORKLOADS = {
    "uniform_65536": dict(kind="uniform", n=65536, seed=1, n_crit=16),
    "plummer_2p24": dict(kind="plummer", n=1 << 24, seed=2, n_crit=16),
    "clustered_2p27": dict(kind="clustered", n=1 << 27, seed=3, n_crit=16),
    "batched_4096": dict(kind="batched", n_sets=4096, seed=4, n_crit=16),
    "stress_2p26": dict(kind="stress", n=1 << 26, seed=5, n_crit=16),
    "disk_2p24": dict(kind="disk", n=1 << 24, seed=6, n_crit=16),
}


def workload(kind: str, n: int | None = None, seed: int = 0, **kw):
    """Draw positions and masses of one single-set workload kind at size n."""
    if kind == "uniform":
        return uniform_cube(n, seed)
    if kind == "plummer":
        return plummer(n, seed, **kw)
    if kind == "clustered":
        return clustered_halos(n, seed, **kw)
    if kind == "stress":
        return precision_stress(n, seed, **kw)
    if kind == "disk":
        return exponential_disk(n, seed, **kw)
    raise ValueError(f"unknown workload kind {kind!r}")
