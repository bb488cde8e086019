"""Closed-form pins of the oracle's gravity (Sec. 2.1, Eq. 1).

The oracle's direct sum and its tree walk share one softened point-mass law,
a = -m r / (|r|^2 + eps^2)^(3/2) with r = x_target - x_source (G = 1), and the
walk adds the quadrupole term of a cell's traceless tensor.  Comparing the
two routines with each other cannot show a mistake they share, so these
tests hold each to values fixed by the mathematics alone:
  - two bodies at hand-chosen separations and softening lengths (sign, power
    and softening of the law);
  - Newton's shell theorem: outside a uniform spherical shell the field is
    that of a point mass at its centre, inside it vanishes (holds only for an
    inverse-square law);
  - a lone particle feels nothing (self-interaction excluded);
  - a cell of two equal masses seen from far along their axis: the monopole
    plus quadrupole of the walk equals the series of the exact two-body sum
    through second order, 2m/D^2 (1 + 3 a^2/D^2), with a = h/2.
"""
import math

import numpy as np
import pytest

import oracle


def _pair(x1, m1, eps):
    """Acceleration of a massless particle at the origin from one body."""
    pos = np.array([[0.0, 0.0, 0.0], x1], dtype=np.float32)
    mass = np.array([0.0, m1], dtype=np.float32)
    return oracle.direct_acc(pos, mass, np.array([0]), eps)[0]


@pytest.mark.parametrize("x1,m1,eps,expect", [
    # |r|^2 = 25, eps = 0: a = m (3, 4, 0) / 125, towards the body
    ((3.0, 4.0, 0.0), 2.0, 0.0, (6.0 / 125, 8.0 / 125, 0.0)),
    # |r|^2 + eps^2 = 25 + 11 = 36, 36^(3/2) = 216
    ((3.0, 4.0, 0.0), 2.0, math.sqrt(11.0), (6.0 / 216, 8.0 / 216, 0.0)),
    # twice the distance, a quarter of the pull (inverse square)
    ((0.0, -6.0, 8.0), 1.0, 0.0, (0.0, -6.0 / 1000, 8.0 / 1000)),
    # |r|^2 + eps^2 = 1 + 3 = 4, 4^(3/2) = 8
    ((0.0, 0.0, -1.0), 0.5, math.sqrt(3.0), (0.0, 0.0, -0.5 / 8)),
])
def test_two_bodies_closed_form(x1, m1, eps, expect):
    a = _pair(x1, m1, eps)
    assert np.allclose(a, expect, rtol=1e-14, atol=1e-17)


def test_two_bodies_newton_third_law():
    pos = np.array([[0.25, -0.5, 1.0], [2.0, 0.75, -1.5]], dtype=np.float32)
    mass = np.array([3.0, 0.5], dtype=np.float32)
    a = oracle.direct_acc(pos, mass, np.array([0, 1]), 0.1)
    # m0 a0 = -m1 a1
    assert np.allclose(3.0 * a[0], -0.5 * a[1], rtol=1e-14, atol=0)


def test_lone_particle_feels_nothing():
    pos = np.array([[0.3, 0.2, 0.1]], dtype=np.float32)
    for eps in (0.0, 0.01):
        a = oracle.direct_acc(pos, np.array([1.0], np.float32), np.array([0]), eps)
        assert np.array_equal(a, np.zeros((1, 3)))


def _fibonacci_shell(n, radius):
    """n nearly uniform points on a sphere (golden-angle spiral)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _shell_acc(target):
    n, R, M = 4000, 1.0, 2.0
    shell = _fibonacci_shell(n, R)
    pos = np.vstack([shell, np.asarray(target)[None, :]]).astype(np.float32)
    mass = np.concatenate([np.full(n, M / n), [0.0]]).astype(np.float32)
    Mf = float(mass[:n].astype(np.float64).sum())
    return oracle.direct_acc(pos, mass, np.array([n]), 0.0)[0], Mf, pos[n].astype(np.float64)


@pytest.mark.parametrize("target", [(3.0, 0.0, 0.0), (0.0, -1.8, 1.2), (1.5, 1.5, -1.5)])
def test_shell_theorem_outside(target):
    """Outside the shell: a = -M x / |x|^3 (centre at the origin)."""
    a, M, x = _shell_acc(target)
    expect = -M * x / np.linalg.norm(x) ** 3
    assert np.linalg.norm(a - expect) <= 2e-4 * np.linalg.norm(expect)


@pytest.mark.parametrize("target", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.1), (0.0, 0.5, 0.0)])
def test_shell_theorem_inside(target):
    """Inside the shell the pulls cancel: |a| is a sampling residue, far
    below the M / R^2 scale (a softened or non-inverse-square law leaves a
    net pull of order M / R^2 off centre)."""
    a, M, _ = _shell_acc(target)
    assert np.linalg.norm(a) <= 2e-3 * M


def test_shell_theorem_through_the_tree_walk():
    """The walk at an opening angle that accepts cells gives the same closed
    form outside the shell (monopole + quadrupole of cells of the shell)."""
    n, R, M = 4000, 1.0, 2.0
    shell = _fibonacci_shell(n, R)
    x = np.array([6.0, 1.0, -2.0])
    pos = np.vstack([shell, x[None, :]]).astype(np.float32)
    mass = np.concatenate([np.full(n, M / n), [0.0]]).astype(np.float32)
    t = oracle.build_tree(pos, 8)
    Mc, com, q, _ = oracle.moments(t, pos, mass)
    a = oracle.tree_walk(t, pos, mass, Mc, com, q, np.array([n]), 0.6, 0.0, True)[0]
    xf = pos[n].astype(np.float64)
    Mf = float(mass[:n].astype(np.float64).sum())
    expect = -Mf * xf / np.linalg.norm(xf) ** 3
    assert np.linalg.norm(a - expect) <= 2e-4 * np.linalg.norm(expect)


def _axis_pair_walk(use_quad):
    """Target at the origin; two equal masses m at z = D - a and z = D + a
    (D = 1, a = h / 2).  With n_crit 2 the root splits and the pair's depth-1
    cell (side ~D/2, distance D) is accepted at theta 0.75."""
    h = 0.0625                      # exact in FP32
    m = 0.5
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.0 - h / 2], [0.0, 0.0, 1.0 + h / 2]],
                   dtype=np.float32)
    mass = np.array([0.0, m, m], dtype=np.float32)
    t = oracle.build_tree(pos, 2)
    assert t.n_cells == 3                     # root + two depth-1 leaves
    Mc, com, q, _ = oracle.moments(t, pos, mass)
    a = oracle.tree_walk(t, pos, mass, Mc, com, q, np.array([0]), 0.75, 0.0, use_quad)[0]
    return a, m, 1.0, h / 2


def test_quadrupole_of_an_axis_pair_closed_form():
    a, m, D, h2 = _axis_pair_walk(True)
    exact = m / (D - h2) ** 2 + m / (D + h2) ** 2          # the two-body sum, +z
    series2 = 2 * m / D ** 2 * (1 + 3 * h2 ** 2 / D ** 2)  # through second order
    rest = 2 * m / D ** 2 * 5 * h2 ** 4 / D ** 4           # leading term dropped
    assert abs(a[0]) < 1e-15 and abs(a[1]) < 1e-15
    # the walk's monopole + quadrupole is the second-order series exactly
    assert abs(a[2] - series2) <= 1e-13 * series2
    # which differs from the exact sum by the fourth-order term only
    assert abs((exact - a[2]) - rest) <= 0.1 * rest


def test_monopole_alone_misses_the_second_order_term():
    a, m, D, h2 = _axis_pair_walk(False)
    assert abs(a[2] - 2 * m / D ** 2) <= 1e-13 * 2 * m / D ** 2
