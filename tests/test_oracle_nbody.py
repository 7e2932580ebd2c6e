"""Pins of the oracle's planar n-body right-hand side (the form of the
Pleiades problem the paper integrates with RKCK, Section 4.1).

Fixed by mechanics rather than by the formula: Runge-Kutta methods keep
linear invariants exactly, so total momentum stays constant and the centre
of mass moves on a straight line to rounding; energy drifts only within
the tolerance; a two-body circular orbit follows its closed form; forces
obey Newton's third law.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import workloads as W

RKCK, RKC = 0, 1


def split(y, n):
    return y[:n], y[n:2 * n], y[2 * n:3 * n], y[3 * n:]


def energy(m, y, G=1.0):
    n = m.size
    x, yy, u, v = split(y, n)
    kin = 0.5 * np.sum(m * (u * u + v * v))
    pot = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            pot -= G * m[i] * m[j] / np.hypot(x[j] - x[i], yy[j] - yy[i])
    return kin + pot


def test_forces_obey_the_third_law():
    m, base = W.pleiades_base()
    mod = O.model(O.KIND_NBODY, 28, 1, masses=m)
    f = O.rhs(mod, [1.0], base)
    _, _, ax, ay = split(f, 7)
    assert abs(np.sum(m * ax)) <= 1e-13 * np.sum(np.abs(m * ax))
    assert abs(np.sum(m * ay)) <= 1e-13 * np.sum(np.abs(m * ay))
    # and the positions' derivatives are the velocities
    np.testing.assert_array_equal(f[:14], base[14:])


def test_rkck_keeps_momentum_and_moves_the_centre_of_mass_linearly():
    w = W.pleiades(16, seed=3)
    m = w.aux["masses"]
    r = O.integrate_workload(w)
    assert np.all(r.status == 0)
    for i in range(w.nsys):
        y0, y1 = w.y0[:, i], r.y[:, i]
        x0, yy0, u0, v0 = split(y0, 7)
        x1, yy1, u1, v1 = split(y1, 7)
        scale = np.sum(m * (np.abs(u0) + np.abs(v0)))
        assert abs(np.sum(m * u1) - np.sum(m * u0)) <= 1e-12 * scale
        assert abs(np.sum(m * v1) - np.sum(m * v0)) <= 1e-12 * scale
        M = m.sum()
        cx0, cx1 = np.sum(m * x0) / M, np.sum(m * x1) / M
        assert abs(cx1 - (cx0 + w.tend * np.sum(m * u0) / M)) <= 1e-12 * (1 + abs(cx0))


def test_energy_drift_is_within_tolerance():
    w = W.pleiades(8, seed=5)
    m = w.aux["masses"]
    r = O.integrate_workload(w)
    for i in range(w.nsys):
        e0, e1 = energy(m, w.y0[:, i]), energy(m, r.y[:, i])
        assert abs(e1 - e0) <= 1e-7 * abs(e0), (e0, e1)


@pytest.mark.parametrize("method", [RKCK, RKC])
def test_two_body_circular_orbit(method):
    # masses 1 and 3 at distance d on a circular orbit about the centre of
    # mass: the separation vector turns at omega = sqrt(G (m1 + m2) / d^3)
    m1, m2, d, G = 1.0, 3.0, 2.0, 1.5
    M = m1 + m2
    omega = np.sqrt(G * M / d ** 3)
    r1, r2 = d * m2 / M, d * m1 / M
    y0 = np.array([-r1, r2, 0.0, 0.0, 0.0, 0.0, -omega * r1, omega * r2])
    mod = O.model(O.KIND_NBODY, 8, 1, masses=[m1, m2])
    T = 2.0
    res = O.integrate(mod, method, y0[:, None], np.array([[G]]), 0.0, T, 1e-10, 1e-12)
    th = omega * T
    exact = np.array([-r1 * np.cos(th), r2 * np.cos(th), -r1 * np.sin(th), r2 * np.sin(th),
                      r1 * omega * np.sin(th), -r2 * omega * np.sin(th), -r1 * omega * np.cos(th),
                      r2 * omega * np.cos(th)])
    tol = 1e-7 if method == RKCK else 1e-5   # RKC is second order: rtol^(2/3)-sized global error
    np.testing.assert_allclose(res.y[:, 0], exact, atol=tol * d)
