"""Pins of the oracle's RKC (Section 2.2) and power method (Appendix).

The m-stage step on y' = lambda y must equal the damped shifted Chebyshev
stability polynomial P_m(z) = a_m + b_m T_m(w0 + w1 z), evaluated here with
numpy's Clenshaw recurrence and hyperbolic closed forms -- not with the
oracle's three-term recurrence.  Stage times are checked against the closed
form c_j = (T_m'/T_m'')(T_j''/T_j'), the empirical order against 2 and the
power method against eigenvalues from numpy.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as cheb

import oracle as O

KAPPA = 2.0 / 13.0


def cheb_at(m, x):
    """T_m(x), T_m'(x), T_m''(x) for x > 1 from x = cosh(theta)."""
    th = math.acosh(x)
    sh, ch = math.sinh(th), math.cosh(th)
    T = math.cosh(m * th)
    Tp = m * math.sinh(m * th) / sh
    Tpp = m * (m * math.cosh(m * th) * sh - math.sinh(m * th) * ch) / sh ** 3
    return T, Tp, Tpp


def stability_poly(m):
    w0 = 1.0 + KAPPA / m ** 2
    T, Tp, Tpp = cheb_at(m, w0)
    w1 = Tp / Tpp
    b = Tpp / Tp ** 2
    a = 1.0 - b * T
    e = np.zeros(m + 1)
    e[m] = 1.0
    return (lambda z: a + b * cheb.chebval(w0 + w1 * np.asarray(z), e)), w0, w1


@pytest.mark.parametrize("m", [2, 3, 5, 8, 13, 21, 34, 50])
def test_one_step_is_damped_chebyshev_polynomial(m):
    P, w0, w1 = stability_poly(m)
    mod = O.model(O.KIND_LINEAR, 1, 1)
    beta = (1.0 + w0) / w1          # where w0 + w1 z reaches -1
    for z in np.linspace(-beta, 0.0, 23):
        h = 0.5
        y = O.rkc_step(mod, [z / h], [1.0], h, m)[0]
        assert y == pytest.approx(P(z), abs=1e-12 * max(1.0, m * m / 10.0)), (m, z)


def test_stability_polynomial_is_second_order_and_bounded():
    for m in (2, 4, 10, 30):
        P, w0, w1 = stability_poly(m)
        # P(z) = 1 + z + z^2/2 + O(z^3): numerical Taylor coefficients
        eps = 1e-3
        p0 = P(0.0)
        d1 = (P(eps) - P(-eps)) / (2 * eps)
        d2 = (P(eps) - 2 * p0 + P(-eps)) / eps ** 2
        assert p0 == pytest.approx(1.0, abs=1e-14)
        assert d1 == pytest.approx(1.0, rel=1e-6)
        assert d2 == pytest.approx(1.0, rel=1e-4)
        # stable on the interval the stage-count rule uses: h sigma <= (m^2-1)/1.54
        z = np.linspace(-(m * m - 1) / 1.54, 0.0, 400)
        assert np.all(np.abs(P(z)) <= 1.0 + 1e-12)


@pytest.mark.parametrize("m", [2, 3, 7, 16, 40])
def test_stage_times_match_closed_form(m):
    co = O.rkc_coeffs(m)
    c = co["c"]
    w0 = 1.0 + KAPPA / m ** 2
    _, Tpm, Tppm = cheb_at(m, w0)
    for j in range(2, m + 1):
        _, Tpj, Tppj = cheb_at(j, w0)
        assert c[j] == pytest.approx(Tpm / Tppm * Tppj / Tpj, rel=1e-11)
    assert c[m] == pytest.approx(1.0, rel=1e-12)
    _, Tp2, _ = cheb_at(2, w0)
    assert c[1] == pytest.approx(c[2] / Tp2, rel=1e-12)      # Tp2 = 4 w0
    for j in range(2, m):
        assert abs(c[j] - (j * j - 1) / (m * m - 1)) < 0.05


def test_time_dependent_rhs_is_integrated_exactly():
    mod = O.model(O.KIND_TIME, 1, 1)
    for m in (2, 5, 11):
        t0, h = 0.3, 0.25
        y = O.rkc_step(mod, [0.0], [1.0], h, m, t=t0)[0]
        assert y == pytest.approx(1.0 + t0 * h + h * h / 2, rel=1e-14)


def test_second_order_convergence():
    mod = O.model(O.KIND_VDP, 2, 1)
    ys = [O.fixed_steps(mod, [1.0], [2.0, 0.0], 1, 1.0 / n, n, stages=4) for n in (16, 32, 64, 128, 256)]
    diffs = [np.abs(ys[k] - ys[k + 1]).max() for k in range(len(ys) - 1)]
    slopes = [math.log2(diffs[k] / diffs[k + 1]) for k in range(len(diffs) - 1)]
    assert 1.85 < slopes[-1] < 2.15, slopes


def test_adaptive_global_error_scales_as_tol_two_thirds():
    # local error per step ~ h^3 is held at tol, so h ~ tol^(1/3) and the
    # global error of a second-order method ~ h^2 ~ tol^(2/3)
    mod = O.model(O.KIND_LINEAR, 1, 1)
    errs = []
    tols = [1e-4, 1e-6, 1e-8]
    for rtol in tols:
        r = O.integrate(mod, 1, [[1.0]], [[-1.0]], 0.0, 2.0, rtol, rtol * 1e-3)
        assert r.status[0] == 0
        errs.append(abs(r.y[0, 0] / math.exp(-2.0) - 1.0))
    for rtol, e in zip(tols, errs):
        assert e < 2.0 * rtol ** (2.0 / 3.0)
    slope = math.log(errs[0] / errs[-1]) / math.log(tols[0] / tols[-1])
    assert 0.55 < slope < 0.78, slope


def test_adaptive_stiff_linear_against_expm():
    from scipy.linalg import expm
    M = np.array([[-1.0, 0.5], [0.0, -800.0]])
    y0 = np.array([1.0, 2.0])
    mod = O.model(O.KIND_LINEAR, 2, 4)
    for rtol, atol in [(1e-4, 1e-7), (1e-6, 1e-9)]:
        r = O.integrate(mod, 1, y0[:, None], M.ravel()[:, None], 0.0, 2.0, rtol, atol)
        assert r.status[0] == 0
        exact = expm(2.0 * M) @ y0
        assert abs(r.y[0, 0] / exact[0] - 1.0) < 2.0 * rtol ** (2.0 / 3.0)
        assert abs(r.y[1, 0]) < 10 * atol


def test_zero_rhs_control_flow():
    # f = 0: sigma = 0 after two power iterations, the trial step has zero
    # error so h = hmax, m = 2 and one accepted step closes the interval
    mod = O.model(O.KIND_LINEAR, 1, 1)
    r = O.integrate(mod, 1, [[3.0]], [[0.0]], 0.0, 8.0, 1e-6, 1e-9)
    assert r.n_accept[0] == 1 and r.n_reject[0] == 0
    assert r.n_specrad_iter[0] == 2 and r.n_rhs[0] == 6
    assert r.y[0, 0] == 3.0


def test_power_method_diagonal():
    M = np.diag([-1.0, -5.0, -50.0])
    mod = O.model(O.KIND_LINEAR, 3, 9)
    y = np.array([1.0, 2.0, 3.0])
    v = M @ y
    r, v2, it, st = O.specrad(mod, M.ravel(), y, 10.0, v)
    assert st == 0 and 2 <= it <= 50
    assert r / 1.2 == pytest.approx(50.0, rel=1e-2)
    assert r / 1.2 <= 50.0 * (1 + 1e-12)


def test_power_method_laplacian():
    n, a = 12, 0.02
    dx = 1.0 / (n + 1)
    L = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) * a / dx ** 2
    rho = np.abs(np.linalg.eigvalsh(L)).max()
    assert rho == pytest.approx(4 * a / dx ** 2 * math.sin(n * math.pi / (2 * (n + 1))) ** 2, rel=1e-12)
    mod = O.model(O.KIND_LINEAR, n, n * n)
    y = np.linspace(0.5, 1.5, n)
    r, _, it, st = O.specrad(mod, L.ravel(), y, 10.0, L @ y)
    sigma = r / 1.2
    assert sigma <= rho * (1 + 1e-12)
    assert sigma > 0.9 * rho, (sigma, rho, it)


def test_power_method_nonconvergence_flag():
    # A = [[0, 1], [-100, 0]] maps e1 -> -100 e2 and e2 -> e1, so the ratio
    # |A d| / |d| alternates between 100 and 1 and never settles to 1%
    M = np.array([[0.0, 1.0], [-100.0, 0.0]])
    mod = O.model(O.KIND_LINEAR, 2, 4)
    r, _, it, st = O.specrad(mod, M.ravel(), np.array([1.0, 0.0]), 1.0, np.array([1.0, 0.0]))
    assert it == 50 and st == O.ST_SPECRAD_NOCONV


def test_cross_method_brusselator():
    from paper_1611_02274_gb300 import workloads as W
    w = W.bruss(nsys=4, n=8)
    mod = O.model_for(w)
    ref = O.integrate(mod, 0, w.y0, w.params, 0.0, 10.0, 1e-11, 1e-14)
    rkc = O.integrate(mod, 1, w.y0, w.params, 0.0, 10.0, 1e-6, 1e-9)
    # the power method may stop at 50 iterations on the complex pair of
    # the Brusselator (a warning bit, not a failure)
    assert (ref.status == 0).all() and ((rkc.status & 0xFF) == 0).all()
    rel = np.abs(rkc.y - ref.y) / (np.abs(ref.y) + 1e-9)
    assert rel.max() < 1e-6 ** (2.0 / 3.0), rel.max()
