"""Pins of the oracle's RKCK (Section 2.1, Table 1) against mathematics.

Nothing here retypes the oracle's formulas: the tableau is checked against
the Runge-Kutta order conditions, one step on y' = lambda y against the
stability polynomial expanded in exact rationals (whose first Taylor
coefficients are fixed by order theory alone), adaptive runs against exact
solutions, and the empirical convergence order against 5.
"""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_tableau():
    a, b, c, cs = [], [], [], []
    with open(os.path.join(GOLDEN, "rkck_tableau.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            cols = [x.strip() for x in line.split("|")]
            a.append(Fr(cols[1]))
            b.append([Fr(x) for x in cols[2].split()])
            c.append(Fr(cols[3]))
            cs.append(Fr(cols[4]))
    s = len(a)
    A = [[Fr(0)] * s for _ in range(s)]
    for i in range(s):
        for j, v in enumerate(b[i]):
            A[i][j] = v
    return a, A, c, cs


def _dot(u, v):
    return sum((x * y for x, y in zip(u, v)), Fr(0))


def _matvec(A, v):
    return [_dot(row, v) for row in A]


def order_conditions(A, w, cvec, order):
    """Butcher's order conditions up to ``order`` (trees up to order 5)."""
    s = len(w)
    one = [Fr(1)] * s
    c = cvec
    c2 = [x * x for x in c]
    c3 = [x ** 3 for x in c]
    Ac = _matvec(A, c)
    Ac2 = _matvec(A, c2)
    AAc = _matvec(A, Ac)
    conds = {
        1: [(_dot(w, one), Fr(1))],
        2: [(_dot(w, c), Fr(1, 2))],
        3: [(_dot(w, c2), Fr(1, 3)), (_dot(w, Ac), Fr(1, 6))],
        4: [(_dot(w, c3), Fr(1, 4)), (_dot(w, [x * y for x, y in zip(c, Ac)]), Fr(1, 8)),
            (_dot(w, Ac2), Fr(1, 12)), (_dot(w, AAc), Fr(1, 24))],
        5: [(_dot(w, [x ** 4 for x in c]), Fr(1, 5)),
            (_dot(w, [x * x * y for x, y in zip(c, Ac)]), Fr(1, 10)),
            (_dot(w, [x * y for x, y in zip(c, Ac2)]), Fr(1, 15)),
            (_dot(w, [x * y for x, y in zip(c, AAc)]), Fr(1, 30)),
            (_dot(w, [y * y for y in Ac]), Fr(1, 20)),
            (_dot(w, _matvec(A, c3)), Fr(1, 20)),
            (_dot(w, _matvec(A, [x * y for x, y in zip(c, Ac)])), Fr(1, 40)),
            (_dot(w, _matvec(A, Ac2)), Fr(1, 60)),
            (_dot(w, _matvec(A, AAc)), Fr(1, 120))],
    }
    return [pair for k in range(1, order + 1) for pair in conds[k]]


def test_golden_tableau_satisfies_order_conditions():
    a, A, c, cs = load_tableau()
    for i in range(len(a)):
        assert sum(A[i], Fr(0)) == a[i], f"row sum of stage {i + 1}"
    for lhs, rhs in order_conditions(A, c, a, 5):
        assert lhs == rhs
    for lhs, rhs in order_conditions(A, cs, a, 4):
        assert lhs == rhs
    # the embedded weights are NOT fifth order (else the error estimate vanishes)
    assert any(l != r for l, r in order_conditions(A, cs, a, 5)[8:])


def stability_poly(A, w):
    """Coefficients of R(z) = 1 + sum_k z^k w^T A^(k-1) 1 (exact)."""
    s = len(w)
    v = [Fr(1)] * s
    coef = [Fr(1)]
    for _ in range(s):
        coef.append(_dot(w, v))
        v = _matvec(A, v)
    return coef


def test_stability_polynomials_have_taylor_coefficients():
    a, A, c, cs = load_tableau()
    R5 = stability_poly(A, c)
    R4 = stability_poly(A, cs)
    for k in range(6):
        assert R5[k] == Fr(1, math.factorial(k))
    for k in range(5):
        assert R4[k] == Fr(1, math.factorial(k))
    assert R4[5] != Fr(1, 120)


def _polyval(coef, z):
    return sum(float(ck) * z ** k for k, ck in enumerate(coef))


@pytest.mark.parametrize("z", [-3.0, -1.0, -0.25, -0.01, 0.3, 1.0])
def test_one_step_on_linear_scalar(z):
    a, A, c, cs = load_tableau()
    R5 = stability_poly(A, c)
    R4 = stability_poly(A, cs)
    lam, h, y0 = -2.0, -z / 2.0, 1.7
    m = O.model(O.KIND_LINEAR, 1, 1)
    yo, ye = O.rkck_step(m, [lam], [y0], h)
    assert yo[0] == pytest.approx(_polyval(R5, z) * y0, rel=4e-15, abs=1e-16)
    # the difference polynomial starts at z^5; evaluate it without cancellation
    want_err = _polyval([x - y for x, y in zip(R5, R4)], z) * y0
    assert ye[0] == pytest.approx(want_err, rel=1e-9, abs=1e-18)


def test_one_step_on_linear_system_is_matrix_polynomial():
    a, A, c, cs = load_tableau()
    R5 = [float(x) for x in stability_poly(A, c)]
    rng = np.random.default_rng(1)
    M = rng.normal(size=(4, 4))
    h = 0.3
    y0 = rng.normal(size=4)
    m = O.model(O.KIND_LINEAR, 4, 16)
    yo, _ = O.rkck_step(m, M.ravel(), y0, h)
    P = sum(ck * np.linalg.matrix_power(h * M, k) for k, ck in enumerate(R5))
    np.testing.assert_allclose(yo, P @ y0, rtol=1e-13, atol=1e-14)


def test_stage_times_integrate_time_exactly():
    # y' = t: a consistent fifth-order method is exact for a polynomial in t
    m = O.model(O.KIND_TIME, 1, 1)
    t0, h = 0.7, 0.4
    yo, _ = O.rkck_step(m, [0.0], [2.0], h, t=t0)
    assert yo[0] == pytest.approx(2.0 + t0 * h + h * h / 2, rel=1e-15)


@pytest.mark.parametrize("rtol", [1e-4, 1e-6, 1e-8, 1e-10])
def test_adaptive_harmonic_oscillator(rtol):
    # van der Pol with mu = 0 is y1'' = -y1: exact cos/sin
    m = O.model(O.KIND_VDP, 2, 1)
    y0 = np.array([[1.0, 0.3], [0.0, -1.2]])
    r = O.integrate(m, 0, y0, [[0.0, 0.0]], 0.0, 20.0, rtol, 0.0)
    assert (r.status == 0).all()
    for i in range(2):
        a, b = y0[0, i], y0[1, i]
        exact = np.array([a * math.cos(20) + b * math.sin(20), -a * math.sin(20) + b * math.cos(20)])
        err = np.abs(r.y[:, i] - exact).max()
        assert err < 200 * rtol, (rtol, err)


def test_adaptive_error_is_proportional_to_tolerance():
    m = O.model(O.KIND_LINEAR, 1, 1)
    errs = []
    for rtol in [1e-5, 1e-7, 1e-9]:
        r = O.integrate(m, 0, [[1.0]], [[-1.0]], 0.0, 5.0, rtol, 0.0)
        errs.append(abs(r.y[0, 0] - math.exp(-5.0)) / math.exp(-5.0))
        assert errs[-1] < 50 * rtol
    assert errs[0] > errs[1] > errs[2]


def test_zero_rhs_takes_two_accepted_steps():
    # f = 0: err = 0, the first step (h = T/2) is accepted, h grows by the
    # maximum factor 5 (capped at hmax = T) and the last step closes the interval
    m = O.model(O.KIND_LINEAR, 1, 1)
    r = O.integrate(m, 0, [[3.0]], [[0.0]], 0.0, 8.0, 1e-6, 1e-9)
    assert r.n_accept[0] == 2 and r.n_reject[0] == 0 and r.n_rhs[0] == 12
    assert r.y[0, 0] == 3.0


def test_fifth_order_convergence():
    m = O.model(O.KIND_VDP, 2, 1)
    y0 = [2.0, 0.0]
    ys = [O.fixed_steps(m, [1.0], y0, 0, 1.0 / n, n) for n in (8, 16, 32, 64, 128)]
    diffs = [np.abs(ys[k] - ys[k + 1]).max() for k in range(len(ys) - 1)]
    slopes = [math.log2(diffs[k] / diffs[k + 1]) for k in range(len(diffs) - 1)]
    assert 4.7 < slopes[-1] < 5.3, slopes


def test_paper_constants_are_consistent():
    consts = {}
    with open(os.path.join(GOLDEN, "constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            consts[k] = float(Fr(v)) if "/" in v else float(v)
    # ERRCON is the error at which the growth rule S err^PGROW reaches the cap 5
    errcon = (consts["MAX_GROWTH"] / consts["SAFETY"]) ** (1.0 / consts["PGROW"])
    assert errcon == pytest.approx(consts["ERRCON"], rel=2e-3)


def test_embedded_error_estimate_is_fifth_order_in_h():
    # y5 - y4 is the local error of the fourth-order solution: O(h^5) on a
    # nonlinear problem, which pins every c_i - c*_i against the stages
    m = O.model(O.KIND_VDP, 2, 1)
    errs = [np.abs(O.rkck_step(m, [1.5], [1.2, -0.4], h)[1]).max() for h in (0.04, 0.02, 0.01)]
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert 4.8 < slopes[-1] < 5.2, slopes
