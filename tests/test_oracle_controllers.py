"""Pins of the oracle's step-size controllers against an independent
50-digit restatement (mpmath) on linear 2 x 2 systems y' = A y.

For a linear right-hand side one step of either method has a closed form,
so the restatement needs none of the oracle's step code:
  * RKCK (Section 2.1): y_{n+1} = R5(hA) y_n and the embedded error
    Delta = (R5 - R4)(hA) y_n, with R5 and R4 the stability polynomials of
    the golden Table 1 (exact rationals, pinned by the order conditions);
  * RKC (Section 2.2): y_{n+1} = P_m(hA) y_n with P_m(z) = a_m + b_m T_m(w0 +
    w1 z), w0 = 1 + (2/13)/m^2, w1 = T_m'(w0)/T_m''(w0), b_m =
    T_m''(w0)/T_m'(w0)^2, a_m = 1 - b_m T_m(w0) (Chebyshev T_m and its
    derivatives from the textbook identities T_m' = m U_{m-1} and
    (x^2 - 1) T_m'' = m ((m + 1) T_m - U_m)).
The controllers are restated from the paper's text: RKCK's Eq. E:hnew with
safety factor 0.9, exponents -1/5 (growth) and -1/4 (shrink), growth cap 5
below ERRCON = 1.89e-4 and the factor-of-ten limit P1 = 0.1 (reading R1);
RKC's rejection rule h = 0.8 h / err^(1/3), Eqs. dtnp1 / rkc-f with err_old
and h_old, the initial-step rule (Euler trial of size 1/sigma), the stage
count m = 1 + floor(sqrt(1.54 h sigma + 1)) with its cap
m_max = round(sqrt(rtol / (10 uround))).  The spectral radius comes from the
Gershgorin bound (reading R23), which for a constant Jacobian A is the
largest absolute row sum: a closed form.

The oracle is stopped after K attempts (attempt cap) and its carry state --
time reached, next step size, h_old, err_old, accepted-step count -- and its
counters are compared with the restatement's after the same K attempts.
Every run includes at least one rejected step.
"""
import numpy as np
import pytest

import oracle as O

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp

from test_oracle_rkck import load_tableau, stability_poly  # noqa: E402

UROUND = mpmath.mpf("2.22e-16")
# Agreement of the FP64 oracle with the 50-digit restatement.  An error
# estimate is a difference that cancels to ~err * rtol of the state, so its
# FP64 value carries an absolute rounding error of ~1e-9 (in units of the
# tolerance) whatever its size: ERR_ABS.  Step sizes depend on err^(1/3) or
# err^(2/3) and agree to REL where the estimate is not tiny (a tiny one makes
# the growth cap 10 bind).  Accept / reject decisions, stage counts and
# evaluation counts must agree exactly.
REL = 1e-6
ERR_ABS = 1e-8
REL_NL = 1e-3


def mpmat(A):
    return mpmath.matrix([[mpmath.mpf(float(x)) for x in row] for row in A])


def poly_of_matrix(coef, M):
    """sum_k coef[k] M^k (Horner)."""
    n = M.rows
    acc = mpmath.zeros(n, n)
    I = mpmath.eye(n)
    for c in reversed(coef):
        acc = acc * M + I * mpmath.mpf(c.numerator) / c.denominator
    return acc


def run_linear(A, y0, t0, tend, rtol, atol, method, K, specrad=O.SPECRAD_POWER, carry=None):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    mod = O.model(O.KIND_LINEAR, n, n * n)
    cin = None if carry is None else np.asarray(carry, dtype=np.float64).reshape(-1, 1)
    return O.integrate(mod, method, np.asarray(y0, np.float64).reshape(n, 1), A.reshape(n * n, 1), t0, tend,
                       rtol, atol, max_attempts=K, nthreads=1, carry_out=True, carry_in=cin, specrad=specrad)


# ------------------------------------------------------------------ RKCK

def rkck_restated(A, y0, t0, tend, rtol, atol, K, h0=None):
    """Section 2.1's adaptive RKCK (rkckDriver control flow) for K attempts;
    h0 = a carried first step size (reading R21), else half the interval."""
    mp.dps = 50
    _, Atab, c, cs = load_tableau()
    r5 = stability_poly(Atab, c)
    r4 = stability_poly(Atab, cs)
    L = max(len(r5), len(r4))
    r5 = list(r5) + [0] * (L - len(r5))
    r4 = list(r4) + [0] * (L - len(r4))
    from fractions import Fraction as Fr
    e = [Fr(a) - Fr(b) for a, b in zip(r5, r4)]
    r5 = [Fr(a) for a in r5]
    Am = mpmat(A)
    y = mpmath.matrix([mpmath.mpf(float(v)) for v in y0])
    t, tend = mpmath.mpf(t0), mpmath.mpf(tend)
    hmax = abs(tend - t)
    hmin = mpmath.mpf("1e-20")
    delta = mpmath.mpf(atol) / mpmath.mpf(rtol)          # reading R2
    h = hmax / 2 if h0 is None else mpmath.mpf(h0)
    acc = rej = 0
    trace = []
    for _ in range(K):
        if not t < tend:
            break
        h = min(tend - t, h)
        F = Am * y
        y5 = poly_of_matrix(r5, Am * h) * y
        D = poly_of_matrix(e, Am * h) * y
        err = max(abs(D[i]) / (abs(y[i]) + abs(h * F[i]) + delta) for i in range(len(y0))) / mpmath.mpf(rtol)
        if err > 1:   # reject: shrink by 0.9 err^(-1/4), at most by the factor ten P1
            rej += 1
            h = max(mpmath.mpf("0.9") * h * err ** mpmath.mpf(-0.25), mpmath.mpf("0.1") * h)
            trace.append(("reject", err))
        else:         # accept: grow by 0.9 err^(-1/5), by 5 below ERRCON
            acc += 1
            t = t + h
            h = mpmath.mpf("0.9") * h * err ** mpmath.mpf(-0.2) if err > mpmath.mpf("1.89e-4") else 5 * h
            h = max(hmin, min(hmax, h))
            y = y5
            trace.append(("accept", err))
    return dict(t=t, h=h, y=y, acc=acc, rej=rej, trace=trace)


RKCK_CASES = {
    # stiff-ish coupled pair: the first h = 0.5 is rejected, then accepted steps grow
    "coupled": ([[-40.0, 6.0], [3.0, -2.0]], [1.0, 0.5], 1e-6, 1e-9),
    # rotation with decay: complex eigenvalues, a rejection at the start
    "rotation": ([[-0.5, 9.0], [-9.0, -0.5]], [1.0, 0.0], 1e-7, 1e-10),
}


@pytest.mark.parametrize("case", sorted(RKCK_CASES))
@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_rkck_controller_decisions(case, K):
    A, y0, rtol, atol = RKCK_CASES[case]
    ref = rkck_restated(A, y0, 0.0, 1.0, rtol, atol, K)
    r = run_linear(A, y0, 0.0, 1.0, rtol, atol, 0, K)
    assert (int(r.n_accept[0]), int(r.n_reject[0])) == (ref["acc"], ref["rej"]), ref["trace"]
    assert int(r.n_rhs[0]) == 6 * (ref["acc"] + ref["rej"])
    c = r.carry[:, 0]
    assert c[1] == pytest.approx(float(ref["t"]), rel=REL, abs=1e-300)        # time reached
    assert c[2] == pytest.approx(float(ref["h"]), rel=REL)                    # next step size
    np.testing.assert_allclose(r.y[:, 0], [float(v) for v in ref["y"]], rtol=REL, atol=1e-300)


@pytest.mark.parametrize("h0", [0.075, 0.03])
@pytest.mark.parametrize("K", [1, 2, 3])
def test_rkck_growth_rule_branches(h0, K):
    # a carried first step size puts the first error estimate on either side
    # of ERRCON = 1.89e-4: ~6e-4 (growth 0.9 err^(-1/5) ~ 4.0) and ~6e-6
    # (growth capped at 5)
    A, y0, rtol, atol = [[-1.0, 1.0], [0.0, -1.0]], [1.0, 0.3], 1e-6, 1e-9
    ref = rkck_restated(A, y0, 0.0, 1.0, rtol, atol, K, h0=h0)
    first = float(ref["trace"][0][1])
    assert (1.89e-4 < first < 1.89e-3) if h0 == 0.075 else (first < 1.89e-4), first
    carry = [1.0, 0.0, h0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    r = run_linear(A, y0, 0.0, 1.0, rtol, atol, 0, K, carry=carry)
    assert (int(r.n_accept[0]), int(r.n_reject[0])) == (ref["acc"], ref["rej"]), ref["trace"]
    c = r.carry[:, 0]
    assert c[1] == pytest.approx(float(ref["t"]), rel=REL)
    assert c[2] == pytest.approx(float(ref["h"]), rel=REL)
    np.testing.assert_allclose(r.y[:, 0], [float(v) for v in ref["y"]], rtol=REL)


def test_rkck_runs_include_rejections():
    for A, y0, rtol, atol in RKCK_CASES.values():
        ref = rkck_restated(A, y0, 0.0, 1.0, rtol, atol, 5)
        assert ref["rej"] >= 1 and ref["acc"] >= 2, ref["trace"]


# ------------------------------------------------------------------- RKC

def cheb(m, x):
    """T_m(x), T_m'(x), T_m''(x) at x != +-1."""
    T = mpmath.chebyt(m, x)
    Tp = m * mpmath.chebyu(m - 1, x)
    Tpp = m * ((m + 1) * T - mpmath.chebyu(m, x)) / (x * x - 1)
    return T, Tp, Tpp


def rkc_poly_factory(m):
    w0 = 1 + mpmath.mpf(2) / 13 / (m * m)
    T, Tp, Tpp = cheb(m, w0)
    w1 = Tp / Tpp
    b = Tpp / (Tp * Tp)
    a = 1 - b * T
    return lambda z: a + b * mpmath.chebyt(m, w0 + w1 * z)


def sym_matrix(lams, theta):
    c, s = np.cos(theta), np.sin(theta)
    Q = np.array([[c, -s], [s, c]])
    return Q @ np.diag(lams) @ Q.T, Q


def rkc_restated(lams, theta, y0, t0, tend, rtol, atol, K, carry=None):
    """Section 2.2's adaptive RKC (rkcDriver control flow, readings R4, R6,
    R9) on y' = A y, A = Q diag(lams) Q^T, sigma from the Gershgorin bound,
    for K attempts."""
    mp.dps = 50
    A, Q = sym_matrix(lams, theta)
    Am = mpmat(A)
    Qm = mpmat(Q)
    lm = [mpmath.mpf(float(v)) for v in lams]
    rtol, atol = mpmath.mpf(rtol), mpmath.mpf(atol)
    n = 2
    y = mpmath.matrix([mpmath.mpf(float(v)) for v in y0])
    t, tend = mpmath.mpf(t0), mpmath.mpf(tend)
    mmax = max(2, int(mpmath.nint(mpmath.sqrt(rtol / (10 * UROUND)))))
    hmax = abs(tend - t)
    hmin = 10 * UROUND * max(abs(t), hmax)
    # Gershgorin: the largest absolute row sum of the (constant) Jacobian,
    # summed in double as the bound is defined on the FP64 Jacobian
    G = mpmath.mpf(float(max(abs(A[i, 0]) + abs(A[i, 1]) for i in range(2))))
    F = Am * y
    err_old = h_old = h = mpmath.mpf(0)
    num_step, sr_step, sigma, rejected = 0, -1, None, False
    n_rhs = 1
    if carry is not None:   # the controller and the spectral-radius schedule resume (reading R21)
        h, sigma, h_old, err_old = (mpmath.mpf(float(v)) for v in (carry[2], carry[3], carry[4], carry[5]))
        num_step, sr_step, rejected = int(carry[6]), int(carry[7]), bool(carry[8])
    acc = rej = 0
    trace = []
    for _ in range(K):
        if not t < tend:
            break
        if 1.1 * h >= abs(tend - t):
            h = abs(tend - t)
        # once per need (reading R4): no estimate yet, after a rejection, or
        # every 25 accepted steps
        if sigma is None or rejected or (num_step % 25 == 0 and sr_step != num_step):
            sigma, sr_step = G, num_step
        if h < UROUND:   # initial step: Euler trial of size 1/sigma
            h = hmax
            if sigma * h > 1:
                h = 1 / sigma
            h = max(h, hmin)
            fz = Am * (y + h * F)
            n_rhs += 1
            est = h * mpmath.sqrt(sum(((fz[i] - F[i]) / (atol + rtol * abs(y[i]))) ** 2 for i in range(n)) / n)
            h = max(mpmath.mpf("0.1") * h / mpmath.sqrt(est), hmin) if mpmath.mpf("0.1") * h < hmax * mpmath.sqrt(est) else hmax
        m = 1 + int(mpmath.floor(mpmath.sqrt(mpmath.mpf("1.54") * h * sigma + 1)))
        if m > mmax:
            m = mmax
            h = mpmath.mpf(m * m - 1) / (mpmath.mpf("1.54") * sigma)
        P = rkc_poly_factory(m)
        Pm = Qm * mpmath.diag([P(h * lam) for lam in lm]) * Qm.T
        ynew = Pm * y
        Fnew = Am * ynew
        n_rhs += m
        err = mpmath.sqrt(sum(((mpmath.mpf("0.8") * (y[i] - ynew[i]) + mpmath.mpf("0.4") * h * (F[i] + Fnew[i]))
                               / (atol + rtol * max(abs(ynew[i]), abs(y[i])))) ** 2 for i in range(n)) / n)
        if err > 1:   # rejection: h = 0.8 h / err^(1/3), unclamped (reading R6)
            rej += 1
            h = mpmath.mpf("0.8") * h / mpmath.cbrt(err)
            rejected = True
            trace.append(("reject", m, err))
            continue
        acc += 1
        rejected = False
        t = t + h
        num_step += 1
        fac = mpmath.mpf(10)
        if h_old < UROUND:   # first accepted step
            t2 = mpmath.cbrt(err)
            if mpmath.mpf("0.8") < fac * t2:
                fac = mpmath.mpf("0.8") / t2
        else:                # Eqs. dtnp1 / rkc-f: the ratio of two error-per-step estimates
            t1 = mpmath.mpf("0.8") * h * mpmath.cbrt(err_old)
            t2 = h_old * err ** (mpmath.mpf(2) / 3)
            if t1 < fac * t2:
                fac = t1 / t2
        err_old, h_old = err, h
        y, F = ynew, Fnew
        h = h * max(mpmath.mpf("0.1"), fac)
        h = max(hmin, min(hmax, h))
        trace.append(("accept", m, err))
    return dict(t=t, h=h, y=y, acc=acc, rej=rej, h_old=h_old, err_old=err_old, num_step=num_step, n_rhs=n_rhs,
                trace=trace)


def check_rkc(lams, theta, y0, tend, rtol, atol, K, carry=None, controller=True):
    """Decisions and counts always; the controller's step sizes and error
    estimates too unless the estimate is dominated by FP64 rounding
    (hundreds of stages), where only the noise-robust decisions count."""
    A, _ = sym_matrix(lams, theta)
    ref = rkc_restated(lams, theta, y0, 0.0, tend, rtol, atol, K, carry=carry)
    r = run_linear(A, y0, 0.0, tend, rtol, atol, 1, K, specrad=O.SPECRAD_GERSHGORIN, carry=carry)
    assert (int(r.n_accept[0]), int(r.n_reject[0])) == (ref["acc"], ref["rej"]), ref["trace"]
    assert int(r.n_specrad_iter[0]) == 0
    assert int(r.n_rhs[0]) == ref["n_rhs"], ref["trace"]   # F0, the trial, m per attempt
    c = r.carry[:, 0]
    assert c[1] == pytest.approx(float(ref["t"]), rel=REL, abs=1e-300)
    if not controller:
        np.testing.assert_allclose(r.y[:, 0], [float(v) for v in ref["y"]], rtol=1e-9)
        return ref
    assert c[2] == pytest.approx(float(ref["h"]), rel=REL)
    assert c[4] == pytest.approx(float(ref["h_old"]), rel=REL, abs=1e-300)
    assert c[5] == pytest.approx(float(ref["err_old"]), rel=REL, abs=ERR_ABS)
    assert int(c[6]) == ref["num_step"]
    np.testing.assert_allclose(r.y[:, 0], [float(v) for v in ref["y"]], rtol=REL, atol=1e-300)
    return ref


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_rkc_cold_start_decisions(K):
    # cold start: the initial-step rule, then Eq. rkc-f's first-step factor
    # and the dtnp1 / rkc-f ratio; the stiff mode sets m
    check_rkc([-2000.0, -1.5], 0.3, [1.0, 0.7], 1.0, 1e-6, 1e-9, K)


@pytest.mark.parametrize("K", [1, 2])
@pytest.mark.parametrize("scale", [0.7, 1.5])
def test_rkc_initial_step_branch(K, scale):
    # for f = A y the Euler trial gives est = h^2 q, q the RMS of
    # A^2 y / (atol + rtol |y|), so the rule picks 0.1 / sqrt(q) when that is
    # below hmax and hmax otherwise: an interval of 0.7 or 1.5 times
    # 0.1 / sqrt(q) lands on either side of the test
    lams, theta, y0 = [-2000.0, -1.5], 0.3, np.array([1.0, 0.7])
    A, _ = sym_matrix(lams, theta)
    q = np.sqrt(np.mean((A @ A @ y0 / (1e-9 + 1e-6 * np.abs(y0))) ** 2))
    tend = scale * 0.1 / np.sqrt(q)
    check_rkc(lams, theta, list(y0), tend, 1e-6, 1e-9, K)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_rkc_warm_start_with_forced_rejection(K):
    # a carried step size far too large for the accuracy: the first attempt
    # is rejected (h = 0.8 h / err^(1/3)); later steps use err_old / h_old
    lams, theta = [-500.0, -0.8], 1.1
    A, _ = sym_matrix(lams, theta)
    G = max(abs(A[0, 0]) + abs(A[0, 1]), abs(A[1, 0]) + abs(A[1, 1]))
    v = [1.0, 0.0]
    carry = [1.0, 0.0, 0.4, G, 0.2, 0.5, 3, 3, 0.0] + v
    ref = check_rkc(lams, theta, [1.0, -0.4], 2.0, 1e-6, 1e-9, K, carry=carry)
    assert ref["trace"][0][0] == "reject"


@pytest.mark.parametrize("K", [2, 3, 4])
def test_rkc_first_accepted_step_factor(K):
    # a carry with h_old = 0 (no accepted step yet): the carried step is
    # rejected, the next one accepted with err ~0.5, where Eq. rkc-f's
    # first-step branch gives fac = 0.8 / err^(1/3) < 10; then the
    # h_old / err_old ratio
    lams, theta = [-300.0, -0.5], 0.4
    A, _ = sym_matrix(lams, theta)
    G = max(abs(A[0, 0]) + abs(A[0, 1]), abs(A[1, 0]) + abs(A[1, 1]))
    carry = [1.0, 0.0, 2e-3, G, 0.0, 0.0, 3, 3, 0.0, 1.0, 0.0]
    ref = check_rkc(lams, theta, [1.0, 0.2], 1.0, 1e-6, 1e-9, K, carry=carry)
    first = next(tr for tr in ref["trace"] if tr[0] == "accept")
    assert 7.3e-4 < float(first[2]) < 1.0, ref["trace"]


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_rkc_stage_cap(K):
    # rtol 1e-9 gives m_max = round(sqrt(450.45)) = 671.  A carried spectral
    # radius of 1e9 (kept: no rejection, no 25-step re-estimate in K steps)
    # asks for m ~ 1240 at the carried h and for more after each accepted
    # step (the slow modes keep err ~ 6e-3, so h grows), so every step takes
    # m = 671 and h = (671^2 - 1) / (1.54 sigma).  With 671 stages the FP64
    # error estimate is dominated by rounding: only the decisions, the
    # stage counts and the capped step sizes are compared.
    lams, theta = [-1.0, -2.0], 0.7
    carry = [1.0, 0.0, 1e-2, 1e9, 1e-12, 0.5, 3, 3, 0.0, 1.0, 0.0]
    ref = check_rkc(lams, theta, [1.0, 0.5], 1.0, 1e-9, 1e-12, K, carry=carry, controller=False)
    assert all(tr[1] == 671 for tr in ref["trace"]) and ref["acc"] == K, ref["trace"]
    assert float(ref["t"]) == pytest.approx(K * (671.0 ** 2 - 1) / (1.54 * 1e9), rel=1e-14)


def test_rkc_runs_include_rejections_and_both_factor_rules():
    cold = rkc_restated([-2000.0, -1.5], 0.3, [1.0, 0.7], 0.0, 1.0, 1e-6, 1e-9, 5)
    assert cold["acc"] >= 2
    lams, theta = [-500.0, -0.8], 1.1
    A, _ = sym_matrix(lams, theta)
    G = max(abs(A[0, 0]) + abs(A[0, 1]), abs(A[1, 0]) + abs(A[1, 1]))
    warm = rkc_restated(lams, theta, [1.0, -0.4], 0.0, 2.0, 1e-6, 1e-9, 5,
                        carry=[1.0, 0.0, 0.4, G, 0.2, 0.5, 3, 3, 0.0, 1.0, 0.0])
    assert warm["rej"] >= 1 and warm["acc"] >= 2, warm["trace"]


# -------------------------------------------- RKC on a nonlinear system

def rkc_stage_coefficients(m):
    """mu~_1 and (mu_j, nu_j, mu~_j, gamma~_j), j = 2..m, from Section 2.2's
    formulas: b_j = T_j''(w0) / T_j'(w0)^2 (j >= 2), b_0 = b_1 = b_2
    (reading R3), a_j = 1 - b_j T_j(w0), mu~_1 = b_1 w1, mu_j = 2 b_j w0 /
    b_{j-1}, nu_j = -b_j / b_{j-2}, mu~_j = 2 b_j w1 / b_{j-1},
    gamma~_j = -a_{j-1} mu~_j."""
    w0 = 1 + mpmath.mpf(2) / 13 / (m * m)
    _, Tpm, Tppm = cheb(m, w0)
    w1 = Tpm / Tppm
    b, a = {}, {}
    for j in range(2, m + 1):
        T, Tp, Tpp = cheb(j, w0)
        b[j] = Tpp / (Tp * Tp)
        a[j] = 1 - b[j] * T
    b[0] = b[1] = b[2]
    a[1] = 1 - b[1] * w0
    mut1 = b[1] * w1
    stages = [(2 * b[j] * w0 / b[j - 1], -b[j] / b[j - 2], 2 * b[j] * w1 / b[j - 1],
               -a[j - 1] * (2 * b[j] * w1 / b[j - 1])) for j in range(2, m + 1)]
    return mut1, stages


def vdp_restated_rkc(mu, y0, tend, rtol, atol, K):
    """RKC on van der Pol (y1' = y2, y2' = mu (1 - y1^2) y2 - y1) for K
    attempts, sigma from the Gershgorin bound of the analytic Jacobian,
    stages by the recurrence of Eqs. E:rkc0-E:rkcs."""
    mp.dps = 50
    mu = mpmath.mpf(mu)
    rtol, atol = mpmath.mpf(rtol), mpmath.mpf(atol)

    def f(y):
        return [y[1], mu * (1 - y[0] ** 2) * y[1] - y[0]]

    def gersh(y):
        return max(mpmath.mpf(1), abs(mu * (-2 * y[0]) * y[1] - 1) + abs(mu * (1 - y[0] ** 2)))

    y = [mpmath.mpf(float(v)) for v in y0]
    t, tend = mpmath.mpf(0), mpmath.mpf(tend)
    mmax = max(2, int(mpmath.nint(mpmath.sqrt(rtol / (10 * UROUND)))))
    hmax, hmin = tend, 10 * UROUND * tend
    F = f(y)
    n_rhs, h, h_old, err_old = 1, mpmath.mpf(0), mpmath.mpf(0), mpmath.mpf(0)
    num_step, sr_step, sigma, rejected = 0, -1, None, False
    acc = rej = 0
    trace = []
    for _ in range(K):
        if 1.1 * h >= abs(tend - t):
            h = abs(tend - t)
        if sigma is None or rejected or (num_step % 25 == 0 and sr_step != num_step):
            sigma, sr_step = gersh(y), num_step
        if h < UROUND:   # initial step: an Euler trial of size 1/sigma
            h = hmax
            if sigma * h > 1:
                h = 1 / sigma
            h = max(h, hmin)
            fz = f([y[i] + h * F[i] for i in range(2)])
            n_rhs += 1
            est = h * mpmath.sqrt(sum(((fz[i] - F[i]) / (atol + rtol * abs(y[i]))) ** 2 for i in range(2)) / 2)
            h = max(mpmath.mpf("0.1") * h / mpmath.sqrt(est), hmin) if mpmath.mpf("0.1") * h < hmax * mpmath.sqrt(est) else hmax
        m = 1 + int(mpmath.floor(mpmath.sqrt(mpmath.mpf("1.54") * h * sigma + 1)))
        if m > mmax:
            m = mmax
            h = mpmath.mpf(m * m - 1) / (mpmath.mpf("1.54") * sigma)
        mut1, stages = rkc_stage_coefficients(m)
        w2, w1 = y, [y[i] + mut1 * h * F[i] for i in range(2)]
        for (muj, nuj, mutj, gtj) in stages:
            fj = f(w1)
            wj = [(1 - muj - nuj) * y[i] + muj * w1[i] + nuj * w2[i] + mutj * h * fj[i] + gtj * h * F[i]
                  for i in range(2)]
            w2, w1 = w1, wj
        ynew = w1
        Fnew = f(ynew)
        n_rhs += m
        err = mpmath.sqrt(sum(((mpmath.mpf("0.8") * (y[i] - ynew[i]) + mpmath.mpf("0.4") * h * (F[i] + Fnew[i]))
                               / (atol + rtol * max(abs(ynew[i]), abs(y[i])))) ** 2 for i in range(2)) / 2)
        if err > 1:
            rej += 1
            rejected = True
            h = mpmath.mpf("0.8") * h / mpmath.cbrt(err)
            trace.append(("reject", m, err))
            continue
        acc += 1
        rejected = False
        t += h
        num_step += 1
        fac = mpmath.mpf(10)
        if h_old < UROUND:
            t2 = mpmath.cbrt(err)
            if mpmath.mpf("0.8") < fac * t2:
                fac = mpmath.mpf("0.8") / t2
        else:
            t1 = mpmath.mpf("0.8") * h * mpmath.cbrt(err_old)
            t2 = h_old * err ** (mpmath.mpf(2) / 3)
            if t1 < fac * t2:
                fac = t1 / t2
        err_old, h_old = err, h
        y, F = ynew, Fnew
        h = max(hmin, min(hmax, h * max(mpmath.mpf("0.1"), fac)))
        trace.append(("accept", m, err))
    return dict(t=t, h=h, y=y, acc=acc, rej=rej, h_old=h_old, err_old=err_old, n_rhs=n_rhs, trace=trace)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_rkc_nonlinear_start_decisions(K):
    # van der Pol at mu = 8 from (1.5, 3): the Euler trial of size 1/sigma
    # sees the nonlinearity, so the initial-step rule's result depends on
    # the trial size (for a linear f it would not)
    mu, y0, tend, rtol, atol = 8.0, [1.5, 3.0], 20.0, 1e-6, 1e-9
    ref = vdp_restated_rkc(mu, y0, tend, rtol, atol, K)
    r = O.integrate(O.model(O.KIND_VDP, 2, 1), 1, np.array(y0).reshape(2, 1), np.array([[mu]]), 0.0, tend,
                    rtol, atol, max_attempts=K, nthreads=1, carry_out=True, specrad=O.SPECRAD_GERSHGORIN)
    assert (int(r.n_accept[0]), int(r.n_reject[0])) == (ref["acc"], ref["rej"]), ref["trace"]
    assert int(r.n_rhs[0]) == ref["n_rhs"], ref["trace"]
    c = r.carry[:, 0]
    # the first accepted estimate is ~1e-6 (FP64 carries it to ~1e-4
    # relative) and enters the next step size as err_old^(1/3): step sizes
    # and later estimates agree to REL_NL after it, decisions exactly
    assert c[1] == pytest.approx(float(ref["t"]), rel=REL_NL, abs=1e-300)
    assert c[2] == pytest.approx(float(ref["h"]), rel=REL_NL)
    assert c[5] == pytest.approx(float(ref["err_old"]), rel=REL_NL, abs=ERR_ABS)
    np.testing.assert_allclose(r.y[:, 0], [float(v) for v in ref["y"]], rtol=REL_NL)


def test_rkc_nonlinear_start_depends_on_the_trial_size():
    # the check above would see a different trial size: the first step size
    # moves by far more than REL when the trial is 1 / (2 sigma)
    mp.dps = 50
    mu, y0, rtol, atol = mpmath.mpf(8), [mpmath.mpf("1.5"), mpmath.mpf(3)], mpmath.mpf("1e-6"), mpmath.mpf("1e-9")

    def f(y):
        return [y[1], mu * (1 - y[0] ** 2) * y[1] - y[0]]

    F = f(y0)
    sigma = max(mpmath.mpf(1), abs(mu * (-2 * y0[0]) * y0[1] - 1) + abs(mu * (1 - y0[0] ** 2)))

    def first_h(h):
        fz = f([y0[i] + h * F[i] for i in range(2)])
        est = h * mpmath.sqrt(sum(((fz[i] - F[i]) / (atol + rtol * abs(y0[i]))) ** 2 for i in range(2)) / 2)
        return mpmath.mpf("0.1") * h / mpmath.sqrt(est)

    assert abs(first_h(1 / sigma) / first_h(1 / (2 * sigma)) - 1) > 10 * REL_NL

