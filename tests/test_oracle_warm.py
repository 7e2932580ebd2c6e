"""Pins of the oracle's warm restart (the outer global-step loop of Section 3
with the controller state carried from one call to the next).

The defining property: a run stopped by the attempt cap and continued from
the time it reached with the carried state repeats the uninterrupted run
step for step, so the final states agree bit for bit and the accepted /
rejected counts add up.  (The per-call quantities hmax = |tend - t0| and
hmin do not bind on these stiff workloads.)  A cold carry (flag 0) is no
carry at all.  Carry mode RESTART is the continuation with the
spectral-radius schedule started again.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import workloads as W

RKCK, RKC = 0, 1


def one(w, i):
    """System i of a workload, as a one-system batch."""
    return W.subset(w, np.array([i]))


def split_run(m, method, w1, K):
    """Stop after K attempts, then continue to tend from the time reached."""
    a = O.integrate(m, method, w1.y0, w1.params, w1.t0, w1.tend, w1.rtol, w1.atol,
                    max_attempts=K, nthreads=1, carry_out=True)
    t_k = float(a.carry[1, 0])
    b = O.integrate(m, method, a.y, w1.params, t_k, w1.tend, w1.rtol, w1.atol,
                    nthreads=1, carry_in=a.carry, carry_out=True)
    return a, b


@pytest.mark.parametrize("K", [1, 2, 24, 25, 26, 60])
def test_rkc_split_run_repeats_the_uninterrupted_run(K):
    w = W.massaction(12, seed=21)
    m = O.model_for(w)
    for i in range(w.nsys):
        w1 = one(w, i)
        full = O.integrate(m, RKC, w1.y0, w1.params, w1.t0, w1.tend, w1.rtol, w1.atol, nthreads=1,
                           carry_out=True)
        a, b = split_run(m, RKC, w1, K)
        assert a.status[0] & 0xFF == O.ST_MAX_ATTEMPTS and a.carry[0, 0] == 1.0
        assert 0.0 < a.carry[1, 0] < w1.tend
        np.testing.assert_array_equal(b.y, full.y)
        assert a.n_accept[0] + b.n_accept[0] == full.n_accept[0]
        assert a.n_reject[0] + b.n_reject[0] == full.n_reject[0]
        # the same power-method iterations, plus F(t, y) evaluated again at the restart
        assert a.n_specrad_iter[0] + b.n_specrad_iter[0] == full.n_specrad_iter[0]
        assert a.n_rhs[0] + b.n_rhs[0] == full.n_rhs[0] + 1
        # and it ends in the same controller state
        np.testing.assert_array_equal(b.carry[2:, 0], full.carry[2:, 0])


@pytest.mark.parametrize("K", [1, 5, 40])
def test_rkck_split_run_repeats_the_uninterrupted_run(K):
    w = W.vdp(10, seed=8)
    m = O.model_for(w)
    for i in range(w.nsys):
        w1 = one(w, i)
        full = O.integrate(m, RKCK, w1.y0, w1.params, w1.t0, w1.tend, w1.rtol, w1.atol, nthreads=1,
                           carry_out=True)
        a, b = split_run(m, RKCK, w1, K)
        np.testing.assert_array_equal(b.y, full.y)
        assert a.n_accept[0] + b.n_accept[0] == full.n_accept[0]
        assert a.n_reject[0] + b.n_reject[0] == full.n_reject[0]
        assert b.carry[2, 0] == full.carry[2, 0]


def test_cold_carry_is_no_carry():
    w = W.massaction(16, seed=3)
    m = O.model_for(w)
    cold = np.zeros((O.carry_words(w.neq), w.nsys))
    for method in (RKCK, RKC):
        r0 = O.integrate(m, method, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol)
        r1 = O.integrate(m, method, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol, carry_in=cold)
        np.testing.assert_array_equal(r0.y, r1.y)
        np.testing.assert_array_equal(r0.n_rhs, r1.n_rhs)


def test_carry_contents_after_a_cold_call():
    w = W.massaction(16, seed=5)
    m = O.model_for(w)
    r = O.integrate(m, RKC, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol, carry_out=True)
    c = r.carry
    assert np.all(c[0] == 1.0) and np.all(c[1] == w.tend)
    assert np.all(c[2] > 0) and np.all(c[3] > 0)                  # next h, sigma
    np.testing.assert_array_equal(c[6], r.n_accept)              # accepted steps of this call
    # the estimate is at most 25 accepted steps old (the one due at a multiple
    # of 25 is made at the next loop top, which a finished system never reaches)
    assert np.all(c[7] <= c[6]) and np.all(c[6] - c[7] <= 25)
    assert np.all(c[8] == 0)                                     # ended on an accepted step
    # h_old is the last accepted step, which landed on tend
    assert np.all(c[4] > 0) and np.all(c[4] <= w.tend)


def test_warm_chain_saves_the_start_up():
    # ten global steps over the same interval: warm restarts skip the power
    # method and the trial step at every global step after the first
    w = W.massaction(32, seed=9)
    m = O.model_for(w)
    edges = np.linspace(w.t0, w.tend, 11)
    runs = {}
    for warm in (False, True):
        y, carry, rhs = w.y0.copy(), None, np.zeros(w.nsys)
        for t_a, t_b in zip(edges[:-1], edges[1:]):
            r = O.integrate(m, RKC, y, w.params, t_a, t_b, w.rtol, w.atol, carry_in=carry, carry_out=True)
            y, rhs = r.y, rhs + r.n_rhs
            carry = r.carry if warm else None
        runs[warm] = (y, rhs)
    ref = O.integrate(m, RKC, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol)
    for warm, (y, rhs) in runs.items():
        e = np.abs(y - ref.y) / (np.abs(ref.y) + w.atol)
        assert e.max() < 5e-3, (warm, e.max())
    assert runs[True][1].sum() < runs[False][1].sum()


def test_restart_mode_is_continue_with_the_schedule_reset():
    w = W.massaction(24, seed=17)
    m = O.model_for(w)
    t1 = 0.4 * w.tend
    a = O.integrate(m, RKC, w.y0, w.params, w.t0, t1, w.rtol, w.atol, carry_out=True)
    c = a.carry.copy()
    r = O.integrate(m, RKC, a.y, w.params, t1, w.tend, w.rtol, w.atol, carry_in=c, carry_out=True,
                    carry_mode=O.CARRY_RESTART)
    c2 = c.copy()
    c2[6], c2[7], c2[8] = 0.0, -1.0, 0.0
    k = O.integrate(m, RKC, a.y, w.params, t1, w.tend, w.rtol, w.atol, carry_in=c2, carry_out=True,
                    carry_mode=O.CARRY_CONTINUE)
    np.testing.assert_array_equal(r.y, k.y)
    np.testing.assert_array_equal(r.n_rhs, k.n_rhs)
    np.testing.assert_array_equal(r.carry, k.carry)
    # the schedule restarted: sigma is estimated at the call start, from the carried eigenvector
    assert np.all(r.n_specrad_iter > 0)
    np.testing.assert_array_equal(r.carry[6], r.n_accept)
