"""Constant-volume kinetics with a temperature equation (Section 4.2's form)
on the GPU against the oracle, on a synthetic 57-species, 766-reaction
mechanism.

Plain FP64: identical accepted / rejected counts on >= 99.9 % of systems
and final states within 1e-9 -- the rates through the series exponential,
omega summed per species in reaction order, the temperature equation's
sums in species order -- for one call and for the paper's chain of
10 global steps of 1e-6 s with warm restarts.  The mixed form follows the
oracle within the mixed-form bound and keeps sum_i Y_i = 1.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def gpu_chain(w, precision, edges, carry_mode=None, method="rkc"):
    import torch
    h = B.register_workload(w)
    try:
        y = torch.from_numpy(np.ascontiguousarray(w.y0)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(w.params)).cuda()
        carry = B.carry_like(w.neq, w.nsys) if carry_mode is not None else None
        tot = {k: np.zeros(w.nsys, np.int64) for k in ("n_accept", "n_reject", "n_rhs")}
        status = np.zeros(w.nsys, np.int32)
        for t_a, t_b in zip(edges[:-1], edges[1:]):
            cnt = B.counters_like(w.nsys, "cuda")
            y = B.integrate(method, h, y, p, float(t_a), float(t_b), w.rtol, w.atol, y_out=y, counters=cnt,
                            precision=precision, carry=carry, carry_mode=carry_mode or 0, sync=True)
            for k in tot:
                tot[k] += getattr(cnt, k).cpu().numpy()
            status |= cnt.status.cpu().numpy()
        return y.cpu().numpy(), tot, status
    finally:
        B.release(h)


def oracle_chain(w, edges, carry_mode=None, method=1):
    m = O.model_for(w)
    y, carry = w.y0.copy(), None
    tot = {k: np.zeros(w.nsys, np.int64) for k in ("n_accept", "n_reject", "n_rhs")}
    for t_a, t_b in zip(edges[:-1], edges[1:]):
        r = O.integrate(m, method, y, w.params, float(t_a), float(t_b), w.rtol, w.atol,
                        carry_in=carry if carry_mode is not None else None, carry_out=True,
                        carry_mode=carry_mode or 0)
        y, carry = r.y, r.carry
        for k in tot:
            tot[k] += getattr(r, k)
    return y, tot


def check_same(w, yg, tg, yo, to):
    same = (tg["n_accept"] == to["n_accept"]) & (tg["n_reject"] == to["n_reject"])
    assert same.mean() >= 0.999
    np.testing.assert_array_equal(tg["n_rhs"][same], to["n_rhs"][same])
    assert rel_err(yg, yo, w.atol)[same].max() <= 1e-9


def test_fp64_single_call_reproduces_oracle():
    w = W.kinetics(300, seed=21)
    edges = np.array([w.t0, w.tend])
    yg, tg, sg = gpu_chain(w, B.ODE_PREC_FP64, edges)
    yo, to = oracle_chain(w, edges)
    assert ((sg & 0xFF) == 0).all()
    check_same(w, yg, tg, yo, to)


@pytest.mark.parametrize("mode", [B.ODE_CARRY_CONTINUE, B.ODE_CARRY_RESTART])
def test_fp64_global_steps_with_warm_restart(mode):
    w = W.kinetics(200, seed=22)
    edges = np.linspace(0.0, 1e-5, 11)         # 10 global steps of 1e-6 s
    yg, tg, _ = gpu_chain(w, B.ODE_PREC_FP64, edges, carry_mode=mode)
    yo, to = oracle_chain(w, edges, carry_mode=mode)
    check_same(w, yg, tg, yo, to)


def test_fp64_rkck_reproduces_oracle():
    w = W.kinetics(120, seed=23, tend=2e-6)
    edges = np.array([w.t0, w.tend])
    yg, tg, _ = gpu_chain(w, B.ODE_PREC_FP64, edges, method="rkck")
    yo, to = oracle_chain(w, edges, method=0)
    check_same(w, yg, tg, yo, to)


def test_lean_against_oracle_and_invariants():
    w = W.kinetics(1000, seed=24)
    edges = np.array([w.t0, w.tend])
    yg, tg, sg = gpu_chain(w, B.ODE_PREC_MIXED_LEAN, edges)
    yo, _ = oracle_chain(w, edges)
    assert ((sg & 0xFF) == 0).all()
    e = rel_err(yg, yo, w.atol)
    # trace species (Y ~ 1e-8) carry FP32 rounding of the large rates that
    # feed them: judge the error in units of the solver's own tolerance
    e_tol = (np.abs(yg - yo) / (w.atol + w.rtol * np.abs(yo))).max(axis=0)
    print("kinetics lean: relative p99.9", np.quantile(e, 0.999), "median", np.median(e),
          "in tolerances p99.9", np.quantile(e_tol, 0.999), "max", e_tol.max(), "mean n_rhs", tg["n_rhs"].mean())
    assert np.median(e) < 1e-4
    assert np.quantile(e_tol, 0.999) < 100.0
    assert np.abs(yg[1:].sum(axis=0) - 1.0).max() < 1e-5
    # temperature within a fraction of a kelvin of the oracle's
    assert np.abs(yg[0] - yo[0]).max() < 0.5


def test_unsupported_spectral_bound_is_refused():
    import torch
    w = W.kinetics(4, seed=1)
    h = B.register_workload(w)
    try:
        with pytest.raises(B.BatchOdeError) as e:
            B.integrate("rkc", h, torch.from_numpy(w.y0).cuda(), torch.from_numpy(w.params).cuda(), w.t0, w.tend,
                        w.rtol, w.atol, specrad=B.ODE_SPECRAD_GERSHGORIN, sync=True)
        assert e.value.code == B.ODE_ERR_UNSUPPORTED
    finally:
        B.release(h)


def one_reaction_workload(nsys, seed):
    """A -> B with a constant rate (beta = Ea = 0), equal weights and constant
    heat capacities: Y_A = Y_A0 exp(-k t), and the heat of reaction warms
    the gas in proportion to the A converted (as in the oracle's pins)."""
    k, dh, Wt = 2.0e4, 3000.0, 0.03
    mech = W.Mechanism(2, np.array([[0, 1, 1, 0], [0, 1, 1, 0]]), np.array([Wt, Wt]),
                       np.array([[3.5, 0.0, 0.0, dh], [3.5, 0.0, 0.0, 0.0]]),
                       np.array([1], np.int32), np.array([[0, -1]], np.int32),
                       np.array([1], np.int32), np.array([[1, -1]], np.int32),
                       np.array([np.log10(k)]), np.array([0.0]), np.array([0.0]), kmin=1e-30, kmax=1e30)
    rng = np.random.default_rng(seed)
    ya = rng.uniform(0.5, 1.0, nsys)
    y0 = np.stack([rng.uniform(1000.0, 1500.0, nsys), ya, 1.0 - ya])
    rho = rng.uniform(0.2, 1.0, (1, nsys))
    w = W.Workload("kin_one", W.RHS_KINETICS, W.METHOD_RKC, nsys, 3, np.ascontiguousarray(y0), rho, 0.0, 1e-4,
                   1e-8, 1e-14, aux={"mechanism": mech})
    return w, k, dh, Wt


@pytest.mark.parametrize("method", ["rkc", "rkck"])
def test_single_reaction_mechanism(method):
    # two species, one single-reactant reaction: most lanes of each warp hold
    # nothing, and the rate-of-progress product takes the unit slot
    w, k, dh, Wt = one_reaction_workload(256, seed=25)
    edges = np.array([w.t0, w.tend])
    mid = 1 if method == "rkc" else 0
    yg, tg, sg = gpu_chain(w, B.ODE_PREC_FP64, edges, method=method)
    yo, to = oracle_chain(w, edges, method=mid)
    assert ((sg & 0xFF) == 0).all()
    check_same(w, yg, tg, yo, to)
    ya = w.y0[1] * np.exp(-k * w.tend)
    T = w.y0[0] + dh * (w.y0[1] - ya) / (3.5 - 1.0)   # (R/W) dh dY / ((R/W)(3.5 - 1))
    tol = 1e-6 if method == "rkck" else 1e-4
    np.testing.assert_allclose(yg[1], ya, rtol=tol)
    np.testing.assert_allclose(yg[0], T, rtol=tol)
    yl, _, sl = gpu_chain(w, B.ODE_PREC_MIXED_LEAN, edges, method=method)
    assert ((sl & 0xFF) == 0).all()
    np.testing.assert_allclose(yl[1], ya, rtol=1e-3)
    np.testing.assert_allclose(yl[1:].sum(axis=0), 1.0, rtol=1e-5)
