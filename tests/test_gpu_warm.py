"""Warm restart across calls (the outer global-step loop of Section 3) on the
GPU against the oracle's.

The plain FP64 form must reproduce the oracle's chain of global steps bit
for bit -- final states, counters and the carried controller state,
eigenvector included -- on every system whose step sequence matches (at
least 99.9 %).  The lean form follows the oracle's warm chain within the
mixed-form error bound and saves the start-up evaluations of every global
step after the first.  Both carry modes are checked: CONTINUE (the exact
continuation) and RESTART (spectral-radius schedule started again each
call).  Mapping, cost order and the mapping-timing runs do not touch the
carry.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

from gpu_util import rel_err

pytestmark = pytest.mark.gpu

RKCK, RKC = 0, 1


def gpu_chain(w, method, precision, edges, warm, mapping=B.ODE_MAP_THREAD, order_by_rhs=False,
              mode=B.ODE_CARRY_CONTINUE):
    import torch
    h = B.register_workload(w)
    try:
        y = torch.from_numpy(np.ascontiguousarray(w.y0)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(w.params)).cuda()
        carry = B.carry_like(w.neq, w.nsys)
        tot = {k: np.zeros(w.nsys, np.int64) for k in ("n_accept", "n_reject", "n_rhs")}
        status = np.zeros(w.nsys, np.int32)
        cost = None
        for t_a, t_b in zip(edges[:-1], edges[1:]):
            cnt = B.counters_like(w.nsys, "cuda")
            if not warm:
                carry.zero_()
            y = B.integrate("rkck" if method == RKCK else "rkc", h, y, p, float(t_a), float(t_b), w.rtol, w.atol,
                            y_out=y, counters=cnt, precision=precision, mapping=mapping, carry=carry,
                            carry_mode=mode, cost=cost, sync=True)
            for k in tot:
                tot[k] += getattr(cnt, k).cpu().numpy()
            status |= cnt.status.cpu().numpy()
            if order_by_rhs:
                cost = cnt.n_rhs             # int32 counters order the next call
        return y.cpu().numpy(), tot, status, carry.cpu().numpy()
    finally:
        B.release(h)


def oracle_chain(w, method, edges, warm, mode=O.CARRY_CONTINUE):
    m = O.model_for(w)
    y, carry = w.y0.copy(), None
    tot = {k: np.zeros(w.nsys, np.int64) for k in ("n_accept", "n_reject", "n_rhs")}
    for t_a, t_b in zip(edges[:-1], edges[1:]):
        r = O.integrate(m, method, y, w.params, float(t_a), float(t_b), w.rtol, w.atol,
                        carry_in=carry if warm else None, carry_out=True, carry_mode=mode)
        y, carry = r.y, r.carry
        for k in tot:
            tot[k] += getattr(r, k)
    return y, tot, carry


@pytest.mark.parametrize("warm,mode", [(True, 0), (True, 1), (False, 0)])
def test_fp64_rkc_chain_reproduces_oracle(warm, mode):
    w = W.massaction(1500, seed=12)
    edges = np.linspace(w.t0, w.tend, 6)
    yg, tg, _, cg = gpu_chain(w, RKC, B.ODE_PREC_FP64, edges, warm, mode=mode)
    yo, to, co = oracle_chain(w, RKC, edges, warm, mode=mode)
    same = (tg["n_accept"] == to["n_accept"]) & (tg["n_reject"] == to["n_reject"])
    assert same.mean() >= 0.999
    np.testing.assert_array_equal(tg["n_rhs"][same], to["n_rhs"][same])
    assert rel_err(yg, yo, w.atol)[same].max() <= 1e-9
    if warm:
        # the carried state: flag, time, h, sigma, h_old, err_old, counts, eigenvector
        np.testing.assert_array_equal(cg[:, same], co[:, same])


def test_fp64_rkck_chain_reproduces_oracle():
    w = W.vdp(3000, seed=14)
    edges = np.linspace(w.t0, w.tend, 5)
    yg, tg, _, cg = gpu_chain(w, RKCK, B.ODE_PREC_FP64, edges, True)
    yo, to, co = oracle_chain(w, RKCK, edges, True)
    same = (tg["n_accept"] == to["n_accept"]) & (tg["n_reject"] == to["n_reject"])
    assert same.mean() >= 0.999
    assert rel_err(yg, yo, w.atol)[same].max() <= 1e-9
    np.testing.assert_array_equal(cg[:, same], co[:, same])


@pytest.mark.parametrize("mode", [B.ODE_CARRY_CONTINUE, B.ODE_CARRY_RESTART])
def test_lean_warm_chain_against_oracle_and_cold(mode):
    w = W.massaction(4000, seed=15)
    edges = np.linspace(w.t0, w.tend, 11)
    yw, tw, sw, cw = gpu_chain(w, RKC, B.ODE_PREC_MIXED_LEAN, edges, True, mode=mode)
    yc, tc, sc, _ = gpu_chain(w, RKC, B.ODE_PREC_MIXED_LEAN, edges, False)
    yo, to, _ = oracle_chain(w, RKC, edges, True, mode=mode)
    assert ((sw & 0xFF) == 0).all() and ((sc & 0xFF) == 0).all()
    e = rel_err(yw, yo, w.atol)
    print("lean warm chain (mode", mode, ") vs oracle: p99.9", np.quantile(e, 0.999), "median", np.median(e),
          "mean n_rhs warm", tw["n_rhs"].mean(), "cold", tc["n_rhs"].mean())
    assert np.quantile(e, 0.999) < 1e-4
    assert np.all(cw[0] == 1.0) and np.allclose(cw[1], w.tend, rtol=0, atol=1e-12 * w.tend)
    # the power method and the trial step are skipped after the first global step
    assert tw["n_rhs"].sum() < tc["n_rhs"].sum()


def test_carry_survives_mapping_order_and_tuning():
    # >= 32768 systems: ODE_MAP_AUTO times its candidates on the first call;
    # the order of the later calls comes from the previous call's counters
    w = W.vdp(40000, seed=16)
    edges = np.linspace(w.t0, w.tend, 4)
    ref = gpu_chain(w, RKC, B.ODE_PREC_MIXED_LEAN, edges, True, mapping=B.ODE_MAP_THREAD)
    for mapping, order in ((B.ODE_MAP_AUTO, True), (B.ODE_MAP_QUEUE, False)):
        got = gpu_chain(w, RKC, B.ODE_PREC_MIXED_LEAN, edges, True, mapping=mapping, order_by_rhs=order)
        np.testing.assert_array_equal(got[0], ref[0])
        for k in ref[1]:
            np.testing.assert_array_equal(got[1][k], ref[1][k], err_msg=k)
        np.testing.assert_array_equal(got[3], ref[3])
