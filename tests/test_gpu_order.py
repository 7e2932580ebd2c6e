"""Longest-first ordering of a batch by per-system cost estimates.

The order kernels are integer work: the result must be a permutation whose
cost classes (65535 steps of the float bit pattern between the smallest and
largest positive cost; NaN and values <= 0 form class 0) never increase,
with exactly the class counts a host histogram gives.  Which of several equal-class systems comes first is
not fixed, so only that is left unchecked.  Integrating through the order
must give bit for bit the results of the unordered call.
"""
import numpy as np
import pytest

from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def host_class(c):
    c = np.asarray(c, dtype=np.float32)
    pos = c > 0
    bits = c.view(np.uint32).astype(np.int64)
    if not pos.any():
        return np.zeros(c.size, dtype=np.int64)
    lo, hi = bits[pos].min(), bits[pos].max()
    return np.where(pos, 1 + (bits - lo) * 65535 // (hi - lo + 1), 0)


def check_order(cost_np):
    import torch
    cost = torch.from_numpy(cost_np.astype(np.float32)).cuda()
    idx = B.cost_order(cost).cpu().numpy().astype(np.int64)
    n = cost_np.size
    assert idx.shape == (n,)
    np.testing.assert_array_equal(np.sort(idx), np.arange(n))           # a permutation
    cls = host_class(cost_np)[idx]
    assert np.all(np.diff(cls) <= 0)                                     # longest first
    np.testing.assert_array_equal(np.bincount(cls, minlength=65536),
                                  np.bincount(host_class(cost_np), minlength=65536))


def test_host_classes_span_the_range():
    c = np.array([1.0, 2.0, 4.0, np.nan, 0.0], dtype=np.float32)
    np.testing.assert_array_equal(host_class(c), [1, 1 + 8388608 * 65535 // (16777216 + 1), 65535, 0, 0])


@pytest.mark.parametrize("n", [1, 31, 256, 100003])
def test_order_is_a_descending_permutation(n):
    rng = np.random.default_rng(n)
    c = np.exp(rng.normal(7.0, 1.0, size=n))
    check_order(c)


def test_order_special_values():
    c = np.array([np.nan, -1.0, 0.0, np.inf, 1e-30, 3.0, 3.0, 1e30, -np.inf, 2.0, np.nan] * 97)
    check_order(c)
    import torch
    idx = B.cost_order(torch.from_numpy(c.astype(np.float32)).cuda()).cpu().numpy()
    assert np.isinf(c[idx[0]]) and c[idx[0]] > 0                       # +inf is the most expensive


def test_order_all_nonpositive():
    check_order(np.array([0.0, -2.0, np.nan] * 50))


def test_int32_costs_order_like_their_float_values():
    import torch
    rng = np.random.default_rng(11)
    c = rng.integers(-5, 5000, size=70001).astype(np.int32)
    idx = B.cost_order(torch.from_numpy(c).cuda()).cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(np.sort(idx), np.arange(c.size))
    cls = host_class(c.astype(np.float32))
    assert np.all(np.diff(cls[idx]) <= 0)


def test_order_many_equal_costs():
    # heavy contention on a few classes (the scatter's aggregated atomics)
    rng = np.random.default_rng(5)
    c = rng.choice([10.0, 20.0, 40.0], size=300000)
    check_order(c)


def run(w, method, precision, mapping, cost=None):
    import torch
    h = B.register_workload(w)
    try:
        y0 = torch.from_numpy(np.ascontiguousarray(w.y0)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(w.params)).cuda()
        cnt = B.counters_like(w.nsys, "cuda")
        c = None if cost is None else torch.from_numpy(cost.astype(np.float32)).cuda()
        y = B.integrate(method, h, y0, p, w.t0, w.tend, w.rtol, w.atol, counters=cnt, precision=precision,
                        mapping=mapping, cost=c, sync=True)
        out = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "status")}
        out["y"] = y.cpu().numpy()
        return out
    finally:
        B.release(h)


@pytest.mark.parametrize("mapping", [B.ODE_MAP_THREAD, B.ODE_MAP_QUEUE, B.ODE_MAP_AUTO])
@pytest.mark.parametrize("case", ["vdp_rkck_f64", "mass_rkc_lean"])
def test_ordered_integration_is_bitwise_unchanged(case, mapping):
    if case == "vdp_rkck_f64":
        w, method, prec = W.vdp(40000, seed=2), "rkck", B.ODE_PREC_FP64
    else:
        w, method, prec = W.massaction(5000, seed=6), "rkc", B.ODE_PREC_MIXED_LEAN
    ref = run(w, method, prec, B.ODE_MAP_THREAD)
    # the true cost of the reference run, and a scrambled one
    for cost in (ref["n_rhs"].astype(np.float64), np.random.default_rng(1).permutation(ref["n_rhs"]) * 1.0):
        got = run(w, method, prec, mapping, cost=cost)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
