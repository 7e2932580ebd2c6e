"""The mapping of systems onto the GPU changes where each system runs, not
what it computes: every mapping gives the same final states and counters
bit for bit.  ODE_MAP_AUTO on a batch large enough to trigger the mapping
timing runs (which integrate a sample of the batch first) must leave the
result untouched, also when the call integrates in place."""
import numpy as np
import pytest

from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TUNE_MIN = 32768  # batches from this size on are timed under ODE_MAP_AUTO


def run(w, method, precision, mapping, in_place=False, block_size=0):
    import torch
    h = B.register_workload(w)   # a fresh handle: AUTO times its mappings again
    try:
        y0 = torch.from_numpy(np.ascontiguousarray(w.y0)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(w.params)).cuda()
        cnt = B.counters_like(w.nsys, "cuda")
        y_out = y0 if in_place else None
        y = B.integrate(method, h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=y_out, counters=cnt,
                        precision=precision, mapping=mapping, block_size=block_size, sync=True)
        out = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "status")}
        out["y"] = y.cpu().numpy()
        return out
    finally:
        B.release(h)


def assert_same(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("precision", [B.ODE_PREC_FP64, B.ODE_PREC_MIXED_LEAN])
def test_vdp_mappings_agree_bitwise(precision):
    w = W.vdp(TUNE_MIN + 1234, seed=11)
    ref = run(w, "rkck", precision, B.ODE_MAP_THREAD)
    for mapping, bs in ((B.ODE_MAP_QUEUE, 0), (B.ODE_MAP_THREAD, 64), (B.ODE_MAP_AUTO, 0), (B.ODE_MAP_AUTO, 96)):
        assert_same(run(w, "rkck", precision, mapping, block_size=bs), ref)


def test_auto_tuning_in_place_keeps_initial_states():
    # the timing runs must not write the sample's results over y0
    w = W.massaction(TUNE_MIN + 100, seed=4)
    w.tend = 2e-5   # a short interval keeps the plain FP64 runs quick
    ref = run(w, "rkc", B.ODE_PREC_FP64, B.ODE_MAP_THREAD)
    got = run(w, "rkc", B.ODE_PREC_FP64, B.ODE_MAP_AUTO, in_place=True)
    assert_same(got, ref)


def test_ragged_plan_in_place_tuning():
    import torch
    from test_gpu_ragged import build_plan
    b = W.mixed(nsys=3000, seed=9)
    b.tend = np.where(b.kind == B.ODE_RHS_BRUSS1D, 0.5, 1.0)
    outs = []
    for in_place in (False, True):
        B.tuning_reset()   # both plans time their candidates
        plan, y, cnt, hs = build_plan(b, B.ODE_PREC_MIXED_LEAN, B.ODE_MAP_AUTO, in_place=in_place)
        plan.launch()
        torch.cuda.synchronize()
        outs.append((y.cpu().numpy(), cnt.n_accept.cpu().numpy(), [d["mapping"] for d in plan.info()]))
        plan.destroy()
        for h in hs:
            B.release(h)
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert set(outs[0][2]) <= {B.ODE_MAP_THREAD, B.ODE_MAP_QUEUE}
