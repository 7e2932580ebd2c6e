"""The allocation-free RKC entry point, rkc_integrate_noalloc.

It exists for callers that may not allocate GPU memory (a fixed memory
budget, another framework's allocator, code that must not fail on an
allocation mid-job): all its scratch is one static device array.  Here it is
called through the C ABI on host arrays and checked against rkc_integrate
(the allocating entry point, same built-in kernels) within the plain-form
tolerance of the parity tests, on two calls in a row -- the second call finds
the first call's contents in the shared array.  This file is collected last
so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9  # the plain FP64 parity tolerance (max |y - y_ref| / (|y_ref| + atol))


def reference(h, w, prec):
    cnt = B.counters_like(w.nsys)
    y = B.integrate("rkc", h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol, counters=cnt,
                    precision=prec, codegen=B.ODE_CODEGEN_OFF)
    return y, cnt


def noalloc(h, w, prec):
    cnt = B.counters_like(w.nsys)
    y = B.integrate_noalloc(h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol, counters=cnt,
                            precision=prec)
    return y, cnt


def rel(y, ref, atol):
    return float((np.abs(y - ref) / (np.abs(ref) + atol)).max())


@pytest.mark.parametrize("prec", [B.ODE_PREC_FP64, B.ODE_PREC_MIXED_LEAN])
def test_noalloc_matches_rkc_integrate_twice(prec):
    # two different batches back to back: the second call runs on the
    # scratch the first one left behind (cursor, staged arrays)
    cases = [W.massaction(3000, seed=31), W.bruss(200, n=32, seed=32)]
    for w in cases:
        h = B.register_workload(w)
        try:
            y_ref, c_ref = reference(h, w, prec)
            y_na, c_na = noalloc(h, w, prec)
            assert rel(y_na, y_ref, w.atol) <= TOL
            np.testing.assert_array_equal(c_na.n_accept, c_ref.n_accept)
            np.testing.assert_array_equal(c_na.n_reject, c_ref.n_reject)
            np.testing.assert_array_equal(c_na.status, c_ref.status)
            assert (c_na.n_accept > 0).all()
        finally:
            B.release(h)


def test_noalloc_rejects_batches_beyond_the_scratch():
    w = W.massaction(8)
    h = B.register_workload(w)
    try:
        n = B.NOALLOC_SCRATCH_BYTES // (8 * 14) + 1024   # more than the scratch can stage
        y0 = np.full((13, n), 1.0 / 13)
        p = np.full((1, n), 1500.0)
        with pytest.raises(B.BatchOdeError) as e:
            B.integrate_noalloc(h, y0, p, 0.0, 1e-6, 1e-6, 1e-12)
        assert e.value.code == B.ODE_ERR_ARG and "split" in str(e.value)
        # a batch that fits still runs after the rejection
        y = B.integrate_noalloc(h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol)
        assert np.isfinite(y).all()
    finally:
        B.release(h)
