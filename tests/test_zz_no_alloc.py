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


def reference(h, w, prec, specrad=0):
    cnt = B.counters_like(w.nsys)
    y = B.integrate("rkc", h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol, counters=cnt,
                    precision=prec, codegen=B.ODE_CODEGEN_OFF, specrad=specrad)
    return y, cnt


def noalloc(h, w, prec, specrad=0, stream=None):
    cnt = B.counters_like(w.nsys)
    y = B.integrate_noalloc(h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol, counters=cnt,
                            precision=prec, specrad=specrad, stream=stream)
    return y, cnt


def same_results(w, a, b):
    (y_a, c_a), (y_b, c_b) = a, b
    assert rel(y_a, y_b, w.atol) <= TOL
    for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status"):
        np.testing.assert_array_equal(getattr(c_a, k), getattr(c_b, k))


def stiff_bruss():
    # diffusion 100 on every other grid at rtol 1e-3: steps of up to ~90
    # stages, past the scratch's 32-stage coefficient table (coefficients
    # recomputed per stage) and inside rkc_integrate's 256-stage table
    w = W.bruss(64, n=32, seed=34)
    w.params[0, ::2] = 100.0
    return W.Workload(w.name, w.kind, w.method, w.nsys, w.neq, w.y0, w.params, 0.0, 2.0, 1e-3, 1e-6,
                      bruss_n=w.bruss_n)


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


def test_noalloc_long_steps_past_the_table():
    w = stiff_bruss()
    h = B.register_workload(w)
    try:
        for _ in range(2):
            a, b = reference(h, w, B.ODE_PREC_FP64), noalloc(h, w, B.ODE_PREC_FP64)
            same_results(w, a, b)
        c = b[1]
        stages = (c.n_rhs - c.n_specrad_iter) / np.maximum(1, c.n_accept + c.n_reject)
        assert stages.max() > 32, stages.max()
    finally:
        B.release(h)


def test_noalloc_gershgorin_mode():
    # the spectral-radius option reaches the kernel: the bound replaces the
    # power method (no power iterations) and the results equal rkc_integrate's
    w = W.massaction(1000, seed=35)
    h = B.register_workload(w)
    try:
        a = reference(h, w, B.ODE_PREC_FP64, specrad=B.ODE_SPECRAD_GERSHGORIN)
        b = noalloc(h, w, B.ODE_PREC_FP64, specrad=B.ODE_SPECRAD_GERSHGORIN)
        same_results(w, a, b)
        assert (b[1].n_specrad_iter == 0).all()
        assert not np.array_equal(b[1].n_rhs, noalloc(h, w, B.ODE_PREC_FP64)[1].n_rhs)
    finally:
        B.release(h)


def test_noalloc_allocates_nothing_aliases_and_recovers():
    import torch
    w = W.massaction(2000, seed=36)
    h = B.register_workload(w)
    try:
        ref = reference(h, w, B.ODE_PREC_FP64)
        noalloc(h, w, B.ODE_PREC_FP64)          # warm-up: set-up and first launches done
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        # in place (y_out aliases y0) on pinned host arrays
        y = torch.from_numpy(w.y0.copy()).pin_memory()
        p = torch.from_numpy(w.params.copy()).pin_memory()
        cnt = B.counters_like(w.nsys)
        B.integrate_noalloc(h, y.numpy(), p.numpy(), w.t0, w.tend, w.rtol, w.atol, y_out=y.numpy(), counters=cnt)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        same_results(w, ref, (y.numpy(), cnt))
        # a refused call (a precision this entry point does not build) queues
        # nothing; the next call, on another stream, runs normally
        with pytest.raises(B.BatchOdeError) as e:
            B.integrate_noalloc(h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol,
                                precision=B.ODE_PREC_F2)
        assert e.value.code == B.ODE_ERR_ARG
        s2 = torch.cuda.Stream()
        same_results(w, ref, noalloc(h, w, B.ODE_PREC_FP64, stream=s2.cuda_stream))
    finally:
        B.release(h)

