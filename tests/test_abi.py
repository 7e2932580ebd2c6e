"""The C ABI library builds, loads and exports every declared entry point;
host-side validation answers without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\([^;]*\)\s*;", text, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    lib = B.load()
    names = declared_functions()
    assert set(B.EXPORTED) <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert "sm_103a" in B.version()


def test_register_validation():
    with pytest.raises(B.BatchOdeError) as e:
        B.register(99, 2)
    assert e.value.code == B.ODE_ERR_ARG
    with pytest.raises(B.BatchOdeError):
        B.register(B.ODE_RHS_VDP, 3)
    with pytest.raises(B.BatchOdeError):
        B.register(B.ODE_RHS_BRUSS1D, 7)
    net = W.make_network(0)
    bad = W.Network(net.n_species, net.n_reac, net.reac.copy(), net.n_prod, net.prod, net.log10A,
                    net.beta, net.Ea)
    bad.reac[0, 0] = 13
    with pytest.raises(B.BatchOdeError):
        B.register(B.ODE_RHS_MASSACTION, 13, network=bad)
    h = B.register(B.ODE_RHS_MASSACTION, 13, network=net)
    assert h > 0
    B.release(h)
    with pytest.raises(B.BatchOdeError) as e:
        B.release(h)
    assert e.value.code == B.ODE_ERR_HANDLE


def test_integrate_argument_errors_before_any_launch():
    h = B.register(B.ODE_RHS_VDP, 2)
    y = np.zeros((2, 4))
    p = np.ones((1, 4))
    for kw, code in [(dict(rtol=0.0), B.ODE_ERR_ARG), (dict(atol=-1.0), B.ODE_ERR_ARG),
                     (dict(t0=1.0, tend=0.0), B.ODE_ERR_ARG)]:
        args = dict(t0=0.0, tend=1.0, rtol=1e-6, atol=1e-9)
        args.update(kw)
        with pytest.raises(B.BatchOdeError) as e:
            B.integrate("rkck", h, y, p, **args)
        assert e.value.code == code
    with pytest.raises(B.BatchOdeError) as e:
        B.integrate("rkc", h + 1000, y, p, 0.0, 1.0, 1e-6, 1e-9)
    assert e.value.code == B.ODE_ERR_HANDLE
    # an empty batch is a successful no-op
    B.integrate("rkck", h, np.zeros((2, 0)), np.zeros((1, 0)), 0.0, 1.0, 1e-6, 1e-9)
    o = B.Opts()
    o.reserved[2] = 1
    rc = B.load().rkck_integrate(h, 4, C.c_void_p(y.ctypes.data), C.c_void_p(p.ctypes.data), 0.0, 1.0,
                                 1e-6, 1e-9, C.byref(o), C.c_void_p(y.ctypes.data), None, None)
    assert rc == B.ODE_ERR_ARG
    # cost ordering, proposals and logs need device arrays
    cost = np.ones(4, dtype=np.float32)
    with pytest.raises(B.BatchOdeError) as e:
        B.integrate("rkck", h, y, p, 0.0, 1.0, 1e-6, 1e-9, cost=cost)
    assert e.value.code == B.ODE_ERR_ARG
    carry = np.zeros((B.carry_words(2), 4))
    with pytest.raises(B.BatchOdeError) as e:
        B.integrate("rkc", h, y, p, 0.0, 1.0, 1e-6, 1e-9, carry=carry)
    assert e.value.code == B.ODE_ERR_ARG
    B.release(h)
    # the stand-alone order: bad sizes and NULL arrays are refused before any launch
    L = B.load()
    assert L.ode_cost_order(None, -1, None, None) == B.ODE_ERR_ARG
    assert L.ode_cost_order(None, 5, None, None) == B.ODE_ERR_ARG
    assert L.ode_cost_order(None, 0, None, None) == B.ODE_OK


def test_network_and_log_options_are_checked_before_any_launch():
    # the in-kernel network is for the two-float RKC forms, the
    # spectral-radius log for the plain FP64 RKC; both refused elsewhere
    # before any device work (no GPU needed to see it)
    lib = B.load()
    w = W.massaction(4, seed=0)
    h = B.register_workload(w)
    y, p = np.ascontiguousarray(w.y0), np.ascontiguousarray(w.params)
    args = (h, 4, C.c_void_p(y.ctypes.data), C.c_void_p(p.ctypes.data), w.t0, w.tend, w.rtol, w.atol)
    out = np.empty_like(y)
    for fn, prec, field, code in ((lib.rkc_integrate, B.ODE_PREC_FP64, "mlp", B.ODE_ERR_UNSUPPORTED),
                                  (lib.rkck_integrate, B.ODE_PREC_F2_LEAN, "mlp", B.ODE_ERR_UNSUPPORTED),
                                  (lib.rkc_integrate, B.ODE_PREC_MIXED, "mlp", B.ODE_ERR_UNSUPPORTED),
                                  (lib.rkc_integrate, B.ODE_PREC_F2_LEAN, "log_sr", B.ODE_ERR_UNSUPPORTED),
                                  (lib.rkc_integrate, B.ODE_PREC_FP64, "log_sr", B.ODE_ERR_ARG)):
        o = B.Opts()
        o.precision = prec
        o.io = B.ODE_IO_HOST
        if field == "mlp":
            o.mlp = 7
        else:
            o.log_sr = C.c_void_p(out.ctypes.data)  # records 0: refused
        rc = fn(*args, C.byref(o), C.c_void_p(out.ctypes.data), None, None)
        assert rc == code, (field, prec, rc)
    o = B.Opts()
    o.mlp = 7
    rc = lib.rkc_integrate_noalloc(*args, C.byref(o), C.c_void_p(out.ctypes.data), None, None)
    assert rc == B.ODE_ERR_ARG
    B.release(h)


def test_two_float_rkck_families_are_checked_before_any_launch():
    # the two-float RKCK is built for van der Pol systems and chains: other
    # families are refused by the argument checks (no GPU needed), while
    # these two pass them and go on to the device
    lib = B.load()
    cases = ((W.massaction(4, seed=0), B.ODE_ERR_UNSUPPORTED), (W.bruss(4, n=3, seed=0), B.ODE_ERR_UNSUPPORTED),
             (W.vdp(4, seed=0), None))
    for w, code in cases:
        h = B.register_workload(w)
        y, p = np.ascontiguousarray(w.y0), np.ascontiguousarray(w.params)
        out = np.empty_like(y)
        for prec in (B.ODE_PREC_F2, B.ODE_PREC_F2_LEAN):
            o = B.Opts()
            o.precision = prec
            o.io = B.ODE_IO_HOST
            rc = lib.rkck_integrate(h, 4, C.c_void_p(y.ctypes.data), C.c_void_p(p.ctypes.data), w.t0, w.tend,
                                    w.rtol, w.atol, C.byref(o), C.c_void_p(out.ctypes.data), None, None)
            if code is not None:
                assert rc == code, (w.name, prec, rc)
            else:
                assert rc != B.ODE_ERR_UNSUPPORTED and rc != B.ODE_ERR_ARG, (w.name, prec, rc)
        assert lib.ode_rhs_prepare(h, 0, B.ODE_PREC_F2_LEAN) == (B.ODE_ERR_UNSUPPORTED if code else B.ODE_OK)
        B.release(h)


def test_generated_network_kernels_compile():
    """ode_rhs_prepare compiles the straight-line network kernels (NVRTC);
    without a device this is a compile-only check."""
    import ctypes
    try:
        ctypes.CDLL("libnvrtc.so.13")
    except OSError:
        pytest.skip("NVRTC not installed")
    w = W.massaction(8)
    h = B.register_workload(w)
    for m in ("rkc", "rkck"):
        for p in (B.ODE_PREC_FP64, B.ODE_PREC_MIXED):
            B.prepare(h, m, p)
    assert B.load().ode_rhs_prepare(h, 7, 0) == B.ODE_ERR_ARG
    B.release(h)
    # other families need no preparation
    h = B.register(B.ODE_RHS_VDP, 2)
    B.prepare(h, "rkck")
    B.release(h)
