"""Spectral-radius modes on the GPU (the Appendix's power method and the
Gershgorin bound it names as the alternative) against the oracle.

Plain FP64: with GERSHGORIN (sigma = max_i sum_j |J_ij| of the analytic
Jacobian) and POWER_CAPPED (the power method's 1.2 sigma capped at that
bound) the kernels reproduce the oracle's counts and final states on every
family -- the bound's arithmetic and summation order are the oracle's.
Lean form: GERSHGORIN runs no power iteration and stays within the mixed
form's error bound.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

from gpu_util import rel_err

pytestmark = pytest.mark.gpu

MODES = [B.ODE_SPECRAD_GERSHGORIN, B.ODE_SPECRAD_POWER_CAPPED]


def run(w, precision, specrad, codegen=B.ODE_CODEGEN_AUTO):
    import torch
    h = B.register_workload(w)
    try:
        y0 = torch.from_numpy(np.ascontiguousarray(w.y0)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(w.params)).cuda()
        cnt = B.counters_like(w.nsys, "cuda")
        y = B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, counters=cnt, precision=precision,
                        specrad=specrad, codegen=codegen, sync=True)
        out = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        out["y"] = y.cpu().numpy()
        return out
    finally:
        B.release(h)


def oracle(w, specrad):
    return O.integrate(O.model_for(w), 1, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol, specrad=specrad)


def chain_workload(nsys, n, seed):
    """A uniform batch of n-oscillator van der Pol chains (coupling 0.1)."""
    rng = np.random.default_rng(seed)
    y0 = rng.uniform(-2.0, 2.0, size=(2 * n, nsys))
    mu = 10.0 ** rng.uniform(-1.0, 1.0, size=(1, nsys))
    return W.Workload("chain", W.RHS_VDP_CHAIN, W.METHOD_RKC, nsys, 2 * n, y0, mu, 0.0, 2.0, 1e-6, 1e-9)


def workloads():
    w_vdp = W.vdp(600, seed=4)
    w_br = W.bruss(300, n=32, seed=4)
    w_br.tend = 2.0
    w_ma = W.massaction(800, seed=4)
    return [("vdp", w_vdp, B.ODE_CODEGEN_AUTO), ("bruss", w_br, B.ODE_CODEGEN_AUTO),
            ("chain", chain_workload(400, 12, 4), B.ODE_CODEGEN_AUTO),
            ("mass-generated", w_ma, B.ODE_CODEGEN_ON), ("mass-generic", w_ma, B.ODE_CODEGEN_OFF)]


@pytest.mark.parametrize("specrad", MODES)
@pytest.mark.parametrize("name,w,codegen", workloads())
def test_fp64_modes_reproduce_oracle(name, w, codegen, specrad):
    g = run(w, B.ODE_PREC_FP64, specrad, codegen)
    r = oracle(w, specrad)
    same = (g["n_accept"] == r.n_accept) & (g["n_reject"] == r.n_reject)
    assert same.mean() >= 0.999, name
    np.testing.assert_array_equal(g["n_rhs"][same], r.n_rhs[same])
    np.testing.assert_array_equal(g["n_specrad_iter"][same], r.n_specrad_iter[same])
    assert rel_err(g["y"], r.y, w.atol)[same].max() <= 1e-9
    np.testing.assert_array_equal(g["status"], r.status)
    if specrad == B.ODE_SPECRAD_GERSHGORIN:
        assert np.all(g["n_specrad_iter"] == 0)


@pytest.mark.parametrize("specrad", MODES)
def test_lean_modes_against_oracle(specrad):
    w = W.massaction(3000, seed=9)
    g = run(w, B.ODE_PREC_MIXED_LEAN, specrad)
    r = oracle(w, specrad)
    assert ((g["status"] & 0xFF) == 0).all()
    e = rel_err(g["y"], r.y, w.atol)
    print("lean specrad", specrad, "p99.9", np.quantile(e, 0.999), "mean n_rhs", g["n_rhs"].mean(),
          "oracle", r.n_rhs.mean())
    assert np.quantile(e, 0.999) < 1e-4
    if specrad == B.ODE_SPECRAD_GERSHGORIN:
        assert np.all(g["n_specrad_iter"] == 0)
