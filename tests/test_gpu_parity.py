"""Parity of the CUDA integrators with the CPU FP64 oracle.

Plain FP64 form: identical accepted / rejected counts on >= 99.9% of systems
and a final-state error (max_i |y - y_ref| / (|y_ref| + atol)) of at most
1e-9 on every system whose step sequence matches.  Mixed form: the error
against the FP64 oracle is bounded per workload (the oracle takes different
steps than an FP32-stage integrator, so counts are not compared).
Sizes span several blocks, teams with ragged lane tails and partial warps.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

from gpu_util import rel_err, run_gpu, same_counts, summary

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


def check_fp64(w, mapping=B.ODE_MAP_AUTO, method=None, codegen=B.ODE_CODEGEN_AUTO):
    ref = O.integrate_workload(w) if method is None else O.integrate(
        O.model_for(w), 0 if method == "rkck" else 1, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol)
    g = run_gpu(w, mapping=mapping, method=method, codegen=codegen)
    s = summary(g, ref, w.atol)
    same = same_counts(g, ref)
    assert same.mean() >= 0.999, s
    assert s["max_same"] <= FP64_TOL, s
    np.testing.assert_array_equal(g["status"], ref.status)
    np.testing.assert_array_equal(g["n_rhs"][same], ref.n_rhs[same])
    np.testing.assert_array_equal(g["n_specrad_iter"][same], ref.n_specrad_iter[same])
    return s


@pytest.mark.parametrize("mapping", [B.ODE_MAP_QUEUE, B.ODE_MAP_THREAD])
def test_vdp_rkck_fp64_full_batch(mapping):
    # the full 4096-system van der Pol batch
    check_fp64(W.vdp(4096), mapping)


@pytest.mark.parametrize("nsys", [1, 33, 1000])
def test_vdp_ragged_batch_sizes(nsys):
    check_fp64(W.vdp(nsys, seed=7))


def test_vdp_rkc_fp64():
    w = W.vdp(777, seed=3)
    check_fp64(w, method="rkc")


CODEGENS = [B.ODE_CODEGEN_ON, B.ODE_CODEGEN_OFF]


@pytest.mark.parametrize("codegen", CODEGENS)
@pytest.mark.parametrize("mapping", [B.ODE_MAP_QUEUE, B.ODE_MAP_THREAD])
def test_massaction_rkc_fp64(mapping, codegen):
    # generated (straight-line network) and generic kernels both reproduce the oracle
    check_fp64(W.massaction(1500, seed=1), mapping, codegen=codegen)


@pytest.mark.parametrize("codegen", CODEGENS)
def test_massaction_rkck_fp64(codegen):
    # RKCK on the stiff network: many steps, so a shorter interval
    w = W.massaction(300, seed=2, tend=2e-6)
    check_fp64(w, method="rkck", codegen=codegen)


def test_massaction_other_network_sizes():
    # a 20-species, 40-reaction network exercises the larger generic kernels
    net = W.make_network(5, n_species=20, n_reactions=40)
    base = W.massaction(200, seed=6)
    rng = np.random.default_rng(6)
    c = rng.uniform(0.01, 1.0, (20, 200))
    c /= c.sum(axis=0)
    w = W.Workload("massaction20", W.RHS_MASSACTION, W.METHOD_RKC, 200, 20, c, base.params, 0.0, 2e-5,
                   1e-6, 1e-12, network=net)
    for cg in CODEGENS:
        check_fp64(w, codegen=cg)


@pytest.mark.parametrize("n", [32, 1, 5, 33, 100, 128])
def test_brusselator_rkc_fp64(n):
    w = W.bruss(160 if n == 32 else 48, n=n, seed=n)
    check_fp64(w)


@pytest.mark.parametrize("n", [3, 32])
def test_brusselator_rkck_fp64(n):
    w = W.bruss(40, n=n, seed=11)
    w.tend = 1.0
    check_fp64(w, method="rkck")


def chain_workload(nsys, n, seed, method):
    rng = np.random.default_rng(seed)
    mu = 10.0 ** rng.uniform(-1, 1, nsys)
    y0 = rng.uniform(-2, 2, (2 * n, nsys))
    return W.Workload("chain", W.RHS_VDP_CHAIN, method, nsys, 2 * n, y0, mu[None, :].copy(),
                      0.0, 5.0, 1e-6, 1e-9)


@pytest.mark.parametrize("n", [1, 3, 32, 40, 64])
@pytest.mark.parametrize("method", ["rkck", "rkc"])
def test_chain_fp64(n, method):
    w = chain_workload(40, n, n, W.METHOD_RKCK if method == "rkck" else W.METHOD_RKC)
    check_fp64(w)


def test_end_equals_start_copies_state():
    w = W.massaction(100)
    w.tend = w.t0
    g = run_gpu(w)
    np.testing.assert_array_equal(g["y"], w.y0)
    assert (g["n_accept"] == 0).all() and (g["n_rhs"] == 1).all()


def test_attempt_cap_status_matches_oracle():
    w = W.vdp(200, seed=5)
    ref = O.integrate_workload(w, max_attempts=50)
    g = run_gpu(w, max_attempts=50)
    np.testing.assert_array_equal(g["status"], ref.status)
    assert (g["status"] == B.ODE_ST_MAX_ATTEMPTS).any()
    same = same_counts(g, ref)
    assert same.mean() >= 0.999
    assert rel_err(g["y"], ref.y, w.atol)[same].max() <= FP64_TOL


def test_nonfinite_parameter_ends_with_status():
    w = W.vdp(64, seed=9)
    w.params[0, 5] = np.nan
    ref = O.integrate_workload(w)
    g = run_gpu(w)
    assert ref.status[5] != 0
    np.testing.assert_array_equal(g["status"], ref.status)


def test_host_buffers_match_device_buffers():
    w = W.massaction(700, seed=4)
    h = B.register_workload(w)
    cnt = B.counters_like(w.nsys)
    y_host = B.integrate("rkc", h, w.y0.copy(), w.params.copy(), w.t0, w.tend, w.rtol, w.atol, counters=cnt)
    B.release(h)
    g = run_gpu(w)
    np.testing.assert_array_equal(y_host, g["y"])
    np.testing.assert_array_equal(cnt.n_accept, g["n_accept"])


def test_in_place_output():
    import torch
    w = W.vdp(300, seed=8)
    h = B.register_workload(w)
    y = torch.from_numpy(w.y0.copy()).cuda()
    p = torch.from_numpy(w.params).cuda()
    B.integrate("rkck", h, y, p, w.t0, w.tend, w.rtol, w.atol, y_out=y, sync=True)
    B.release(h)
    g = run_gpu(w)
    np.testing.assert_array_equal(y.cpu().numpy(), g["y"])


# ------------------------------------------------------------- mixed form

MIXED_CASES = {
    "vdp": (lambda: W.vdp(2048, seed=21), 2e-3),
    "massaction": (lambda: W.massaction(2048, seed=22), 2e-3),
    "bruss": (lambda: W.bruss(128, seed=23), 2e-3),
}


@pytest.mark.parametrize("method", ["rkc", "rkck"])
def test_mixed_generated_matches_generic(method):
    # the generated network code and the generic kernels compute the same
    # FP32 arithmetic up to evaluation order: both stay close to the oracle
    w = W.massaction(1024, seed=24, tend=1e-4 if method == "rkc" else 2e-6)
    ref = O.integrate(O.model_for(w), 0 if method == "rkck" else 1, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol)
    for cg in CODEGENS:
        g = run_gpu(w, precision=B.ODE_PREC_MIXED, method=method, codegen=cg)
        assert (g["status"] & 0xFF == 0).all()
        assert np.quantile(rel_err(g["y"], ref.y, w.atol), 0.99) < 1e-3


@pytest.mark.parametrize("prec", [B.ODE_PREC_MIXED, B.ODE_PREC_MIXED_LEAN])
@pytest.mark.parametrize("name", sorted(MIXED_CASES))
def test_mixed_form_error_against_fp64_oracle(name, prec, record_property):
    make, bound = MIXED_CASES[name]
    w = make()
    ref = O.integrate_workload(w)
    g = run_gpu(w, precision=prec)
    assert (g["status"] & 0xFF == 0).all()
    e = rel_err(g["y"], ref.y, w.atol)
    record_property("max_err", float(e.max()))
    record_property("p999_err", float(np.quantile(e, 0.999)))
    print(name, prec, "mixed error vs oracle: max", e.max(), "p99.9", np.quantile(e, 0.999), "median", np.median(e))
    assert np.quantile(e, 0.999) < bound
