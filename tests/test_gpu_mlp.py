"""The learned proposal's kernels against the FP64 reference network, and
what the trained proposal (first step, spectral radius, cost) changes in RKC
integration.

Forward outputs and loss gradients are compared with oracle/mlp.py evaluated
at the BF16-rounded weights the kernels use (FP32 accumulation on the GPU).
The pipeline test logs (state -> first accepted h, sigma) pairs with the
plain FP64 solver on held-out seeds, trains on the GPU, proposes for an
evaluation batch and integrates it with and without the proposals.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def make_net(n_in=14, seed=3):
    import torch
    rng = np.random.default_rng(seed)
    net = B.MLP(n_in, seed=seed)
    norm = np.zeros(M.NORM_SIZE, dtype=np.float32)
    norm[:n_in] = rng.normal(size=n_in)
    norm[33:33 + n_in] = rng.uniform(0.5, 2.0, size=n_in)
    norm[66:66 + n_in] = -1e30
    norm[99:99 + n_in] = 1e30
    norm[132:135] = rng.normal(size=3)
    norm[135:138] = rng.uniform(0.5, 2.0, size=3)
    net.set_params(norm=norm)
    X = rng.normal(size=(700, n_in)).astype(np.float32)
    Y = rng.normal(size=(700, 3)).astype(np.float32)
    return net, norm, X, Y, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()


def test_forward_matches_oracle():
    net, norm, X, _, Xt, _ = make_net()
    params, _ = net.get_params()
    out = net.apply(Xt).cpu().numpy()
    ref = M.forward(M.bf16_round(params), norm, X)
    np.testing.assert_allclose(out, ref, rtol=2e-4, atol=2e-4 * np.abs(ref).max())
    net.release()


def test_gradient_matches_oracle():
    net, norm, X, Y, Xt, Yt = make_net()
    params, _ = net.get_params()
    g, loss = net.gradient(Xt, Yt)
    loss_ref, g_ref = M.loss_and_grad(M.bf16_round(params), norm, X, Y)
    g = g.cpu().numpy()
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    # element by element: every weight's and bias's gradient (FP32 sums of
    # 700 samples' terms on the GPU against FP64): 1e-3 relative, and an
    # absolute floor of 1e-5 of the largest gradient for the near-zero ones
    np.testing.assert_allclose(g, g_ref, rtol=1e-3, atol=1e-5 * np.abs(g_ref).max())
    # summary per block of the parameter vector (W1, b1, W2, b2 + W3 + b3)
    for lo, hi in [(0, 64 * 14), (64 * 14, 64 * 15), (64 * 15, 64 * 15 + 4096), (params.size - 195, params.size)]:
        assert np.linalg.norm(g[lo:hi] - g_ref[lo:hi]) <= 1e-3 * np.linalg.norm(g_ref[lo:hi]) + 1e-9
    net.release()


def test_training_reduces_loss():
    import torch
    rng = np.random.default_rng(7)
    X = rng.normal(size=(20000, 6)).astype(np.float32)
    Y = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1], X[:, 2] * X[:, 3], np.cos(X[:, 4]) - X[:, 5]],
                 axis=1).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    net = B.MLP(6, seed=1)
    net.fit_normalization(Xt, Yt)
    hist = net.train(Xt, Yt, epochs=15, batch=512, lr=3e-3, seed=2)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.25 * hist[0], hist
    # the trained weights reproduce the oracle's loss on the same rows
    params, norm = net.get_params()
    _, loss = net.gradient(Xt[:2000], Yt[:2000])
    assert loss == pytest.approx(M.loss_and_grad(M.bf16_round(params), norm, X[:2000], Y[:2000])[0], rel=1e-3)
    net.release()


def log_pairs(w, counters=None):
    """(features -> log h, log sigma of the first accepted step, log n_rhs), by the plain FP64 solver."""
    import torch
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).cuda()
    p = torch.from_numpy(w.params).cuda()
    log = torch.full((w.nsys, w.neq + 4), float("nan"), dtype=torch.float32, device="cuda")
    B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, precision=B.ODE_PREC_FP64, log_xy=log,
                counters=counters, sync=True)
    B.release(h)
    ok = torch.isfinite(log).all(dim=1)
    return log[ok, :w.neq + 1].contiguous(), log[ok, w.neq + 1:].contiguous()


def test_training_log_records_the_first_step():
    w = W.massaction(300, seed=41)
    cnt = B.counters_like(w.nsys, "cuda")
    X, Y = log_pairs(w, cnt)
    assert X.shape[0] == 300 and Y.shape[1] == 3
    X, Y = X.cpu().numpy(), Y.cpu().numpy()
    np.testing.assert_allclose(X[:, :13], np.log(np.maximum(np.abs(w.y0.T), 1e-30)), rtol=1e-6)
    np.testing.assert_allclose(X[:, 13], w.params[0], rtol=1e-6)
    # the last column is the log of the system's whole right-hand-side count
    np.testing.assert_allclose(Y[:, 2], np.log(cnt.n_rhs.cpu().numpy()), rtol=1e-6)
    # and the oracle takes the same number of evaluations (plain FP64 parity)
    ref = O.integrate_workload(w)
    np.testing.assert_array_equal(cnt.n_rhs.cpu().numpy(), ref.n_rhs)


def test_proposal_pipeline_gain(record_property):
    import torch
    # train on held-out seeds
    X, Y = log_pairs(W.massaction(1 << 15, seed=1001))
    net = B.MLP(14, seed=0)
    net.fit_normalization(X, Y)
    hist = net.train(X, Y, epochs=30, batch=1024, lr=3e-3, seed=0)
    assert hist[-1] < hist[0]
    # evaluate on another seed, with and without the proposal
    w = W.massaction(8192, seed=5)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).cuda()
    p = torch.from_numpy(w.params).cuda()
    h0, s0, cost = net.propose(y0, p, with_cost=True)
    runs = {}
    for name, kw in (("plain", {}), ("proposal", dict(h0=h0, sigma0=s0)),
                     ("proposal_ordered", dict(h0=h0, sigma0=s0, cost=cost))):
        cnt = B.counters_like(w.nsys, "cuda")
        y = B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, counters=cnt,
                        precision=B.ODE_PREC_MIXED_LEAN, sync=True, **kw)
        runs[name] = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        runs[name]["y"] = y.cpu().numpy()
    B.release(h)
    net.release()
    ref = O.integrate_workload(w)
    pr, pl = runs["proposal"], runs["plain"]
    # taking the systems longest-first changes nothing but the time
    for k in pr:
        np.testing.assert_array_equal(runs["proposal_ordered"][k], pr[k], err_msg=k)
    # the predicted cost tracks the actual one
    c_pred = np.log(cost.cpu().numpy())
    c_true = np.log(pr["n_rhs"].astype(np.float64))
    corr = float(np.corrcoef(c_pred, c_true)[0, 1])
    record_property("cost_corr", corr)
    print("log-cost correlation", corr)
    assert corr > 0.8
    used = np.mean((pr["status"] & B.ODE_ST_PROPOSED) != 0)
    runs.pop("proposal_ordered")
    rej = {k: float(np.sum(r["n_reject"]) / np.sum(r["n_accept"] + r["n_reject"])) for k, r in runs.items()}
    rhs = {k: float(np.mean(r["n_rhs"])) for k, r in runs.items()}
    sr = {k: float(np.mean(r["n_specrad_iter"])) for k, r in runs.items()}
    err = {k: float(np.quantile(rel_err(r["y"], ref.y, w.atol), 0.999)) for k, r in runs.items()}
    for key, val in (("proposal_used", used), ("reject_rate", rej), ("mean_rhs", rhs), ("mean_specrad_iter", sr),
                     ("p999_err", err)):
        record_property(key, val)
    print("proposal used", used, "reject rate", rej, "mean RHS", rhs, "mean power iterations", sr, "p99.9 err", err)
    assert used > 0.9
    assert ((pr["status"] & 0xFF) == 0).all()
    # the initial power method and trial step are skipped where the proposal is used
    assert sr["proposal"] < sr["plain"]
    # accuracy is kept: the error test still judges every step
    assert err["proposal"] < 5 * err["plain"] + 1e-6
