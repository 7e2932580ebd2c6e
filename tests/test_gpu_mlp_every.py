"""The proposal network evaluated inside the two-float RKC kernel at every
spectral-radius point (ode_opts.mlp), its training data and its pieces.

- The warp-level tensor-core evaluation (mma.sync, BF16 inputs, weights
  and activations, FP32 accumulation) against oracle/mlp.py with BF16
  rounding of the operands, for one, two and three k-steps of inputs.
- Training with missing targets (NaN): gradients element by element
  against the FP64 reference, the normalisation over the present values.
- The spectral-radius log of the plain FP64 solver: its first record is the
  first-step record; every record's sigma is 1.2 x the spectral radius of
  the Jacobian (numpy eigenvalues of the oracle's analytic Jacobian) at
  the state it logs.
- Integration with the network in the kernel: the power method all but
  disappears, the evaluations it took are saved, the step sequence keeps
  its accepted-step count and reject rate, and the final states stay
  within the 1e-5 bar of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

from gpu_util import rel_err

pytestmark = pytest.mark.gpu

TARGET = 1e-5


def random_net(n_in, seed):
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
    return net, norm, rng


@pytest.mark.parametrize("n_in", [14, 20, 33])
def test_warp_evaluation_matches_oracle(n_in):
    import torch
    net, norm, rng = random_net(n_in, seed=n_in)
    X = rng.normal(size=(1003, n_in)).astype(np.float32)   # 31 full warps and a ragged one
    params, _ = net.get_params()
    out = net.apply_warp(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = M.forward(M.bf16_round(params), norm, X, bf16_operands=True)[:, :2]
    ys = norm[135:137]
    d = np.abs(out - ref) / ys       # in units of the normalised outputs
    # FP32 sums in another order, and ulp-level differences that flip a
    # BF16 rounding of an input or activation now and then
    assert np.median(d) <= 1e-6, np.median(d)
    assert np.mean(d > 1e-4) <= 0.02, np.mean(d > 1e-4)
    assert d.max() <= 2e-3, d.max()
    # against the FP32-activation path: only the BF16 activations differ
    full = net.apply(torch.from_numpy(X).cuda()).cpu().numpy()[:, :2]
    assert (np.abs(out - full) / ys).max() <= 5e-2
    net.release()


def test_masked_targets_gradient_and_normalisation():
    import torch
    net, norm, rng = random_net(14, seed=5)
    X = rng.normal(size=(900, 14)).astype(np.float32)
    Y = rng.normal(size=(900, 3)).astype(np.float32)
    Y[300:, 0] = np.nan   # spectral-radius records: sigma target only
    Y[300:, 2] = np.nan
    Y[::7, 1] = np.nan
    params, _ = net.get_params()
    g, loss = net.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    loss_ref, g_ref = M.loss_and_grad(M.bf16_round(params), norm, X, Y)
    g = g.cpu().numpy()
    assert np.isfinite(loss) and loss == pytest.approx(loss_ref, rel=1e-4)
    np.testing.assert_allclose(g, g_ref, rtol=1e-3, atol=1e-5 * np.abs(g_ref).max())
    # statistics over the present values only
    net.fit_normalization(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    _, nrm = net.get_params()
    for c in range(3):
        col = Y[:, c].astype(np.float64)
        col = col[np.isfinite(col)]
        assert nrm[132 + c] == pytest.approx(col.mean(), rel=1e-5, abs=1e-6)
        assert nrm[135 + c] == pytest.approx(col.std(), rel=1e-4)
    net.release()


def fp64_logs(w, records, every, counters=None):
    """The plain FP64 solver's first-step log [nsys, neq + 4] and
    spectral-radius log [nsys, records, neq + 2] (NaN where not written)."""
    import torch
    h = B.register_workload(w)
    log = torch.full((w.nsys, w.neq + 4), float("nan"), dtype=torch.float32, device="cuda")
    lsr = torch.full((w.nsys, records, w.neq + 2), float("nan"), dtype=torch.float32, device="cuda")
    B.integrate("rkc", h, torch.from_numpy(w.y0).cuda(), torch.from_numpy(w.params).cuda(), w.t0, w.tend,
                w.rtol, w.atol, precision=B.ODE_PREC_FP64, log_xy=log, log_sr=lsr, log_sr_every=every,
                counters=counters, sync=True)
    B.release(h)
    return log, lsr


def test_spectral_radius_log():
    w = W.massaction(400, seed=43)
    cnt = B.counters_like(w.nsys, "cuda")
    log, lsr = fp64_logs(w, records=6, every=3, counters=cnt)
    log, lsr = log.cpu().numpy(), lsr.cpu().numpy()
    n = w.neq
    # estimate 0 is taken at y0, and (without a rejection before the first
    # accepted step) it is the first step's sigma
    np.testing.assert_allclose(lsr[:, 0, :n], np.log(np.maximum(np.abs(w.y0.T), 1e-30)), rtol=1e-6)
    np.testing.assert_allclose(lsr[:, 0, n], w.params[0], rtol=1e-6)
    assert np.mean(lsr[:, 0, n + 1] == log[:, n + 2]) >= 0.99
    # later records: sigma = 1.2 x the Jacobian's spectral radius at the logged state
    m = O.model_for(w)
    ratios = []
    for i in range(0, w.nsys, 4):
        for r in range(1, 6):
            rec = lsr[i, r]
            if not np.isfinite(rec).all():
                continue
            y = np.exp(rec[:n].astype(np.float64))
            J = O.jacobian(m, w.params[:, i].copy(), y)
            rho = np.abs(np.linalg.eigvals(J)).max()
            sig = np.exp(float(rec[n + 1]))
            ratios.append(sig / (1.2 * rho))
    ratios = np.array(ratios)
    assert ratios.size >= 400
    # the power method's estimate converges to ~1 % (Appendix); a few
    # estimates stop on another eigenvalue's component
    assert np.median(np.abs(ratios - 1)) <= 0.02, np.median(np.abs(ratios - 1))
    assert np.mean(np.abs(ratios - 1) <= 0.1) >= 0.9


def train_every(nsys=1 << 16, seed=1001, epochs=12):
    """A network trained on the first-step records and the spectral-radius
    records of a held-out FP64 run (sigma-only rows carry NaN targets)."""
    import torch
    w = W.massaction(nsys, seed=seed)
    log, lsr = fp64_logs(w, records=8, every=5)
    ok = torch.isfinite(log).all(dim=1)
    X1, Y1 = log[ok, :w.neq + 1], log[ok, w.neq + 1:]
    r = lsr.reshape(-1, w.neq + 2)
    r = r[torch.isfinite(r).all(dim=1)]
    Y2 = torch.full((r.shape[0], 3), float("nan"), device="cuda")
    Y2[:, 1] = r[:, w.neq + 1]
    X = torch.cat([X1, r[:, :w.neq + 1]]).contiguous()
    Y = torch.cat([Y1, Y2]).contiguous()
    net = B.MLP(w.neq + 1, seed=0)
    net.fit_normalization(X, Y)
    hist = net.train(X, Y, epochs=epochs, batch=4096, lr=2e-3, seed=0)
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
    return net


@pytest.mark.parametrize("mapping", [B.ODE_MAP_THREAD, B.ODE_MAP_QUEUE])
def test_network_at_every_spectral_radius_point(mapping):
    import torch
    net = train_every()
    w = W.massaction(16384, seed=6)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).cuda()
    p = torch.from_numpy(w.params).cuda()
    runs = {}
    for name, kw in (("without", {}), ("network", dict(mlp=net))):
        cnt = B.counters_like(w.nsys, "cuda")
        y = B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, counters=cnt, mapping=mapping,
                        precision=B.ODE_PREC_F2_LEAN, sync=True, **kw)
        runs[name] = {k: getattr(cnt, k).cpu().numpy().astype(np.float64)
                      for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter")}
        runs[name]["status"] = cnt.status.cpu().numpy()
        runs[name]["y"] = y.cpu().numpy()
    B.release(h)
    net.release()
    wo, nw = runs["without"], runs["network"]
    assert ((nw["status"] & 0xFF) == 0).all()
    assert np.mean((nw["status"] & B.ODE_ST_PROPOSED) != 0) >= 0.99
    # the power method is gone but for the points after a rejection and the
    # bounds the checks refuse
    assert nw["n_specrad_iter"].mean() <= 0.01 * wo["n_specrad_iter"].mean()
    # its evaluations are saved and nothing else changes in the work
    saved = wo["n_specrad_iter"].mean() - nw["n_specrad_iter"].mean()
    assert nw["n_rhs"].mean() <= wo["n_rhs"].mean() - 0.9 * saved
    assert nw["n_accept"].mean() == pytest.approx(wo["n_accept"].mean(), rel=5e-3)
    rej = {k: r["n_reject"].sum() / (r["n_accept"].sum() + r["n_reject"].sum()) for k, r in runs.items()}
    assert rej["network"] <= 2 * rej["without"] + 1e-6, rej
    # accuracy against the FP64 oracle: the chosen form's bar
    ref = O.integrate_workload(w)
    e = rel_err(nw["y"], ref.y, w.atol)
    print("network: power iterations", nw["n_specrad_iter"].mean(), "of", wo["n_specrad_iter"].mean(),
          "RHS", nw["n_rhs"].mean(), "of", wo["n_rhs"].mean(), "reject", rej, "p99.9", np.quantile(e, 0.999),
          "max", e.max())
    assert np.quantile(e, 0.999) <= TARGET
    assert e.max() <= 10 * TARGET
