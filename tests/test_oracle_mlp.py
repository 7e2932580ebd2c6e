"""Pins of the FP64 reference network: its analytic gradient against central
finite differences (brute force), and special cases fixed by the definition."""
import numpy as np
import pytest

from oracle import mlp as M


YM, YS = 132, 135  # offsets of y_mean[3] and y_scale[3] in the normalisation block


def random_case(n_in=5, n=7, seed=0):
    rng = np.random.default_rng(seed)
    npar = 64 * n_in + 64 + 64 * 64 + 64 + 3 * 64 + 3
    params = rng.normal(scale=0.3, size=npar)
    norm = np.zeros(138)
    norm[:n_in] = rng.normal(size=n_in)
    norm[33:33 + n_in] = rng.uniform(0.5, 2.0, size=n_in)
    norm[YM:YM + 3] = rng.normal(size=3)
    norm[YS:YS + 3] = rng.uniform(0.5, 2.0, size=3)
    X = rng.normal(size=(n, n_in))
    Y = rng.normal(size=(n, 3))
    return params, norm, X, Y


def test_layout_sizes():
    assert M.num_params(5) == 64 * 5 + 64 + 64 * 64 + 64 + 3 * 64 + 3
    assert M.NORM_SIZE == 138


def test_gradient_matches_finite_differences():
    params, norm, X, Y = random_case()
    loss, g = M.loss_and_grad(params, norm, X, Y)
    rng = np.random.default_rng(1)
    idx = rng.choice(params.size, 60, replace=False)
    eps = 1e-6
    for k in idx:
        p1, p2 = params.copy(), params.copy()
        p1[k] += eps
        p2[k] -= eps
        fd = (M.loss_and_grad(p1, norm, X, Y)[0] - M.loss_and_grad(p2, norm, X, Y)[0]) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k


def test_biases_only_network_outputs_biases():
    n_in = 3
    params = np.zeros(64 * n_in + 64 + 4096 + 64 + 192 + 3)
    params[-3:] = [0.7, -1.3, 0.25]
    norm = np.zeros(138)
    norm[33:36] = 1.0
    norm[YM:YM + 3] = [1.0, 2.0, -1.0]
    norm[YS:YS + 3] = [2.0, 3.0, 4.0]
    out = M.forward(params, norm, np.ones((4, n_in)))
    np.testing.assert_allclose(out, [[0.7 * 2 + 1, -1.3 * 3 + 2, 0.25 * 4 - 1]] * 4)


def test_zero_residual_rows_have_zero_loss_and_gradient():
    # targets equal to the outputs: every loss term is at its minimum, zero
    params, norm, X, _ = random_case(n=4)
    Y = M.forward(params, norm, X)
    loss, g = M.loss_and_grad(params, norm, X, Y)
    assert loss == pytest.approx(0.0, abs=1e-12)
    # the pinball term has a kink at zero residual (subgradient 1 - tau);
    # the squared terms contribute nothing
    Y2 = Y.copy()
    Y2[:, 2] += norm[YS + 2] * 0.5          # log-cost residual of -0.5 normalised
    loss2, _ = M.loss_and_grad(params, norm, X, Y2)
    assert loss2 == pytest.approx(0.25)


def test_pinball_loss_prefers_overestimates():
    # an over-estimate of log sigma by d costs (1 - tau) d, an under-estimate tau d
    params, norm, X, Y = random_case(n=1)
    p = M.forward(params, norm, X)
    ys = norm[YS:YS + 3]
    base = M.loss_and_grad(params, norm, X, np.array([[p[0, 0], p[0, 1], p[0, 2]]]))[0]
    up = M.loss_and_grad(params, norm, X, np.array([[p[0, 0], p[0, 1] - ys[1], p[0, 2]]]))[0]
    down = M.loss_and_grad(params, norm, X, np.array([[p[0, 0], p[0, 1] + ys[1], p[0, 2]]]))[0]
    assert base == pytest.approx(0.0, abs=1e-12)
    assert up == pytest.approx(1 - M.TAU) and down == pytest.approx(M.TAU)


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0], dtype=np.float32)
    r = M.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125   # ties to even, then round up
    assert abs(r[3] / -3.14159 - 1) < 2 ** -8


def entry_term(params, norm, X, Y, r, c):
    """Loss term of target (r, c), straight from the definition on the
    network's normalised output."""
    p = (M.forward(params, norm, X[r:r + 1])[0, c] - norm[YM + c]) / norm[YS + c]
    t = (Y[r, c] - norm[YM + c]) / norm[YS + c]
    if c == 1:
        d = t - p
        return M.TAU * d if d > 0 else (M.TAU - 1.0) * d
    return (p - t) ** 2


def test_nan_target_drops_its_term():
    # a NaN target adds nothing: the mean loss loses exactly that entry's term
    params, norm, X, Y = random_case(n=6, seed=3)
    n = X.shape[0]
    loss, _ = M.loss_and_grad(params, norm, X, Y)
    Y2 = Y.copy()
    masked = [(0, 0), (2, 2), (3, 0), (3, 2), (5, 1)]
    for r, c in masked:
        Y2[r, c] = np.nan
    loss2, g2 = M.loss_and_grad(params, norm, X, Y2)
    drop = sum(entry_term(params, norm, X, Y, r, c) for r, c in masked)
    assert loss2 * n == pytest.approx(loss * n - drop, rel=1e-12, abs=1e-12)
    assert np.all(np.isfinite(g2))
    # a row with no target at all adds neither loss nor gradient
    Y3 = Y.copy()
    Y3[4, :] = np.nan
    l_all, g_all = M.loss_and_grad(params, norm, X, Y3)
    keep = [0, 1, 2, 3, 5]
    l_sub, g_sub = M.loss_and_grad(params, norm, X[keep], Y[keep])
    assert l_all * n == pytest.approx(l_sub * len(keep), rel=1e-12)
    np.testing.assert_allclose(g_all * n, g_sub * len(keep), rtol=1e-10, atol=1e-14)


def test_masked_gradient_matches_finite_differences():
    params, norm, X, Y = random_case(n=5, seed=4)
    Y[1, 0] = Y[2, 2] = Y[3, 0] = Y[3, 2] = np.nan  # spectral-radius records: sigma target only
    _, g = M.loss_and_grad(params, norm, X, Y)
    rng = np.random.default_rng(5)
    eps = 1e-6
    for k in rng.choice(params.size, 40, replace=False):
        p1, p2 = params.copy(), params.copy()
        p1[k] += eps
        p2[k] -= eps
        fd = (M.loss_and_grad(p1, norm, X, Y)[0] - M.loss_and_grad(p2, norm, X, Y)[0]) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k
