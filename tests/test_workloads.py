"""The seeded synthetic inputs follow their stated recipe: shapes, ranges,
normalisation, per-family intervals and tolerances, and determinism by seed
(the same seed gives the same batch, another seed another one).  These are
the inputs of every parity test and of the benchmark."""
import numpy as np
import pytest

from paper_1611_02274_gb300 import workloads as W


def test_vdp_recipe():
    w = W.vdp(nsys=4096, seed=0)
    assert (w.neq, w.nsys, w.method, w.kind) == (2, 4096, W.METHOD_RKCK, W.RHS_VDP)
    assert w.y0.shape == (2, 4096) and np.abs(w.y0).max() <= 2.0
    mu = w.params[0]
    assert np.log10(mu).min() >= -1.0 and np.log10(mu).max() <= 1.0
    assert np.log10(mu).std() > 0.5                  # log-uniform, not clustered
    assert (w.t0, w.tend, w.rtol, w.atol) == (0.0, 20.0, 1e-6, 1e-9)


def test_brusselator_recipe():
    n = 32
    w = W.bruss(nsys=2048, n=n, seed=0)
    assert (w.neq, w.bruss_n, w.method) == (2 * n, n, W.METHOD_RKC)
    x = np.arange(1, n + 1) / (n + 1)
    u, v = w.y0[:n], w.y0[n:]
    assert np.abs(u - (1.0 + np.sin(2 * np.pi * x))[:, None]).max() <= 0.1
    assert np.abs(v - 3.0).max() <= 0.1
    a = w.params[0]
    assert a.min() >= 0.01 and a.max() <= 0.05
    assert (w.t0, w.tend, w.rtol, w.atol) == (0.0, 10.0, 1e-5, 1e-8)


def test_massaction_recipe():
    w = W.massaction(nsys=4096, seed=0)
    net = w.network
    assert (net.n_species, len(net.n_reac), w.neq) == (13, 27, 13)
    assert set(net.n_reac) <= {1, 2} and set(net.n_prod) <= {1, 2}
    for j in range(27):
        for q in range(2):
            r, p = net.reac[j][q], net.prod[j][q]
            assert (0 <= r < 13) if q < net.n_reac[j] else r == -1
            assert (0 <= p < 13) if q < net.n_prod[j] else p == -1
    assert net.log10A.min() >= 6 and net.log10A.max() <= 14
    assert np.abs(net.beta).max() <= 1 and net.Ea.min() >= 0 and net.Ea.max() <= 20000
    assert (net.kmin, net.kmax) == (1e-2, 1e6)
    T = w.params[0]
    assert T.min() >= 1000 and T.max() <= 2000
    assert (w.y0 > 0).all()
    np.testing.assert_allclose(w.y0.sum(axis=0), 1.0, rtol=1e-14)
    assert (w.t0, w.tend, w.rtol, w.atol) == (0.0, 1e-4, 1e-6, 1e-12)
    # one network shared by every system, drawn from its own seed
    w2 = W.massaction(nsys=16, seed=5)
    np.testing.assert_array_equal(w2.network.log10A, net.log10A)


def test_mixed_batch_recipe():
    b = W.mixed(nsys=4000, seed=0)
    is_b = b.kind == W.RHS_BRUSS1D
    assert is_b.sum() == 2000                         # half and half
    assert b.n[is_b].min() >= 1 and b.n[is_b].max() <= 128
    assert b.n[~is_b].min() >= 1 and b.n[~is_b].max() <= 64
    np.testing.assert_array_equal(b.neq, 2 * b.n)
    np.testing.assert_array_equal(np.diff(b.offset), b.neq)
    assert b.offset[0] == 0 and b.offset[-1] == b.y0.size
    assert (b.method[is_b] == W.METHOD_RKC).all() and (b.method[~is_b] == W.METHOD_RKCK).all()
    np.testing.assert_array_equal(b.tend, np.where(is_b, 10.0, 20.0))
    np.testing.assert_array_equal(b.rtol, np.where(is_b, 1e-5, 1e-6))
    np.testing.assert_array_equal(b.atol, np.where(is_b, 1e-8, 1e-9))


def test_kinetics_recipe():
    w = W.kinetics(nsys=64, seed=0)
    mech = w.aux["mechanism"]
    S = mech.n_species
    assert (S, len(mech.n_reac), w.neq) == (57, 766, 58)
    np.testing.assert_allclose(w.y0[1:].sum(axis=0), 1.0, rtol=1e-14)
    assert (w.y0[1:] >= 0).all() and (w.y0[0] > 0).all()
    # every reaction balances every element
    for j in range(len(mech.n_reac)):
        left = sum(mech.comp[mech.reac[j][q]] for q in range(mech.n_reac[j]))
        right = sum(mech.comp[mech.prod[j][q]] for q in range(mech.n_prod[j]))
        np.testing.assert_array_equal(left, right)


def test_pleiades_recipe():
    w = W.pleiades(nsys=256, seed=0)
    m = w.aux["masses"]
    np.testing.assert_array_equal(m, np.arange(1, 8))
    assert (w.neq, w.rtol, w.atol, w.method) == (28, 1e-10, 1e-10, W.METHOD_RKCK)
    _, base = W.pleiades_base()
    assert np.abs(w.y0 - base[:, None]).max() < 1e-2   # perturbed copies of one configuration
    u, v = base[14:21], base[21:]
    assert abs(np.sum(m * u)) < 1e-12 and abs(np.sum(m * v)) < 1e-12   # zero total momentum


@pytest.mark.parametrize("make", [lambda s: W.vdp(256, seed=s), lambda s: W.bruss(256, seed=s),
                                  lambda s: W.massaction(256, seed=s), lambda s: W.kinetics(16, seed=s),
                                  lambda s: W.pleiades(64, seed=s)])
def test_seeded_and_deterministic(make):
    a, b, c = make(3), make(3), make(4)
    np.testing.assert_array_equal(a.y0, b.y0)
    np.testing.assert_array_equal(a.params, b.params)
    assert not np.array_equal(a.y0, c.y0)


def test_subset_takes_columns():
    w = W.massaction(nsys=100, seed=1)
    idx = np.array([3, 50, 99])
    s = W.subset(w, idx)
    np.testing.assert_array_equal(s.y0, w.y0[:, idx])
    np.testing.assert_array_equal(s.params, w.params[:, idx])
    assert s.nsys == 3 and s.network is w.network
