"""Pins of the oracle's right-hand sides (mass-action law and Arrhenius
rate of Section 4.2; the synthetic van der Pol, chain and Brusselator
systems) against special cases and spectra fixed by the mathematics."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import workloads as W


def net(reactions, n_species, log10A=None, beta=None, Ea=None):
    R = len(reactions)
    n_reac = np.array([len(r) for r, _ in reactions], dtype=np.int32)
    n_prod = np.array([len(p) for _, p in reactions], dtype=np.int32)
    reac = np.full((R, 2), -1, dtype=np.int32)
    prod = np.full((R, 2), -1, dtype=np.int32)
    for j, (r, p) in enumerate(reactions):
        reac[j, :len(r)] = r
        prod[j, :len(p)] = p
    z = np.zeros(R)
    return W.Network(n_species, n_reac, reac, n_prod, prod,
                     z if log10A is None else np.asarray(log10A, float),
                     z if beta is None else np.asarray(beta, float),
                     z if Ea is None else np.asarray(Ea, float), kmin=1e-30, kmax=1e30)


def fd_jacobian(mod, p, y, eps=1e-6):
    n = len(y)
    J = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = eps
        J[:, j] = (O.rhs(mod, p, y + e) - O.rhs(mod, p, y - e)) / (2 * eps)
    return J


def test_mass_action_law_special_cases():
    # A + B -> C with k = 10^2 and 2A -> B with k = 10^0 (T^0, Ea = 0)
    n = net([([0, 1], [2]), ([0, 0], [1])], 3, log10A=[2.0, 0.0])
    mod = O.model(O.KIND_MASSACTION, 3, 1, network=n)
    a, b, c = 0.3, 0.7, 0.1
    f = O.rhs(mod, [1500.0], [a, b, c])
    r1, r2 = 100.0 * a * b, a * a
    np.testing.assert_allclose(f, [-r1 - 2 * r2, -r1 + r2, r1], rtol=1e-15)


def test_arrhenius_special_values():
    T = 1500.0
    n = net([([0], [1])] * 4, 2, log10A=[0.0, 2.0, 0.0, 3.0], beta=[0.0, 0.0, 1.0, -1.0],
            Ea=[0.0, T * math.log(10.0), 0.0, 0.0])
    mod = O.model(O.KIND_MASSACTION, 2, 1, network=n)
    k = O.rate_constants(mod, T)
    np.testing.assert_allclose(k, [1.0, 10.0, T, 1000.0 / T], rtol=1e-14)
    # clipping to the configured band
    mod.kmin, mod.kmax = 2.0, 100.0
    np.testing.assert_allclose(O.rate_constants(mod, T), [2.0, 10.0, 100.0, 2.0], rtol=1e-14)


@pytest.mark.parametrize("method", [0, 1])
def test_conservative_network_preserves_total(method):
    # only 1 -> 1 and 2 -> 2 reactions: sum(C) is a linear invariant, which
    # every Runge-Kutta method preserves up to rounding
    n = net([([0], [1]), ([1], [2]), ([0, 1], [2, 3]), ([2, 2], [0, 1]), ([3], [0])], 4,
            log10A=[3.0, 2.5, 4.0, 3.5, 2.0])
    mod = O.model(O.KIND_MASSACTION, 4, 1, network=n)
    y0 = np.array([[0.4, 0.1], [0.3, 0.2], [0.2, 0.3], [0.1, 0.4]])
    r = O.integrate(mod, method, y0, [[1500.0, 1200.0]], 0.0, 1e-2, 1e-6, 1e-12)
    assert ((r.status & 0xFF) == 0).all()
    np.testing.assert_allclose(r.y.sum(axis=0), y0.sum(axis=0), rtol=1e-13)
    assert not np.allclose(r.y, y0)


@pytest.mark.parametrize("method,rtol", [(0, 1e-9), (1, 1e-7)])
def test_unimolecular_network_matches_expm(method, rtol):
    from scipy.linalg import expm
    reactions = [([0], [1]), ([1], [2]), ([2], [0]), ([1], [3]), ([3], [1, 2])]
    log10A = [3.0, 2.0, 2.5, 1.0, 3.2]
    n = net(reactions, 4, log10A=log10A)
    mod = O.model(O.KIND_MASSACTION, 4, 1, network=n)
    K = np.zeros((4, 4))
    for (r, p), la in zip(reactions, log10A):
        k = 10.0 ** la
        K[r[0], r[0]] -= k
        for s in p:
            K[s, r[0]] += k
    y0 = np.array([0.5, 0.2, 0.2, 0.1])
    tend = 5e-3
    res = O.integrate(mod, method, y0[:, None], [[1000.0]], 0.0, tend, rtol, 1e-14)
    exact = expm(tend * K) @ y0
    bound = 30 * rtol if method == 0 else 3 * rtol ** (2.0 / 3.0)
    np.testing.assert_allclose(res.y[:, 0], exact, rtol=bound)


def test_brusselator_steady_state_and_spectrum():
    n, a = 6, 0.02
    mod = O.model(O.KIND_BRUSS1D, 2 * n, 1)
    y = np.concatenate([np.ones(n), 3.0 * np.ones(n)])   # u = A, v = B/A, matching the boundary
    np.testing.assert_allclose(O.rhs(mod, [a], y), 0.0, atol=1e-13)
    ev = np.linalg.eigvals(fd_jacobian(mod, [a], y))
    D = a * (n + 1) ** 2
    lam = [-4 * D * math.sin(k * math.pi / (2 * (n + 1))) ** 2 for k in range(1, n + 1)]
    # each Laplacian mode shifts the reaction block [[2, 1], [-3, -1]] (trace 1, det 1)
    want = [l + 0.5 + s * 1j * math.sqrt(3) / 2 for l in lam for s in (1, -1)]
    key = lambda z: (round(z.real, 6), round(z.imag, 6))
    np.testing.assert_allclose(sorted(ev, key=key), sorted(want, key=key), atol=1e-6)


def test_vdp_linearisation_at_origin():
    mod = O.model(O.KIND_VDP, 2, 1)
    for mu in (0.1, 2.0, 10.0):
        ev = np.sort_complex(np.linalg.eigvals(fd_jacobian(mod, [mu], np.zeros(2))))
        want = np.sort_complex(np.roots([1.0, -mu, 1.0]).astype(complex))
        np.testing.assert_allclose(ev, want, atol=1e-8)


def test_vdp_chain_is_coupled_harmonic_chain_at_mu_zero():
    n, c = 5, 0.1
    mod = O.model(O.KIND_VDP_CHAIN, 2 * n, 1, coupling=c)
    y = np.random.default_rng(3).normal(size=2 * n)
    ev = np.linalg.eigvals(fd_jacobian(mod, [0.0], y))
    # free-end chain Laplacian eigenvalues -4 sin^2(k pi / 2n), k = 0..n-1
    om = [math.sqrt(1 + 4 * c * math.sin(k * math.pi / (2 * n)) ** 2) for k in range(n)]
    want = sorted([s * w for w in om for s in (1, -1)])
    np.testing.assert_allclose(sorted(ev.imag), want, atol=1e-8)
    np.testing.assert_allclose(ev.real, 0.0, atol=1e-8)


def test_series_log_exp_pow_against_libm():
    rng = np.random.default_rng(0)
    xs = np.concatenate([10.0 ** rng.uniform(-300, 300, 2000), rng.uniform(0.5, 2.0, 2000), [1.0, 2.0, 0.5]])
    for x in xs:
        assert O.series_log(x) == pytest.approx(math.log(x), rel=1e-15, abs=2e-17)
    for x in np.concatenate([rng.uniform(-700, 700, 2000), rng.uniform(-1, 1, 2000), [0.0, 1.0, -1.0]]):
        assert O.series_exp(x) == pytest.approx(math.exp(x), rel=8e-16)
    # the powers the step-size rules and the Arrhenius rate take
    for e in (-0.25, -0.2, 1.0 / 3.0, 2.0 / 3.0):
        for x in 10.0 ** rng.uniform(-12, 6, 500):
            assert O.series_pow(x, e) == pytest.approx(x ** e, rel=4e-15)
    assert O.series_pow(0.0, 1.0 / 3.0) == 0.0
    assert O.series_log(1.0) == 0.0 and O.series_exp(0.0) == 1.0
