"""Pins of the oracle's Jacobians and Gershgorin spectral-radius bound (the
Appendix names the circle theorem as an upper-bound alternative to the
power method).

Each analytic Jacobian is checked against central differences of the
oracle's own right-hand side; the bound against the eigenvalues numpy finds
(it must never be below the spectral radius) and against cases where it is
exact; and the integrator's use of it (GERSHGORIN: no power iterations;
POWER_CAPPED: the power method's 1.2 sigma never above the bound).
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import workloads as W


def fd_jacobian(m, p, y, rel=1e-6):
    n = y.size
    J = np.empty((n, n))
    for j in range(n):
        h = rel * max(abs(y[j]), 1e-3)
        yp, ym = y.copy(), y.copy()
        yp[j] += h
        ym[j] -= h
        J[:, j] = (O.rhs(m, p, yp) - O.rhs(m, p, ym)) / (2 * h)
    return J


def cases():
    rng = np.random.default_rng(3)
    out = []
    w = W.vdp(4, seed=1)
    out += [("vdp", O.model_for(w), w.params[:, i], w.y0[:, i]) for i in range(4)]
    m = O.model(O.KIND_VDP_CHAIN, 10, 1, coupling=0.1)
    out += [("chain", m, np.array([rng.uniform(0.1, 5)]), rng.uniform(-2, 2, 10)) for _ in range(3)]
    w = W.bruss(3, n=6, seed=2)
    out += [("bruss", O.model_for(w), w.params[:, i], w.y0[:, i]) for i in range(3)]
    w = W.massaction(4, seed=5)
    out += [("mass", O.model_for(w), w.params[:, i], w.y0[:, i]) for i in range(4)]
    w = W.pleiades(3, seed=6)
    out += [("nbody", O.model_for(w), w.params[:, i], w.y0[:, i]) for i in range(3)]
    return out


@pytest.mark.parametrize("name,m,p,y", cases())
def test_jacobian_matches_central_differences(name, m, p, y):
    J = O.jacobian(m, p, y)
    Jfd = fd_jacobian(m, p, y)
    scale = np.abs(J).max(axis=1, keepdims=True) + 1e-300
    assert np.all(np.abs(J - Jfd) <= 1e-5 * scale), name
    # entries that are structurally zero stay exactly zero
    assert np.all(J[np.abs(Jfd) == 0.0] == 0.0)


@pytest.mark.parametrize("name,m,p,y", cases())
def test_bound_is_max_row_sum_and_covers_every_eigenvalue(name, m, p, y):
    J = O.jacobian(m, p, y)
    G = O.gershgorin(m, p, y)
    # the row sums run left to right (numpy's sum pairs terms up and
    # Python's compensates, so the reference is an explicit loop)
    def seq_sum(row):
        acc = 0.0
        for v in row:
            acc = acc + abs(float(v))
        return acc

    assert G == max(seq_sum(row) for row in J)
    rho = np.abs(np.linalg.eigvals(J)).max()
    assert G >= rho * (1 - 1e-12), (name, G, rho)


def test_bound_is_exact_for_a_diagonal_matrix():
    A = np.diag([-1.0, -7.5, -300.0, 2.0])
    m = O.model(O.KIND_LINEAR, 4, 16)
    assert O.gershgorin(m, A.ravel(), np.ones(4)) == 300.0


def test_bound_of_the_laplacian():
    # tridiagonal (1, -2, 1) D: interior rows sum to 4 D, the spectral
    # radius 4 D sin^2(n pi / (2 (n + 1))) approaches it from below
    n, D = 16, 3.0   # n^2 parameters: the oracle stores at most 300
    L = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) * D
    m = O.model(O.KIND_LINEAR, n, n * n)
    G = O.gershgorin(m, L.ravel(), np.ones(n))
    assert G == 4 * D
    # a model too large for the parameter store is refused, not read past
    big = O.model(O.KIND_LINEAR, 18, 300)
    assert np.isnan(O.gershgorin(big, np.zeros(300), np.ones(18)))
    rho = 4 * D * np.sin(n * np.pi / (2 * (n + 1))) ** 2
    assert rho < G < 1.01 * rho


def test_rkc_with_the_bound_needs_no_power_iterations():
    from scipy.linalg import expm
    M = np.array([[-1.0, 0.5], [0.0, -800.0]])
    y0 = np.array([1.0, 2.0])
    m = O.model(O.KIND_LINEAR, 2, 4)
    r = O.integrate(m, 1, y0[:, None], M.ravel()[:, None], 0.0, 2.0, 1e-6, 1e-9,
                    specrad=O.SPECRAD_GERSHGORIN, carry_out=True)
    assert r.status[0] == 0 and r.n_specrad_iter[0] == 0
    assert r.carry[3, 0] == 800.0                        # sigma = the bound, max(1 + 0.5, 0 + 800)
    exact = expm(2.0 * M) @ y0
    assert abs(r.y[0, 0] / exact[0] - 1.0) < 2.0 * 1e-6 ** (2.0 / 3.0)


def test_capped_power_method_never_exceeds_the_bound():
    # diagonal: the power method finds 300 and adds its 20 % margin, the
    # bound is exactly 300
    A = np.diag([-1.0, -20.0, -300.0])
    m = O.model(O.KIND_LINEAR, 3, 9)
    y0 = np.array([[1.0], [1.0], [1.0]])
    plain = O.integrate(m, 1, y0, A.ravel()[:, None], 0.0, 1.0, 1e-6, 1e-9, carry_out=True)
    capped = O.integrate(m, 1, y0, A.ravel()[:, None], 0.0, 1.0, 1e-6, 1e-9, carry_out=True,
                         specrad=O.SPECRAD_POWER_CAPPED)
    assert plain.carry[3, 0] > 300.0
    assert capped.carry[3, 0] == 300.0
    assert capped.n_specrad_iter[0] == plain.n_specrad_iter[0]


def test_gershgorin_mode_on_the_network_workload():
    # the bound is looser than the power method: more stages, no iterations
    w = W.massaction(64, seed=8)
    m = O.model_for(w)
    p = O.integrate(m, 1, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol)
    g = O.integrate(m, 1, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol, specrad=O.SPECRAD_GERSHGORIN)
    assert np.all((g.status & 0xFF) == 0) and np.all(g.n_specrad_iter == 0)
    e = np.abs(g.y - p.y) / (np.abs(p.y) + w.atol)
    assert np.quantile(e, 0.99) < 1e-3
