"""Pins of the oracle's constant-volume kinetics right-hand side (Section
4.2's T and Y_i equations) on a synthetic 57-species, 766-reaction
mechanism.

Fixed by conservation laws, not by the formulas: the mass fractions' rates
sum to zero and every element is conserved (each reaction balances); the
temperature equation makes the mixture's internal energy sum_i Y_i e_i(T)
constant (closed vessel, no heat loss); a single first-order reaction with
a constant rate has a closed-form solution for Y and for T.  Integrations
keep the linear invariants to rounding and the energy within tolerance.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_02274_gb300 import workloads as W

R = W.R_GAS


def thermo(mech, T):
    a = mech.thermo
    cv = (R / mech.W) * (a[:, 0] + a[:, 1] * T + a[:, 2] * T * T - 1.0)
    e = (R * T / mech.W) * (a[:, 0] + a[:, 1] * T / 2 + a[:, 2] * T * T / 3 + a[:, 3] / T - 1.0)
    return cv, e


def random_states(w, n=6, seed=0):
    """Mixtures of every species at assorted temperatures."""
    rng = np.random.default_rng(seed)
    S = w.neq - 1
    out = []
    for _ in range(n):
        Y = rng.dirichlet(np.ones(S) * 0.3)
        T = rng.uniform(800.0, 2500.0)
        rho = rng.uniform(0.1, 1.0)
        out.append((np.concatenate([[T], Y]), rho))
    return out


@pytest.fixture(scope="module")
def wk():
    return W.kinetics(8, seed=2)


def test_mass_and_elements_are_conserved(wk):
    m, mech = O.model_for(wk), wk.aux["mechanism"]
    for y, rho in random_states(wk):
        f = O.rhs(m, [rho], y)
        dY = f[1:]
        assert abs(dY.sum()) <= 1e-12 * np.abs(dY).sum()
        for e in range(4):
            flux = mech.comp[:, e] * dY / mech.W          # mol of element per kg per s
            assert abs(flux.sum()) <= 1e-12 * np.abs(flux).sum() + 1e-300


def test_temperature_equation_conserves_internal_energy(wk):
    # d/dt sum_i Y_i e_i(T) = sum_i e_i dY_i/dt + c_v dT/dt = 0
    m, mech = O.model_for(wk), wk.aux["mechanism"]
    for y, rho in random_states(wk, seed=1):
        f = O.rhs(m, [rho], y)
        cv_i, e_i = thermo(mech, y[0])
        cv = np.sum(y[1:] * cv_i)
        terms = np.concatenate([e_i * f[1:], [cv * f[0]]])
        assert abs(terms.sum()) <= 1e-10 * np.abs(terms).sum()


def one_reaction_mechanism(k, dh):
    """A -> B with equal weights, constant cp, constant k, formation enthalpies
    differing by dh (in units of R)."""
    Wt = 0.03
    return W.Mechanism(2, np.array([[0, 1, 1, 0], [0, 1, 1, 0]]), np.array([Wt, Wt]),
                       np.array([[3.5, 0.0, 0.0, dh], [3.5, 0.0, 0.0, 0.0]]),
                       np.array([1], np.int32), np.array([[0, -1]], np.int32),
                       np.array([1], np.int32), np.array([[1, -1]], np.int32),
                       np.array([np.log10(k)]), np.array([0.0]), np.array([0.0]), kmin=1e-30, kmax=1e30)


@pytest.mark.parametrize("method", [0, 1])
def test_single_reaction_closed_form(method):
    k, dh, T0, rho, tend = 2.0e4, 3000.0, 1200.0, 0.5, 1e-4
    mech = one_reaction_mechanism(k, dh)
    mod = O.model(O.KIND_KINETICS, 3, 1, mechanism=mech)
    y0 = np.array([[T0], [0.9], [0.1]])
    r = O.integrate(mod, method, y0, np.array([[rho]]), 0.0, tend, 1e-10, 1e-14)
    assert r.status[0] == 0
    YA = 0.9 * np.exp(-k * tend)
    cv = (R / mech.W[0]) * (3.5 - 1.0)
    T = T0 + (R / mech.W[0]) * dh * (0.9 - YA) / cv     # energy: the heat of A -> B warms the gas
    tol = 1e-8 if method == 0 else 1e-6
    np.testing.assert_allclose(r.y[:, 0], [T, YA, 1.0 - YA], rtol=tol)


def test_integration_keeps_invariants(wk):
    m, mech = O.model_for(wk), wk.aux["mechanism"]
    r = O.integrate_workload(wk)
    assert np.all(r.status == 0)
    for i in range(wk.nsys):
        y0, y1 = wk.y0[:, i], r.y[:, i]
        assert abs(y1[1:].sum() - 1.0) <= 1e-12
        for e in range(4):
            z0 = np.sum(mech.comp[:, e] * y0[1:] / mech.W)
            z1 = np.sum(mech.comp[:, e] * y1[1:] / mech.W)
            assert abs(z1 - z0) <= 1e-10 * (abs(z0) + 1.0)
        u0 = np.sum(y0[1:] * thermo(mech, y0[0])[1])
        u1 = np.sum(y1[1:] * thermo(mech, y1[0])[1])
        assert abs(u1 - u0) <= 1e-5 * np.abs(y1[1:] * thermo(mech, y1[0])[1]).sum()


def dcv_dT(mech, T):
    a = mech.thermo
    return (R / mech.W) * (a[:, 1] + 2.0 * a[:, 2] * T)


def test_jacobian_against_central_differences(wk):
    m = O.model_for(wk)
    for y, rho in random_states(wk, n=3, seed=7):
        J = O.jacobian(m, [rho], y)
        fd = np.zeros_like(J)
        for l in range(y.size):
            h = 1e-6 * max(abs(y[l]), 1e-6)
            yp, ym = y.copy(), y.copy()
            yp[l] += h
            ym[l] -= h
            fd[:, l] = (O.rhs(m, [rho], yp) - O.rhs(m, [rho], ym)) / (2.0 * h)
        scale = np.abs(J).max(axis=1)
        live = scale > 0                     # species in no reaction have zero rows
        assert (np.abs(J - fd)[live] / scale[live, None]).max() < 1e-4
        assert np.abs(fd[~live]).max(initial=0.0) == 0.0


def test_jacobian_conserves_mass_elements_and_energy(wk):
    # the invariants hold for every state, so their derivatives vanish:
    # sum_i dY_i/dt = 0, sum_i comp_ie / W_i dY_i/dt = 0 and
    # sum_i e_i dY_i/dt + c_v dT/dt = 0 differentiated by each component
    m, mech = O.model_for(wk), wk.aux["mechanism"]
    for y, rho in random_states(wk, n=4, seed=8):
        J = O.jacobian(m, [rho], y)
        f = O.rhs(m, [rho], y)
        JY = J[1:]
        assert np.abs(JY.sum(axis=0)).max() <= 1e-12 * np.abs(JY).sum(axis=0).max()
        for e in range(4):
            g = (mech.comp[:, e] / mech.W) @ JY
            assert np.abs(g).max() <= 1e-11 * (np.abs(mech.comp[:, e] / mech.W) @ np.abs(JY)).max() + 1e-300
        T, Y = y[0], y[1:]
        cv_i, e_i = thermo(mech, T)
        cv = np.sum(Y * cv_i)
        dcv = np.concatenate([[np.sum(Y * dcv_dT(mech, T))], cv_i])
        total = e_i @ JY + dcv * f[0] + cv * J[0]
        total[0] += np.sum(cv_i * f[1:])                    # de_i/dT = c_v,i
        scale = np.abs(e_i) @ np.abs(JY) + np.abs(dcv * f[0]) + np.abs(cv * J[0])
        scale[0] += np.sum(np.abs(cv_i * f[1:]))
        assert (np.abs(total) / scale).max() < 1e-10


def test_single_reaction_jacobian_closed_form():
    # A -> B, constant k, equal weights, constant heat capacities:
    # dY_A/dt = -k Y_A, dY_B/dt = k Y_A, dT/dt = dh k Y_A / (2.5 (Y_A + Y_B))
    k, dh = 2.0e4, 3000.0
    mech = one_reaction_mechanism(k, dh)
    mod = O.model(O.KIND_KINETICS, 3, 1, mechanism=mech)
    T, ya, yb, rho = 1300.0, 0.7, 0.25, 0.4
    J = O.jacobian(mod, [rho], np.array([T, ya, yb]))
    s = ya + yb
    exact = np.array([[0.0, dh * k / (2.5 * s) - dh * k * ya / (2.5 * s * s), -dh * k * ya / (2.5 * s * s)],
                      [0.0, -k, 0.0],
                      [0.0, k, 0.0]])
    np.testing.assert_allclose(J, exact, rtol=1e-13, atol=1e-9)
    assert O.gershgorin(mod, [rho], np.array([T, ya, yb])) == pytest.approx(np.abs(exact).sum(axis=1).max(), rel=1e-14)


def test_gershgorin_bounds_the_spectrum(wk):
    m = O.model_for(wk)
    for y, rho in random_states(wk, n=3, seed=9):
        J = O.jacobian(m, [rho], y)
        G = O.gershgorin(m, [rho], y)
        assert G == pytest.approx(np.abs(J).sum(axis=1).max(), rel=1e-12)
        assert np.abs(np.linalg.eigvals(J)).max() <= G * (1.0 + 1e-12)


def test_rkc_with_the_gershgorin_bound_follows_the_closed_form():
    k, dh, T0, rho, tend = 2.0e4, 3000.0, 1200.0, 0.5, 1e-4
    mech = one_reaction_mechanism(k, dh)
    mod = O.model(O.KIND_KINETICS, 3, 1, mechanism=mech)
    y0 = np.array([[T0], [0.9], [0.1]])
    r = O.integrate(mod, 1, y0, np.array([[rho]]), 0.0, tend, 1e-10, 1e-14, specrad=O.SPECRAD_GERSHGORIN)
    assert r.status[0] == 0 and r.n_specrad_iter[0] == 0
    YA = 0.9 * np.exp(-k * tend)
    T = T0 + dh * (0.9 - YA) / 2.5
    np.testing.assert_allclose(r.y[:, 0], [T, YA, 1.0 - YA], rtol=1e-6)
