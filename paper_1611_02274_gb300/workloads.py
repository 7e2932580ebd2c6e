"""Seeded synthetic workloads for batched ODE integration.

This module only draws random inputs (initial conditions, per-system
parameters, the shared mass-action network) with numpy's PCG64.  It holds
none of the integrators' arithmetic: rate constants, stencils, stage
combinations and error norms are computed by the consumers (the CUDA library
and the CPU oracle), each in its own code.

Layout is the structure-of-arrays layout of the paper's Section 3 (Source
Code): unknown ``j`` of system ``i`` sits at ``y[j, i]`` (C order, i.e. the
flat index ``i + nsys * j``), so neighbouring systems are neighbouring in
memory.  Parameters use the same layout, ``params[p, i]``.

Workload recipes (all FP64, generated on the host):

* ``vdp``        van der Pol, N=2, mu = 10**U(-1, 1), y0 ~ U[-2, 2]^2,
                 t in [0, 20], rtol 1e-6, atol 1e-9.
* ``bruss``      1D Brusselator with n interior points (N = 2n),
                 diffusion a = 10**U(log10 .01, log10 .05),
                 u = 1 + sin(2 pi x_k) + U(-.1, .1), v = 3 + U(-.1, .1),
                 t in [0, 10], rtol 1e-5, atol 1e-8.
* ``massaction`` one network shared by the batch: 13 species, 27 reactions,
                 1-2 reactants and 1-2 products each (species drawn uniformly
                 with replacement), log10 A ~ U[6, 14], b ~ U[-1, 1],
                 Ea ~ U[0, 20000] K; per system T ~ U[1000, 2000] K and
                 concentrations U(0, 1] normalised to sum 1;
                 t in [0, 1e-4], rtol 1e-6, atol 1e-12.
* ``mixed``      ragged batch: half Brusselator grids with n ~ U{1..128},
                 half coupled van der Pol chains with n ~ U{1..64}
                 oscillators, shuffled.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Registered right-hand-side kinds (mirrors the C-ABI enumeration).
RHS_VDP = 1
RHS_VDP_CHAIN = 2
RHS_BRUSS1D = 3
RHS_MASSACTION = 4
RHS_NBODY = 5
RHS_KINETICS = 6

R_GAS = 8.314462618  # J / (mol K)

METHOD_RKCK = 0
METHOD_RKC = 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Network:
    """A mass-action reaction network: reactant/product species per reaction
    (-1 marks an unused slot) and Arrhenius parameters."""

    n_species: int
    n_reac: np.ndarray      # int32 [R]   1 or 2
    reac: np.ndarray        # int32 [R,2] species index or -1
    n_prod: np.ndarray      # int32 [R]
    prod: np.ndarray        # int32 [R,2]
    log10A: np.ndarray      # f64 [R]
    beta: np.ndarray        # f64 [R]
    Ea: np.ndarray          # f64 [R]  (Kelvin; k = A T^b exp(-Ea/T))
    kmin: float = 1e-2
    kmax: float = 1e6

    @property
    def n_reactions(self) -> int:
        return int(self.n_reac.shape[0])


@dataclass
class Workload:
    name: str
    kind: int
    method: int
    nsys: int
    neq: int
    y0: np.ndarray          # f64 [neq, nsys]
    params: np.ndarray      # f64 [n_params, nsys]
    t0: float
    tend: float
    rtol: float
    atol: float
    network: Network | None = None
    bruss_n: int = 0
    aux: dict = field(default_factory=dict)


def make_network(seed: int = 0, n_species: int = 13, n_reactions: int = 27) -> Network:
    """Draw the shared mass-action network from ``seed``."""
    rng = _rng(seed)
    n_reac = rng.integers(1, 3, size=n_reactions).astype(np.int32)
    n_prod = rng.integers(1, 3, size=n_reactions).astype(np.int32)
    reac = rng.integers(0, n_species, size=(n_reactions, 2)).astype(np.int32)
    prod = rng.integers(0, n_species, size=(n_reactions, 2)).astype(np.int32)
    reac[n_reac == 1, 1] = -1
    prod[n_prod == 1, 1] = -1
    log10A = rng.uniform(6.0, 14.0, size=n_reactions)
    beta = rng.uniform(-1.0, 1.0, size=n_reactions)
    Ea = rng.uniform(0.0, 20000.0, size=n_reactions)
    return Network(n_species, n_reac, reac, n_prod, prod, log10A, beta, Ea)


def vdp(nsys: int = 4096, seed: int = 0) -> Workload:
    rng = _rng(seed)
    mu = 10.0 ** rng.uniform(-1.0, 1.0, size=nsys)
    y0 = rng.uniform(-2.0, 2.0, size=(2, nsys))
    return Workload("vdp", RHS_VDP, METHOD_RKCK, nsys, 2, np.ascontiguousarray(y0),
                    mu[None, :].copy(), 0.0, 20.0, 1e-6, 1e-9)


@dataclass
class Mechanism:
    """A closed constant-volume gas mechanism (Section 4.2's form): species
    with element counts (C, H, O, N) and molecular weights, polynomial
    thermodynamics cp/R = a0 + a1 T + a2 T^2 and h/(R T) = a0 + a1 T / 2
    + a2 T^2 / 3 + a3 / T, and irreversible reactions (1-2 reactants and
    products, mass and element balanced) with Arrhenius constants
    k = clip(10^log10A T^beta exp(-Ea / T), kmin, kmax) (Ea in Kelvin)."""

    n_species: int
    comp: np.ndarray        # int [S, 4]
    W: np.ndarray           # f64 [S] kg/mol
    thermo: np.ndarray      # f64 [S, 4] (a0, a1, a2, a3)
    n_reac: np.ndarray      # int32 [R]
    reac: np.ndarray        # int32 [R, 2]
    n_prod: np.ndarray      # int32 [R]
    prod: np.ndarray        # int32 [R, 2]
    log10A: np.ndarray
    beta: np.ndarray
    Ea: np.ndarray
    kmin: float = 1e-2
    kmax: float = 1e7

    @property
    def n_reactions(self) -> int:
        return int(self.n_reac.size)


ELEMENT_W = np.array([12.011e-3, 1.008e-3, 15.999e-3, 14.007e-3])  # C, H, O, N in kg/mol


def make_mechanism(seed: int = 0, n_species: int = 57, n_reactions: int = 766) -> Mechanism:
    """A synthetic mechanism of the size of the paper's ethanol case (57
    species, 766 irreversible reactions): species are C/H/O compositions
    (up to 2 C, 6 H, 3 O, at most 8 atoms, smallest first) plus inert N2;
    each reaction takes 1-2 reactants and recombines their atoms into 1-2
    other species (so mass and elements balance); Arrhenius constants are
    drawn so the clipped rates give a moderately stiff system; formation
    enthalpies favour oxygenated products (exothermic oxidation)."""
    rng = _rng(seed)
    cand = [(c, h, o, 0) for c in range(3) for h in range(7) for o in range(4)
            if 0 < c + h + o <= 8]
    cand.sort(key=lambda x: (sum(x), x))
    comp = cand[:n_species - 1] + [(0, 0, 0, 2)]  # N2 last, inert
    comp = np.array(comp, dtype=np.int64)
    S = len(comp)
    W = comp @ ELEMENT_W
    atoms = comp[:, :3].sum(axis=1)
    thermo = np.zeros((S, 4))
    thermo[:, 0] = 2.5 + 0.8 * (atoms - 1) + rng.uniform(0.0, 0.5, S)   # cp/R at low T
    thermo[:, 1] = rng.uniform(0.0, 4e-4, S) * (atoms > 1)               # mild rise with T
    thermo[:, 2] = -rng.uniform(0.0, 5e-8, S) * (atoms > 1)
    # formation enthalpy / R: oxygen-bearing molecules lower, radicals higher
    thermo[:, 3] = -6000.0 * comp[:, 2] + 2500.0 * (comp[:, 1] % 2) + rng.uniform(-2000.0, 2000.0, S)
    thermo[S - 1, 3] = 0.0
    by_comp = {}
    for i in range(S - 1):
        by_comp.setdefault(tuple(comp[i]), []).append((i,))
    for i in range(S - 1):
        for j in range(i, S - 1):
            by_comp.setdefault(tuple(comp[i] + comp[j]), []).append((i, j))
    reac, prod = [], []
    while len(reac) < n_reactions:
        nr = 1 if rng.random() < 0.25 else 2
        rs = tuple(sorted(rng.integers(0, S - 1, size=nr).tolist()))
        total = tuple(comp[list(rs)].sum(axis=0))
        opts = [q for q in by_comp.get(total, []) if tuple(sorted(q)) != rs]
        if not opts:
            continue
        ps = opts[rng.integers(len(opts))]
        reac.append(list(rs) + [-1] * (2 - len(rs)))
        prod.append(list(ps) + [-1] * (2 - len(ps)))
    reac, prod = np.array(reac, np.int32), np.array(prod, np.int32)
    R = n_reactions
    return Mechanism(S, comp, W, thermo, (reac >= 0).sum(axis=1).astype(np.int32), reac,
                     (prod >= 0).sum(axis=1).astype(np.int32), prod,
                     rng.uniform(4.0, 9.0, R), rng.uniform(-0.5, 0.5, R), rng.uniform(0.0, 15000.0, R))


def kinetics(nsys: int = 16384, seed: int = 0, mech_seed: int = 0, tend: float = 1e-5) -> Workload:
    """Constant-volume ignition-like batches (Section 4.2's form): state
    (T, Y_1..Y_S), fuel (the largest C2 species with O) / O2 / N2 mixtures
    with mass fractions varied per system, T0 ~ U[1000, 1300] K at 1 atm;
    the density (constant in a closed vessel) is the system's parameter.
    The paper integrates 10 global steps of 1e-6 s."""
    mech = make_mechanism(mech_seed)
    S = mech.n_species
    rng = _rng(seed)
    fuel = max((i for i in range(S - 1) if mech.comp[i, 0] == 2 and mech.comp[i, 2] >= 1),
               key=lambda i: (mech.comp[i].sum(), i))
    o2 = next(i for i in range(S) if tuple(mech.comp[i]) == (0, 0, 2, 0))
    n2 = S - 1
    Y = np.zeros((S, nsys))
    yf = rng.uniform(0.03, 0.08, nsys)
    yo = rng.uniform(0.18, 0.23, nsys)
    Y[fuel], Y[o2], Y[n2] = yf, yo, 1.0 - yf - yo
    T0 = rng.uniform(1000.0, 1300.0, nsys)
    Wmix = 1.0 / np.sum(Y / mech.W[:, None], axis=0)
    rho = 101325.0 * Wmix / (R_GAS * T0)
    y0 = np.concatenate([T0[None, :], Y], axis=0)
    return Workload("kinetics", RHS_KINETICS, METHOD_RKC, nsys, S + 1, np.ascontiguousarray(y0),
                    rho[None, :].copy(), 0.0, tend, 1e-6, 1e-10, aux={"mechanism": mech})


def pleiades_base(n: int = 7, base_seed: int = 0):
    """A planar n-body configuration of the Pleiades problem's shape (masses
    1..n, G = 1): bodies spread around a ring of radius 1.5-3.5 with roughly
    bound tangential velocities, pairwise separations at least 0.8, zero
    total momentum.  Returns (masses, state [x.., y.., u.., v..])."""
    rng = _rng(base_seed)
    m = np.arange(1, n + 1, dtype=np.float64)
    while True:
        ang = 2 * np.pi * np.arange(n) / n + rng.uniform(-0.3, 0.3, n)
        rad = rng.uniform(1.5, 3.5, n)
        x, y = rad * np.cos(ang), rad * np.sin(ang)
        d = np.hypot(x[:, None] - x[None, :], y[:, None] - y[None, :]) + np.eye(n) * 1e9
        if d.min() >= 0.8:
            break
    speed = 0.5 * np.sqrt(m.sum() / rad) * rng.uniform(0.8, 1.2, n)
    u, v = -speed * np.sin(ang), speed * np.cos(ang)
    u -= (m * u).sum() / m.sum()
    v -= (m * v).sum() / m.sum()
    return m, np.concatenate([x, y, u, v])


def pleiades(nsys: int = 262144, seed: int = 0, n: int = 7, perturb: float = 1e-3,
             tend: float = 1.0) -> Workload:
    """Copies of one n-body configuration (pleiades_base) with perturbed
    initial states (each component + perturb * N(0, 1), the paper's
    perturbed-IC batch), integrated by RKCK with eps = 1e-10 over [0, tend]."""
    m, base = pleiades_base(n)
    rng = _rng(seed)
    y0 = base[:, None] + perturb * rng.standard_normal((4 * n, nsys))
    G = np.ones((1, nsys))
    return Workload("pleiades", RHS_NBODY, METHOD_RKCK, nsys, 4 * n, np.ascontiguousarray(y0), G,
                    0.0, tend, 1e-10, 1e-10, aux={"masses": m})


def bruss(nsys: int = 65536, n: int = 32, seed: int = 0) -> Workload:
    rng = _rng(seed)
    a = 10.0 ** rng.uniform(np.log10(0.01), np.log10(0.05), size=nsys)
    x = np.arange(1, n + 1, dtype=np.float64) / (n + 1)
    u = 1.0 + np.sin(2.0 * np.pi * x)[:, None] + rng.uniform(-0.1, 0.1, size=(n, nsys))
    v = 3.0 + rng.uniform(-0.1, 0.1, size=(n, nsys))
    y0 = np.ascontiguousarray(np.concatenate([u, v], axis=0))
    return Workload("bruss", RHS_BRUSS1D, METHOD_RKC, nsys, 2 * n, y0,
                    a[None, :].copy(), 0.0, 10.0, 1e-5, 1e-8, bruss_n=n)


def massaction(nsys: int = 1 << 20, seed: int = 0, network_seed: int = 0,
               tend: float = 1e-4) -> Workload:
    net = make_network(network_seed)
    rng = _rng(seed)
    T = rng.uniform(1000.0, 2000.0, size=nsys)
    c = 1.0 - rng.uniform(0.0, 1.0, size=(net.n_species, nsys))   # U(0, 1]
    c = c / c.sum(axis=0, keepdims=True)
    return Workload("massaction", RHS_MASSACTION, METHOD_RKC, nsys, net.n_species,
                    np.ascontiguousarray(c), T[None, :].copy(), 0.0, tend, 1e-6, 1e-12,
                    network=net)


@dataclass
class MixedBatch:
    """Ragged batch.  System i has kind[i] (RHS_BRUSS1D or RHS_VDP_CHAIN),
    n[i] grid points / oscillators, neq[i] = 2 n[i] unknowns stored
    contiguously at y0[offset[i] : offset[i] + neq[i]] (unknown-major within
    a system), one scalar parameter param[i] (a or mu), and method[i]
    (RKC for Brusselator grids, RKCK for chains)."""

    nsys: int
    kind: np.ndarray
    n: np.ndarray
    neq: np.ndarray
    offset: np.ndarray      # int64 [nsys + 1]
    y0: np.ndarray          # f64 [total]
    param: np.ndarray       # f64 [nsys]
    method: np.ndarray
    t0: np.ndarray
    tend: np.ndarray
    rtol: np.ndarray
    atol: np.ndarray
    coupling: float = 0.1


def mixed(nsys: int = 262144, seed: int = 0, max_bruss_n: int = 128,
          max_chain_n: int = 64) -> MixedBatch:
    rng = _rng(seed)
    half = nsys // 2
    kind = np.concatenate([np.full(half, RHS_BRUSS1D), np.full(nsys - half, RHS_VDP_CHAIN)])
    rng.shuffle(kind)
    kind = kind.astype(np.int32)
    is_b = kind == RHS_BRUSS1D
    n = np.where(is_b, rng.integers(1, max_bruss_n + 1, size=nsys),
                 rng.integers(1, max_chain_n + 1, size=nsys)).astype(np.int32)
    neq = (2 * n).astype(np.int32)
    offset = np.zeros(nsys + 1, dtype=np.int64)
    np.cumsum(neq, out=offset[1:])
    a = 10.0 ** rng.uniform(np.log10(0.01), np.log10(0.05), size=nsys)
    mu = 10.0 ** rng.uniform(-1.0, 1.0, size=nsys)
    param = np.where(is_b, a, mu)
    y0 = np.empty(int(offset[-1]), dtype=np.float64)
    noise = rng.uniform(-0.1, 0.1, size=int(offset[-1]))
    chain_ic = rng.uniform(-2.0, 2.0, size=int(offset[-1]))
    for i in range(nsys):
        o, k = int(offset[i]), int(n[i])
        if is_b[i]:
            x = np.arange(1, k + 1, dtype=np.float64) / (k + 1)
            y0[o:o + k] = 1.0 + np.sin(2.0 * np.pi * x) + noise[o:o + k]
            y0[o + k:o + 2 * k] = 3.0 + noise[o + k:o + 2 * k]
        else:
            y0[o:o + 2 * k] = chain_ic[o:o + 2 * k]
    method = np.where(is_b, METHOD_RKC, METHOD_RKCK).astype(np.int32)
    t0 = np.zeros(nsys)
    tend = np.where(is_b, 10.0, 20.0)
    rtol = np.where(is_b, 1e-5, 1e-6)
    atol = np.where(is_b, 1e-8, 1e-9)
    return MixedBatch(nsys, kind, n, neq, offset, y0, param, method, t0, tend, rtol, atol)


def subset(w: Workload, idx: np.ndarray) -> Workload:
    """The same workload restricted to systems ``idx`` (SoA columns)."""
    idx = np.asarray(idx)
    return Workload(w.name, w.kind, w.method, int(idx.size), w.neq,
                    np.ascontiguousarray(w.y0[:, idx]), np.ascontiguousarray(w.params[:, idx]),
                    w.t0, w.tend, w.rtol, w.atol, w.network, w.bruss_n, dict(w.aux))


def mixed_subset(b: MixedBatch, idx: np.ndarray) -> MixedBatch:
    """The ragged batch restricted to systems ``idx`` (states repacked)."""
    idx = np.asarray(idx)
    neq = b.neq[idx].astype(np.int32)
    offset = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(neq, out=offset[1:])
    y0 = np.concatenate([b.y0[b.offset[i]:b.offset[i] + b.neq[i]] for i in idx]) if idx.size else np.empty(0)
    return MixedBatch(int(idx.size), b.kind[idx].copy(), b.n[idx].copy(), neq, offset, y0, b.param[idx].copy(),
                      b.method[idx].copy(), b.t0[idx].copy(), b.tend[idx].copy(), b.rtol[idx].copy(),
                      b.atol[idx].copy(), b.coupling)

