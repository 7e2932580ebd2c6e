"""ctypes front end of the C oracle (test infrastructure only).

Every function here marshals numpy arrays into ``liboracle.so``; all the
arithmetic is in ``ode_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

MAX_REAC = 64
KIND_VDP, KIND_VDP_CHAIN, KIND_BRUSS1D, KIND_MASSACTION, KIND_NBODY, KIND_KINETICS = 1, 2, 3, 4, 5, 6
MAX_BODIES = 16
KIND_LINEAR, KIND_TIME = 100, 101
ST_OK, ST_H_UNDERFLOW, ST_MAX_ATTEMPTS, ST_NONFINITE, ST_SPECRAD_NOCONV = 0, 1, 2, 3, 256
CARRY_FIXED = 9   # warm-restart state: valid, t, h, sigma, h_old, err_old, num_step, sr_step, rejected; then v
CARRY_CONTINUE, CARRY_RESTART = 0, 1
SPECRAD_POWER, SPECRAD_GERSHGORIN, SPECRAD_POWER_CAPPED = 0, 1, 2


def carry_words(neq: int) -> int:
    return CARRY_FIXED + neq


class Model(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("neq", C.c_int32), ("n_params", C.c_int32),
        ("n_species", C.c_int32), ("n_reactions", C.c_int32),
        ("n_reac", C.c_int32 * MAX_REAC), ("reac", (C.c_int32 * 2) * MAX_REAC),
        ("n_prod", C.c_int32 * MAX_REAC), ("prod", (C.c_int32 * 2) * MAX_REAC),
        ("log10A", C.c_double * MAX_REAC), ("beta", C.c_double * MAX_REAC),
        ("Ea", C.c_double * MAX_REAC), ("kmin", C.c_double), ("kmax", C.c_double),
        ("bruss_A", C.c_double), ("bruss_B", C.c_double), ("bruss_ubc", C.c_double),
        ("bruss_vbc", C.c_double), ("coupling", C.c_double), ("masses", C.c_double * MAX_BODIES),
        ("mech", C.c_void_p),
    ]


class Mech(C.Structure):
    """A kinetics mechanism for KIND_KINETICS (pointers into numpy arrays
    that the owning Model keeps alive)."""
    _fields_ = [
        ("n_species", C.c_int32), ("n_reactions", C.c_int32),
        ("W", C.c_void_p), ("thermo", C.c_void_p), ("n_reac", C.c_void_p), ("reac", C.c_void_p),
        ("n_prod", C.c_void_p), ("prod", C.c_void_p), ("log10A", C.c_void_p), ("beta", C.c_void_p),
        ("Ea", C.c_void_p), ("kmin", C.c_double), ("kmax", C.c_double),
    ]


_libs = {}


def lib(libm: bool = False):
    """The oracle library (libm=True: the variant with the C library's
    powers in place of the series of reading R10, for comparison)."""
    if libm not in _libs:
        path = _build.build(libm=libm)
        L = C.CDLL(path)
        P = C.c_void_p
        L.oracle_integrate.argtypes = [P, C.c_int, C.c_int64, P, P, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_int, P, P, P, P, P, P, C.c_int, P, P,
                                       C.c_int, C.c_int]
        L.oracle_jacobian.argtypes = [P, P, P, P]
        L.oracle_gershgorin.argtypes = [P, P, P]
        L.oracle_gershgorin.restype = C.c_double
        L.oracle_integrate_ragged.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, P, P, C.c_int,
                                              P, P, P, P, P, P, C.c_int]
        L.oracle_rhs.argtypes = [P, P, C.c_double, P, P]
        L.oracle_rate_constants.argtypes = [P, C.c_double, P]
        L.oracle_rkck_step.argtypes = [P, P, C.c_double, P, C.c_double, P, P]
        L.oracle_rkc_step.argtypes = [P, P, C.c_double, P, C.c_double, C.c_int, P]
        L.oracle_rkc_coeffs.argtypes = [C.c_int, P, P, P, P, P]
        L.oracle_fixed_steps.argtypes = [P, P, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_int, P, P]
        L.oracle_specrad.argtypes = [P, P, C.c_double, P, C.c_double, P, P, P]
        L.oracle_specrad.restype = C.c_double
        L.oracle_model_size.restype = C.c_int
        for fn in ("oracle_pow", "oracle_exp", "oracle_log"):
            getattr(L, fn).restype = C.c_double
        L.oracle_pow.argtypes = [C.c_double, C.c_double]
        L.oracle_exp.argtypes = [C.c_double]
        L.oracle_log.argtypes = [C.c_double]
        assert L.oracle_model_size() == C.sizeof(Model)
        _libs[libm] = L
    return _libs[libm]


def _p(a: np.ndarray | None):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def model(kind: int, neq: int, n_params: int = 1, network=None, bruss=(1.0, 3.0, 1.0, 3.0),
          coupling: float = 0.1, masses=None, mechanism=None) -> Model:
    assert n_params <= 300, "the oracle stores at most 300 parameters per system"
    m = Model()
    m.kind, m.neq, m.n_params = kind, neq, n_params
    m.bruss_A, m.bruss_B, m.bruss_ubc, m.bruss_vbc = bruss
    m.coupling = coupling
    if mechanism is not None:
        assert kind == KIND_KINETICS and neq == mechanism.n_species + 1
        mk = mechanism
        arrs = {"W": _f64(mk.W), "thermo": _f64(mk.thermo), "n_reac": np.ascontiguousarray(mk.n_reac, np.int32),
                "reac": np.ascontiguousarray(np.where(mk.reac < 0, 0, mk.reac), np.int32),
                "n_prod": np.ascontiguousarray(mk.n_prod, np.int32),
                "prod": np.ascontiguousarray(np.where(mk.prod < 0, 0, mk.prod), np.int32),
                "log10A": _f64(mk.log10A), "beta": _f64(mk.beta), "Ea": _f64(mk.Ea)}
        me = Mech()
        me.n_species, me.n_reactions = mk.n_species, mk.n_reactions
        for k, a in arrs.items():
            setattr(me, k, a.ctypes.data)
        me.kmin, me.kmax = mk.kmin, mk.kmax
        m.mech = C.addressof(me)
        m._keep = (me, arrs)     # the model owns the mechanism's memory
    if masses is not None:
        assert len(masses) <= MAX_BODIES and kind == KIND_NBODY and neq == 4 * len(masses)
        for i, mi in enumerate(masses):
            m.masses[i] = float(mi)
    if network is not None:
        R = network.n_reactions
        assert R <= MAX_REAC
        m.n_species, m.n_reactions = network.n_species, R
        for j in range(R):
            m.n_reac[j] = int(network.n_reac[j])
            m.n_prod[j] = int(network.n_prod[j])
            for q in range(2):
                m.reac[j][q] = int(network.reac[j, q])
                m.prod[j][q] = int(network.prod[j, q])
            m.log10A[j] = float(network.log10A[j])
            m.beta[j] = float(network.beta[j])
            m.Ea[j] = float(network.Ea[j])
        m.kmin, m.kmax = float(network.kmin), float(network.kmax)
    return m


def model_for(w) -> Model:
    """The oracle model of a ``workloads.Workload``."""
    return model(w.kind, w.neq, w.params.shape[0], network=w.network, masses=w.aux.get("masses"),
                 mechanism=w.aux.get("mechanism"))


@dataclass
class Result:
    y: np.ndarray
    n_accept: np.ndarray
    n_reject: np.ndarray
    n_rhs: np.ndarray
    n_specrad_iter: np.ndarray
    status: np.ndarray
    carry: np.ndarray | None = None


def integrate(m: Model, method: int, y0, params, t0: float, tend: float, rtol: float, atol: float,
              max_attempts: int = 1_000_000, nthreads: int = 0, carry_in=None,
              carry_out: bool = False, carry_mode: int = CARRY_CONTINUE,
              specrad: int = SPECRAD_POWER, libm: bool = False) -> Result:
    """Integrate a uniform SoA batch y0[neq, nsys]; method 0 = RKCK, 1 = RKC.
    carry_in (SoA [carry_words(neq), nsys]) resumes a previous call's
    controller state (carry_mode CARRY_CONTINUE or CARRY_RESTART); carry_out
    returns this call's in ``Result.carry``.  specrad: SPECRAD_POWER (the
    Appendix power method), SPECRAD_GERSHGORIN or SPECRAD_POWER_CAPPED."""
    y0 = _f64(y0)
    params = _f64(params)
    nsys = y0.shape[1]
    assert y0.shape[0] == m.neq and params.shape == (m.n_params, nsys)
    y = np.empty_like(y0)
    c = [np.zeros(nsys, dtype=np.int32) for _ in range(5)]
    cin = None if carry_in is None else _f64(carry_in)
    if cin is not None:
        assert cin.shape == (carry_words(m.neq), nsys)
    cout = np.zeros((carry_words(m.neq), nsys)) if carry_out else None
    rc = lib(libm).oracle_integrate(C.byref(m), method, nsys, _p(y0), _p(params), t0, tend, rtol,
                                atol, max_attempts, _p(y), *[_p(a) for a in c], nthreads,
                                _p(cin) if cin is not None else None, _p(cout) if cout is not None else None,
                                carry_mode, specrad)
    if rc != 0:
        raise ValueError(f"oracle_integrate failed ({rc})")
    return Result(y, *c, carry=cout)


def integrate_workload(w, nthreads: int = 0, max_attempts: int = 1_000_000, libm: bool = False) -> Result:
    return integrate(model_for(w), w.method, w.y0, w.params, w.t0, w.tend, w.rtol, w.atol,
                     max_attempts, nthreads, libm=libm)


def integrate_mixed(b, nthreads: int = 0, max_attempts: int = 1_000_000) -> Result:
    """Integrate a ``workloads.MixedBatch`` (ragged, per-system method)."""
    models = (Model * 2)()
    models[0] = model(KIND_BRUSS1D, 0, 1)
    models[1] = model(KIND_VDP_CHAIN, 0, 1, coupling=b.coupling)
    midx = np.where(b.kind == KIND_BRUSS1D, 0, 1).astype(np.int32)
    y = np.empty_like(b.y0)
    nsys = b.nsys
    c = [np.zeros(nsys, dtype=np.int32) for _ in range(5)]
    arrs = [np.ascontiguousarray(b.neq, dtype=np.int32), np.ascontiguousarray(b.offset, dtype=np.int64),
            _f64(b.y0), _f64(b.param), np.ascontiguousarray(b.method, dtype=np.int32), _f64(b.t0),
            _f64(b.tend), _f64(b.rtol), _f64(b.atol)]
    lib().oracle_integrate_ragged(models, _p(midx), nsys, *[_p(a) for a in arrs], max_attempts,
                                  _p(y), *[_p(a) for a in c], nthreads)
    return Result(y, *c)


def jacobian(m: Model, p, y) -> np.ndarray:
    """The oracle's analytic Jacobian df/dy at y, [neq, neq]."""
    p, y = _f64(p), _f64(y)
    J = np.empty((m.neq, m.neq))
    lib().oracle_jacobian(C.byref(m), _p(p), _p(y), _p(J))
    return J


def gershgorin(m: Model, p, y) -> float:
    """The Gershgorin bound max_i sum_j |J_ij| at y."""
    p, y = _f64(p), _f64(y)
    return float(lib().oracle_gershgorin(C.byref(m), _p(p), _p(y)))


def rhs(m: Model, p, y, t: float = 0.0) -> np.ndarray:
    p, y = _f64(p), _f64(y)
    f = np.empty(m.neq)
    lib().oracle_rhs(C.byref(m), _p(p), t, _p(y), _p(f))
    return f


def rate_constants(m: Model, T: float) -> np.ndarray:
    k = np.empty(m.n_reactions)
    lib().oracle_rate_constants(C.byref(m), T, _p(k))
    return k


def rkck_step(m: Model, p, y, h: float, t: float = 0.0):
    p, y = _f64(p), _f64(y)
    yo, ye = np.empty(m.neq), np.empty(m.neq)
    lib().oracle_rkck_step(C.byref(m), _p(p), t, _p(y), h, _p(yo), _p(ye))
    return yo, ye


def rkc_step(m: Model, p, y, h: float, stages: int, t: float = 0.0) -> np.ndarray:
    p, y = _f64(p), _f64(y)
    yo = np.empty(m.neq)
    lib().oracle_rkc_step(C.byref(m), _p(p), t, _p(y), h, stages, _p(yo))
    return yo


def rkc_coeffs(stages: int):
    arrs = [np.zeros(stages + 1) for _ in range(5)]
    lib().oracle_rkc_coeffs(stages, *[_p(a) for a in arrs])
    return dict(zip(("mu", "nu", "mut", "gt", "c"), arrs))


def fixed_steps(m: Model, p, y0, method: int, h: float, nsteps: int, stages: int = 2,
                t0: float = 0.0) -> np.ndarray:
    p, y0 = _f64(p), _f64(y0)
    yo = np.empty(m.neq)
    lib().oracle_fixed_steps(C.byref(m), _p(p), method, stages, t0, h, nsteps, _p(y0), _p(yo))
    return yo


def specrad(m: Model, p, y, hmax: float, v, t: float = 0.0):
    """Returns (1.2 sigma, updated eigenvector v, iterations, status)."""
    p, y = _f64(p), _f64(y)
    v = _f64(v).copy()
    it = np.zeros(1, dtype=np.int32)
    st = np.zeros(1, dtype=np.int32)
    r = lib().oracle_specrad(C.byref(m), _p(p), t, _p(y), hmax, _p(v), _p(it), _p(st))
    return r, v, int(it[0]), int(st[0])


def series_pow(x: float, y: float) -> float:
    return lib().oracle_pow(x, y)


def series_exp(x: float) -> float:
    return lib().oracle_exp(x)


def series_log(x: float) -> float:
    return lib().oracle_log(x)
