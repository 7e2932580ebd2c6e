"""Thin ctypes binding of ``libbatchode.so`` (the C ABI in include/batchode.h).

Argument marshalling only: every integration step runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (their ``data_ptr``);
host arrays (numpy, or pinned torch CPU tensors) are passed with
``io=ODE_IO_HOST``.  There is no CPU fallback: if the library cannot be
built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import workloads as W

ODE_OK = 0
ODE_ERR_ARG, ODE_ERR_HANDLE, ODE_ERR_CUDA, ODE_ERR_UNSUPPORTED, ODE_ERR_NOMEM = -1, -2, -3, -4, -5
ODE_ST_OK, ODE_ST_H_UNDERFLOW, ODE_ST_MAX_ATTEMPTS, ODE_ST_NONFINITE = 0, 1, 2, 3
ODE_ST_SPECRAD_NOCONV = 256
ODE_ST_PROPOSED = 512
MLP_HIDDEN, MLP_MAX_IN, MLP_OUT, MLP_NORM_FLOATS = 64, 33, 3, 138
ODE_RHS_VDP, ODE_RHS_VDP_CHAIN, ODE_RHS_BRUSS1D, ODE_RHS_MASSACTION, ODE_RHS_NBODY, ODE_RHS_KINETICS = 1, 2, 3, 4, 5, 6
ODE_PREC_FP64, ODE_PREC_MIXED, ODE_PREC_MIXED_LEAN, ODE_PREC_F2, ODE_PREC_F2_LEAN = 0, 1, 2, 3, 4
ODE_MAP_AUTO, ODE_MAP_THREAD, ODE_MAP_QUEUE = 0, 1, 2
ODE_IO_DEVICE, ODE_IO_HOST = 0, 1
ODE_CODEGEN_AUTO, ODE_CODEGEN_OFF, ODE_CODEGEN_ON = 0, 1, 2

EXPORTED = ["ode_rhs_register", "ode_rhs_release", "ode_rhs_prepare", "rkck_integrate", "rkc_integrate",
            "rkc_integrate_noalloc", "ode_last_error", "ode_version", "bode_fma_peak", "bode_stoich_bench",
            "ode_mlp_create", "ode_mlp_release", "ode_mlp_num_params", "ode_mlp_fit_normalization",
            "ode_mlp_train", "ode_mlp_gradient", "ode_mlp_apply", "ode_mlp_apply_warp", "ode_mlp_propose", "ode_mlp_get_params",
            "ode_mlp_set_params", "ode_ragged_plan_create", "ode_ragged_plan_launch", "ode_ragged_plan_info",
            "ode_ragged_plan_destroy", "ode_tuning_reset", "ode_cost_order", "ode_cost_order_i32",
            "ode_mapping_info"]
NOALLOC_SCRATCH_BYTES = 16 << 20


class RhsDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("neq", C.c_int32), ("n_params", C.c_int32), ("n_reactions", C.c_int32),
        ("n_reac", C.POINTER(C.c_int32)), ("reac", C.POINTER(C.c_int32)),
        ("n_prod", C.POINTER(C.c_int32)), ("prod", C.POINTER(C.c_int32)),
        ("log10A", C.POINTER(C.c_double)), ("beta", C.POINTER(C.c_double)), ("Ea", C.POINTER(C.c_double)),
        ("kmin", C.c_double), ("kmax", C.c_double),
        ("bruss_A", C.c_double), ("bruss_B", C.c_double), ("bruss_ubc", C.c_double), ("bruss_vbc", C.c_double),
        ("coupling", C.c_double), ("masses", C.POINTER(C.c_double)),
        ("mol_weights", C.POINTER(C.c_double)), ("thermo", C.POINTER(C.c_double)),
    ]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("mapping", C.c_int32), ("max_attempts", C.c_int32),
                ("block_size", C.c_int32), ("io", C.c_int32), ("sync", C.c_int32),
                ("codegen", C.c_int32), ("cost_kind", C.c_int32), ("carry_mode", C.c_int32),
                ("specrad", C.c_int32), ("mlp", C.c_int32), ("log_sr_every", C.c_int32),
                ("log_sr_records", C.c_int32), ("reserved", C.c_int32 * 3),
                ("h0", C.c_void_p), ("sigma0", C.c_void_p), ("log_xy", C.c_void_p), ("cost", C.c_void_p),
                ("carry", C.c_void_p), ("log_sr", C.c_void_p)]


class RaggedBatch(C.Structure):
    _fields_ = [("nsys", C.c_int64), ("rhs", C.c_void_p), ("method", C.c_void_p), ("neq", C.c_void_p),
                ("offset", C.c_void_p), ("y0", C.c_void_p), ("params", C.c_void_p), ("t0", C.c_void_p),
                ("tend", C.c_void_p), ("rtol", C.c_void_p), ("atol", C.c_void_p)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("pad", C.c_int32),
                ("seed", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("n_accept", C.c_void_p), ("n_reject", C.c_void_p), ("n_rhs", C.c_void_p),
                ("n_specrad_iter", C.c_void_p), ("status", C.c_void_p)]


class BatchOdeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"batchode error {code}: {msg}")
        self.code = code


_lib = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbatchode.so")


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libbatchode.so is missing at {path}; the CUDA path cannot run")
    L = C.CDLL(path)
    P = C.c_void_p
    L.ode_rhs_register.argtypes = [C.POINTER(RhsDesc), C.POINTER(C.c_int32)]
    L.ode_rhs_release.argtypes = [C.c_int32]
    L.ode_rhs_prepare.argtypes = [C.c_int32, C.c_int32, C.c_int32]
    for name in ("rkck_integrate", "rkc_integrate", "rkc_integrate_noalloc"):
        fn = getattr(L, name)
        fn.argtypes = [C.c_int32, C.c_int64, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                       C.POINTER(Opts), P, C.POINTER(Stats), P]
    L.ode_last_error.restype = C.c_char_p
    L.ode_version.restype = C.c_char_p
    L.bode_fma_peak.argtypes = [C.c_int, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.bode_stoich_bench.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
    L.ode_ragged_plan_create.argtypes = [C.POINTER(RaggedBatch), C.POINTER(Opts), P, C.POINTER(Stats), P,
                                         C.POINTER(C.c_int64)]
    L.ode_ragged_plan_launch.argtypes = [C.c_int64, P]
    L.ode_ragged_plan_info.argtypes = [C.c_int64, C.POINTER(C.c_int32), P, C.c_int32]
    L.ode_ragged_plan_destroy.argtypes = [C.c_int64]
    L.ode_mlp_create.argtypes = [C.c_int32, C.c_uint64, C.POINTER(C.c_int32)]
    L.ode_mlp_release.argtypes = [C.c_int32]
    L.ode_mlp_num_params.argtypes = [C.c_int32]
    L.ode_mlp_fit_normalization.argtypes = [C.c_int32, P, P, C.c_int64, P]
    L.ode_mlp_train.argtypes = [C.c_int32, P, P, C.c_int64, C.POINTER(TrainOpts), P, P]
    L.ode_mlp_gradient.argtypes = [C.c_int32, P, P, C.c_int64, P, C.POINTER(C.c_float), P]
    L.ode_mlp_apply.argtypes = [C.c_int32, P, C.c_int64, P, P]
    L.ode_mlp_propose.argtypes = [C.c_int32, C.c_int64, C.c_int32, P, P, C.c_float, P, P, P, P]
    L.ode_mlp_get_params.argtypes = [C.c_int32, P, P]
    L.ode_mlp_set_params.argtypes = [C.c_int32, P, P]
    L.ode_cost_order.argtypes = [P, C.c_int64, P, P]
    L.ode_cost_order_i32.argtypes = [P, C.c_int64, P, P]
    L.ode_mapping_info.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P]
    _lib = L
    return L


def _check(rc: int):
    if rc != ODE_OK:
        raise BatchOdeError(rc, load().ode_last_error().decode())


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def register(kind: int, neq: int, network: W.Network | None = None, bruss=(1.0, 3.0, 1.0, 3.0),
             coupling: float = 0.1, masses=None, mechanism: W.Mechanism | None = None) -> int:
    """ode_rhs_register for one family; returns the handle."""
    d = RhsDesc()
    d.kind, d.neq, d.n_params = kind, neq, 1
    d.bruss_A, d.bruss_B, d.bruss_ubc, d.bruss_vbc = bruss
    d.coupling = coupling
    keep = []
    if network is not None:
        arrs = [_i32(network.n_reac), _i32(np.where(network.reac < 0, 0, network.reac).reshape(-1)),
                _i32(network.n_prod), _i32(np.where(network.prod < 0, 0, network.prod).reshape(-1))]
        darrs = [_f64(network.log10A), _f64(network.beta), _f64(network.Ea)]
        keep += arrs + darrs
        d.n_reactions = network.n_reactions
        d.n_reac, d.reac, d.n_prod, d.prod = [a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs]
        d.log10A, d.beta, d.Ea = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in darrs]
        d.kmin, d.kmax = network.kmin, network.kmax
    if mechanism is not None:
        mk = mechanism
        wt, th = _f64(mk.W), _f64(mk.thermo)
        keep += [wt, th]
        d.mol_weights = wt.ctypes.data_as(C.POINTER(C.c_double))
        d.thermo = th.ctypes.data_as(C.POINTER(C.c_double))
        arrs = [_i32(mk.n_reac), _i32(np.where(mk.reac < 0, 0, mk.reac).reshape(-1)),
                _i32(mk.n_prod), _i32(np.where(mk.prod < 0, 0, mk.prod).reshape(-1))]
        darrs = [_f64(mk.log10A), _f64(mk.beta), _f64(mk.Ea)]
        keep += arrs + darrs
        d.n_reactions = mk.n_reactions
        d.n_reac, d.reac, d.n_prod, d.prod = [a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs]
        d.log10A, d.beta, d.Ea = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in darrs]
        d.kmin, d.kmax = mk.kmin, mk.kmax
    if masses is not None:
        mm = _f64(masses)
        keep.append(mm)
        d.masses = mm.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_int32(0)
    _check(load().ode_rhs_register(C.byref(d), C.byref(h)))
    return int(h.value)


def register_workload(w: W.Workload) -> int:
    return register(w.kind, w.neq, network=w.network, masses=w.aux.get("masses"),
                    mechanism=w.aux.get("mechanism"))


def prepare(handle: int, method: str, precision: int = ODE_PREC_FP64):
    """ode_rhs_prepare: compile a mass-action network's generated kernels ahead of time."""
    _check(load().ode_rhs_prepare(handle, 0 if method == "rkck" else 1, precision))


def release(handle: int):
    _check(load().ode_rhs_release(handle))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(x.data_ptr())


@dataclass
class Counters:
    n_accept: object
    n_reject: object
    n_rhs: object
    n_specrad_iter: object
    status: object


def integrate(method: str, handle: int, y0, params, t0: float, tend: float, rtol: float, atol: float,
              y_out=None, counters: Counters | None = None, precision: int = ODE_PREC_FP64,
              mapping: int = ODE_MAP_AUTO, block_size: int = 0, max_attempts: int = 0,
              stream=None, sync: bool = False, codegen: int = ODE_CODEGEN_AUTO, h0=None, sigma0=None,
              log_xy=None, cost=None, carry=None, carry_mode: int = 0, specrad: int = 0, mlp=None,
              log_sr=None, log_sr_every: int = 1):
    """Call rkck_integrate / rkc_integrate.  y0 is [neq, nsys] (torch CUDA
    tensor for device io, numpy array for host io); returns y_out.  log_xy
    rows are [neq + 4]; cost (float32 [nsys], device) orders the batch
    longest-first; carry (float64 [carry_words(neq), nsys], device) is the
    warm-restart state, read and written.  mlp (an MLP or its handle) is
    the network evaluated in-kernel at every spectral-radius point;
    log_sr ([nsys, records, neq + 2] float32, device) the spectral-radius
    training log, every log_sr_every-th estimate."""
    host = isinstance(y0, np.ndarray)
    nsys = int(y0.shape[1])
    if y_out is None:
        y_out = np.empty_like(y0) if host else y0.new_empty(y0.shape)
    o = Opts()
    o.precision, o.mapping, o.block_size, o.max_attempts = precision, mapping, block_size, max_attempts
    o.io = ODE_IO_HOST if host else ODE_IO_DEVICE
    o.sync = 1 if sync else 0
    o.codegen = codegen
    o.h0, o.sigma0, o.log_xy, o.cost, o.carry = _ptr(h0), _ptr(sigma0), _ptr(log_xy), _ptr(cost), _ptr(carry)
    o.cost_kind = 1 if cost is not None and str(getattr(cost, "dtype", "")).endswith("int32") else 0
    o.carry_mode = carry_mode
    o.specrad = specrad
    o.mlp = 0 if mlp is None else int(getattr(mlp, "handle", mlp))
    if log_sr is not None:
        o.log_sr, o.log_sr_every, o.log_sr_records = _ptr(log_sr), log_sr_every, int(log_sr.shape[1])
    s = Stats()
    if counters is not None:
        s.n_accept, s.n_reject, s.n_rhs, s.n_specrad_iter, s.status = [
            _ptr(getattr(counters, k)) for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")]
    if stream is None and not host:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    fn = load().rkck_integrate if method == "rkck" else load().rkc_integrate
    rc = fn(handle, nsys, _ptr(y0), _ptr(params), float(t0), float(tend), float(rtol), float(atol),
            C.byref(o), _ptr(y_out), C.byref(s), C.c_void_p(stream) if stream else None)
    _check(rc)
    return y_out


def integrate_noalloc(handle: int, y0: np.ndarray, params: np.ndarray, t0: float, tend: float, rtol: float,
                      atol: float, y_out: np.ndarray | None = None, counters: Counters | None = None,
                      precision: int = ODE_PREC_FP64, mapping: int = ODE_MAP_AUTO, block_size: int = 0,
                      max_attempts: int = 0, stream=None, specrad: int = 0) -> np.ndarray:
    """rkc_integrate_noalloc on host (numpy) arrays: RKC through a static
    device scratch, with no GPU memory allocated by the library."""
    nsys = int(y0.shape[1])
    if y_out is None:
        y_out = np.empty_like(y0)
    o = Opts()
    o.precision, o.mapping, o.block_size, o.max_attempts = precision, mapping, block_size, max_attempts
    o.specrad = specrad
    s = Stats()
    if counters is not None:
        s.n_accept, s.n_reject, s.n_rhs, s.n_specrad_iter, s.status = [
            _ptr(getattr(counters, k)) for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")]
    rc = load().rkc_integrate_noalloc(handle, nsys, _ptr(y0), _ptr(params), float(t0), float(tend), float(rtol),
                                      float(atol), C.byref(o), _ptr(y_out), C.byref(s),
                                      C.c_void_p(stream) if stream else None)
    _check(rc)
    return y_out


def counters_like(nsys: int, device=None) -> Counters:
    """Per-system counter arrays: torch int32 on ``device`` or numpy on host."""
    if device is None:
        return Counters(*[np.zeros(nsys, dtype=np.int32) for _ in range(5)])
    import torch
    return Counters(*[torch.zeros(nsys, dtype=torch.int32, device=device) for _ in range(5)])


def stoich_bench(handle: int, variant: int, nsys: int, reps: int):
    """bode_stoich_bench: (launch ms, max error vs FP64 relative to the sum
    of |terms|) of the stoichiometry product, variant 0 sparse FP32, 1 TF32
    tensor cores."""
    ms, err = C.c_double(0), C.c_double(float("nan"))
    _check(load().bode_stoich_bench(handle, variant, nsys, reps, C.byref(ms), C.byref(err)))
    return ms.value, err.value


def fma_peak(fp64: bool, iters: int = 1 << 16):
    """Measured FMA-chain throughput of the current device: (GFLOP/s, ms)."""
    g, ms = C.c_double(0), C.c_double(0)
    _check(load().bode_fma_peak(1 if fp64 else 0, iters, C.byref(g), C.byref(ms)))
    return g.value, ms.value


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class MLP:
    """The learned h0 / sigma / cost proposal (ode_mlp_*): inputs are torch
    CUDA tensors, float32, rows contiguous; targets Y are [n, 3] (log h0,
    log sigma, log cost)."""

    def __init__(self, n_in: int, seed: int = 0):
        h = C.c_int32(0)
        _check(load().ode_mlp_create(n_in, seed, C.byref(h)))
        self.handle, self.n_in = int(h.value), n_in
        self.n_params = int(load().ode_mlp_num_params(n_in))

    def release(self):
        if self.handle:
            _check(load().ode_mlp_release(self.handle))
            self.handle = 0

    def fit_normalization(self, X, Y, stream=None):
        _check(load().ode_mlp_fit_normalization(self.handle, _ptr(X), _ptr(Y), int(X.shape[0]), _stream(stream)))

    def train(self, X, Y, epochs: int = 10, batch: int = 4096, lr: float = 1e-3, seed: int = 0, stream=None):
        o = TrainOpts(epochs, batch, lr, 0, seed)
        hist = np.zeros(epochs, dtype=np.float32)
        _check(load().ode_mlp_train(self.handle, _ptr(X), _ptr(Y), int(X.shape[0]), C.byref(o), _ptr(hist),
                                    _stream(stream)))
        return hist

    def gradient(self, X, Y, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = C.c_float(0)
        _check(load().ode_mlp_gradient(self.handle, _ptr(X), _ptr(Y), int(X.shape[0]), _ptr(g), C.byref(loss),
                                       _stream(stream)))
        return g, float(loss.value)

    def apply(self, X, stream=None):
        import torch
        out = torch.empty((X.shape[0], MLP_OUT), dtype=torch.float32, device=X.device)
        _check(load().ode_mlp_apply(self.handle, _ptr(X), int(X.shape[0]), _ptr(out), _stream(stream)))
        return out

    def apply_warp(self, X, stream=None):
        """(log h0, log sigma) [n, 2] as the integration kernels evaluate them in-kernel."""
        import torch
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _check(load().ode_mlp_apply_warp(self.handle, _ptr(X), int(X.shape[0]), _ptr(out), _stream(stream)))
        return out

    def propose(self, y0, params, margin: float = 0.05, stream=None, with_cost: bool = False):
        """(h0, sigma0) or, with_cost, (h0, sigma0, cost) as float32 [nsys]."""
        import torch
        nsys = int(y0.shape[1])
        h0 = torch.empty(nsys, dtype=torch.float32, device=y0.device)
        s0 = torch.empty(nsys, dtype=torch.float32, device=y0.device)
        c = torch.empty(nsys, dtype=torch.float32, device=y0.device) if with_cost else None
        _check(load().ode_mlp_propose(self.handle, nsys, int(y0.shape[0]), _ptr(y0), _ptr(params), margin,
                                      _ptr(h0), _ptr(s0), _ptr(c), _stream(stream)))
        return (h0, s0, c) if with_cost else (h0, s0)

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        nrm = np.zeros(MLP_NORM_FLOATS, dtype=np.float32)
        _check(load().ode_mlp_get_params(self.handle, _ptr(p), _ptr(nrm)))
        return p, nrm

    def set_params(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        n = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        _check(load().ode_mlp_set_params(self.handle, _ptr(p), _ptr(n)))


class RaggedPlan:
    """ode_ragged_plan_*: a workloads.MixedBatch-like ragged batch integrated by
    one CUDA graph.  Host metadata (numpy), device data (torch CUDA tensors)."""

    def __init__(self, handles, method, neq, offset, y0, params, t0, tend, rtol, atol, y_out=None,
                 counters: Counters | None = None, precision: int = ODE_PREC_MIXED_LEAN,
                 mapping: int = ODE_MAP_AUTO, stream=None):
        self._keep = [np.ascontiguousarray(handles, dtype=np.int32), np.ascontiguousarray(method, dtype=np.int32),
                      np.ascontiguousarray(neq, dtype=np.int32), np.ascontiguousarray(offset, dtype=np.int64)]
        self.y_out = y0 if y_out is None else y_out
        self._dev = [y0, params, t0, tend, rtol, atol, self.y_out]
        b = RaggedBatch(len(self._keep[0]), *[_ptr(a) for a in self._keep],
                        *[_ptr(a) for a in (y0, params, t0, tend, rtol, atol)])
        o = Opts()
        o.precision, o.mapping = precision, mapping
        s = Stats()
        if counters is not None:
            self._dev.append(counters)
            s.n_accept, s.n_reject, s.n_rhs, s.n_specrad_iter, s.status = [
                _ptr(getattr(counters, k)) for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")]
        h = C.c_int64(0)
        _check(load().ode_ragged_plan_create(C.byref(b), C.byref(o), _ptr(self.y_out), C.byref(s), _stream(stream),
                                             C.byref(h)))
        self.handle = int(h.value)

    def launch(self, stream=None):
        _check(load().ode_ragged_plan_launch(self.handle, _stream(stream)))

    def info(self):
        n = C.c_int32(0)
        _check(load().ode_ragged_plan_info(self.handle, C.byref(n), None, 0))
        d = np.zeros((max(n.value, 1), 8), dtype=np.int32)
        _check(load().ode_ragged_plan_info(self.handle, C.byref(n), _ptr(d), n.value))
        keys = ("family", "method", "size_class", "systems", "lanes", "points_per_lane", "block", "mapping")
        return [dict(zip(keys, map(int, row))) for row in d[:n.value]]

    def destroy(self):
        if self.handle:
            _check(load().ode_ragged_plan_destroy(self.handle))
            self.handle = 0


CARRY_FIXED = 9
ODE_CARRY_CONTINUE, ODE_CARRY_RESTART = 0, 1
ODE_SPECRAD_POWER, ODE_SPECRAD_GERSHGORIN, ODE_SPECRAD_POWER_CAPPED = 0, 1, 2


def carry_words(neq: int) -> int:
    """Words of warm-restart state per system (ode_opts.carry)."""
    return neq + CARRY_FIXED


def carry_like(neq: int, nsys: int, device="cuda"):
    """A zeroed (cold) warm-restart state for a batch."""
    import torch
    return torch.zeros((carry_words(neq), nsys), dtype=torch.float64, device=device)


def cost_order(cost, stream=None):
    """Longest-first order (int32 torch tensor) of a float32 or int32 CUDA cost vector."""
    import torch
    idx = torch.empty(int(cost.shape[0]), dtype=torch.int32, device=cost.device)
    fn = load().ode_cost_order_i32 if cost.dtype == torch.int32 else load().ode_cost_order
    _check(fn(_ptr(cost), int(cost.shape[0]), _ptr(idx), _stream(stream)))
    return idx


def mapping_info(handle: int, method: str, precision: int, codegen: int = ODE_CODEGEN_AUTO, block_size: int = 0):
    """(mapping, block, tuned) that ODE_MAP_AUTO uses for these options."""
    m, b = C.c_int32(0), C.c_int32(0)
    rc = load().ode_mapping_info(handle, 0 if method == "rkck" else 1, precision, codegen, block_size,
                                 C.byref(m), C.byref(b))
    if rc not in (ODE_OK, ODE_ERR_UNSUPPORTED):
        _check(rc)
    return int(m.value), int(b.value), rc == ODE_OK


def tuning_reset() -> None:
    """Forget cached ODE_MAP_AUTO timings (uniform calls and ragged plans)."""
    _check(load().ode_tuning_reset())


def version() -> str:
    return load().ode_version().decode()
