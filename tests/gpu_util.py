"""Helpers shared by the GPU parity tests: run a workload through the C ABI
and compare with the oracle system by system."""
from __future__ import annotations

import numpy as np

from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W


def run_gpu(w: W.Workload, precision=B.ODE_PREC_FP64, mapping=B.ODE_MAP_AUTO, method=None,
            max_attempts=0, block_size=0, codegen=B.ODE_CODEGEN_AUTO):
    import torch
    dev = torch.device("cuda:0")
    h = B.register_workload(w)
    try:
        y0 = torch.from_numpy(np.ascontiguousarray(w.y0)).to(dev)
        p = torch.from_numpy(np.ascontiguousarray(w.params)).to(dev)
        cnt = B.counters_like(w.nsys, dev)
        m = method or ("rkck" if w.method == W.METHOD_RKCK else "rkc")
        y = B.integrate(m, h, y0, p, w.t0, w.tend, w.rtol, w.atol, counters=cnt, precision=precision,
                        mapping=mapping, max_attempts=max_attempts, block_size=block_size, sync=True,
                        codegen=codegen)
        torch.cuda.synchronize()
        out = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        out["y"] = y.cpu().numpy()
        return out
    finally:
        B.release(h)


def rel_err(y, ref, atol):
    """Per-system max_i |y_i - ref_i| / (|ref_i| + atol)."""
    return (np.abs(y - ref) / (np.abs(ref) + atol)).max(axis=0)


def same_counts(g, ref):
    return (g["n_accept"] == ref.n_accept) & (g["n_reject"] == ref.n_reject)


def summary(g, ref, atol):
    e = rel_err(g["y"], ref.y, atol)
    s = same_counts(g, ref)
    return dict(max=float(e.max()), p999=float(np.quantile(e, 0.999)), same_counts=float(s.mean()),
                max_same=float(e[s].max()) if s.any() else float("nan"))
