"""Benchmark: batched RKC integration of the synthetic mass-action workload.

Workload (one step = one pass of the whole hot path over one batch): the
seeded 13-species / 27-reaction mass-action network, 1,048,576 systems per
GPU, T ~ U[1000, 2000] K, t in [0, 1e-4], rtol 1e-6, atol 1e-12, integrated
by RKC through the C ABI.  The metric is ODE systems integrated per second
by the chosen form (generated network code; FP32 stages, step size and
norms with Kahan-compensated state and the remaining interval as an FP32
pair; thread or queue mapping picked by ODE_MAP_AUTO); the plain FP64 form
is timed beside it on the same inputs, and the CPU oracle on a bounded
sample.  Further legs time the learned proposal, ragged batches, the
spectral-radius modes, the outer global-step loop, the n-body and the
kinetics families.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 run under torch.distributed.run: every rank integrates its own
batch (seed = rank), no collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1611_02274_gb300 import workloads as W  # noqa: E402

NSYS = 1 << 20
METRIC = "ODE systems integrated/s at rtol 1e-6, chosen vs plain FP64 form; % of FP peak"
UNIT = "systems/s"
# nominal ALU peaks from unit counts and the maximum SM clock (152 SMs, 2070 MHz):
# FP32 128 lanes x 2 flops per SM per clock; FP64 the part's rated 1.25 TFLOP/s
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) per system of the chosen kernel, from one ncu
# capture of k_static<RkcMixed<JitMass, false>> (step-end hold, stage points
# without the compensation word) on 262,144 systems of this workload
# (29.883 MB read + 0.899 MB written); traffic grows with the number of
# systems (each state is read once, written once)
NCU_TRAFFIC_BYTES_PER_SYSTEM = (29.88288e6 + 0.89856e6) / 262144


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's x (a step time: the job is as slow as its
    slowest rank); x itself on one rank.  device holds the reduction
    tensor: the rank's GPU under NCCL, the CPU under gloo."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed (each rank its
    own batch of units_per_rank, weak scaling) over the slowest rank's step
    time in milliseconds."""
    return units_per_rank * world / (ms * 1e-3)


# ------------------------------------------------------------ flop accounting

def rhs_flops(w: W.Workload) -> int:
    """Algorithmic flops of one mass-action RHS: per reaction |R| products
    (rate constant times concentrations) and |R| + |P| accumulations."""
    n = w.network
    return int(np.sum(2 * n.n_reac + n.n_prod))


def rkc_flops(w: W.Workload, n_acc, n_rej, n_rhs, n_sr) -> float:
    """Algorithmic flops of RKC runs from the per-system counters: every RHS
    evaluation, plus per attempt N (2 + 9 (m - 1) + 11) vector flops, per
    power iteration 6 N and 8 N for the initial step (FMA = 2 flops)."""
    N = w.neq
    A = n_acc.astype(np.float64) + n_rej
    sum_m = n_rhs.astype(np.float64) - n_sr - 2.0      # minus F(t0) and the initial trial step
    vec = N * (13.0 * A + 9.0 * (sum_m - A)) + 6.0 * N * n_sr + 8.0 * N
    return float(np.sum(n_rhs.astype(np.float64) * rhs_flops(w) + vec))


# ------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1611_02274_gb300 import binding as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = W.massaction(nsys=args.nsys, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    yout = torch.empty_like(y0)
    cnt = B.counters_like(w.nsys, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    MAPPING = {"auto": B.ODE_MAP_AUTO, "thread": B.ODE_MAP_THREAD, "queue": B.ODE_MAP_QUEUE}[args.mapping]

    def step(prec, counters=None):
        B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=yout, counters=counters,
                    precision=prec, mapping=MAPPING, block_size=args.block, stream=stream.cuda_stream)

    CHOSEN = B.ODE_PREC_MIXED_LEAN
    for prec in (CHOSEN, B.ODE_PREC_MIXED, B.ODE_PREC_FP64):
        B.prepare(h, "rkc", prec)       # generated network kernels compiled before any timing

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize()
        evs = []
        barrier()
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()                       # L2 flush between timed iterations
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        total = sum(ms)
        total = max_over_ranks(total, world, dev)
        return total / steps, ms

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None

    # chosen form: timed with the clock sampler running
    with ClockSampler(gpu_id) as clk:
        ms_chosen, per_step = timed(CHOSEN, args.steps, args.warmup)
    clocks = clk.summary()
    # counters of one chosen-form pass (for the flop count) and its output
    step(CHOSEN, cnt)
    torch.cuda.synchronize()
    c_mixed = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
    y_mixed = yout.cpu().numpy()
    flops_mixed = rkc_flops(w, c_mixed["n_accept"], c_mixed["n_reject"], c_mixed["n_rhs"], c_mixed["n_specrad_iter"])

    # the kernel the chosen form ran (ODE_MAP_AUTO's choice unless --mapping fixes it)
    amap, ablock, _ = B.mapping_info(h, "rkc", CHOSEN, block_size=args.block)
    if MAPPING != B.ODE_MAP_AUTO:
        amap, ablock = MAPPING, (args.block or 128)
    kname = ("k_static" if amap == B.ODE_MAP_THREAD else "k_queue") + \
        f"<RkcMixed<JitMass, false>> (generated network code, lean split; block {ablock})"

    ms_mixed64 = ms_plain = None
    c_plain = y_plain = None
    if args.plain_steps > 0:
        # the mixed form with the split as specified (FP64 time, step, norm accumulation)
        ms_mixed64, _ = timed(B.ODE_PREC_MIXED, args.plain_steps, 1)

        # plain FP64 form on the same inputs
        ms_plain, _ = timed(B.ODE_PREC_FP64, args.plain_steps, 1)
        step(B.ODE_PREC_FP64, cnt)
        torch.cuda.synchronize()
        c_plain = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        y_plain = yout.cpu().numpy()
        flops_plain = rkc_flops(w, c_plain["n_accept"], c_plain["n_reject"], c_plain["n_rhs"], c_plain["n_specrad_iter"])

    # end to end through the C ABI with pinned host buffers
    hy0 = torch.from_numpy(w.y0).pin_memory()
    hp = torch.from_numpy(w.params).pin_memory()
    hy = torch.empty_like(hy0).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.integrate("rkc", h, hy0.numpy(), hp.numpy(), w.t0, w.tend, w.rtol, w.atol, y_out=hy.numpy(),
                    precision=CHOSEN, mapping=MAPPING, block_size=args.block)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_step = float(np.mean(e2e_ms))
    e2e_step = max_over_ranks(e2e_step, world, dev)

    value = aggregate_rate(w.nsys, world, ms_chosen)
    achieved = flops_mixed / (ms_chosen * 1e-3) / 1e12
    achieved_plain = flops_plain / (ms_plain * 1e-3) / 1e12 if ms_plain else None

    out = {}
    if rank == 0:
        peak32, _ = B.fma_peak(False, 1 << 20)
        peak64, _ = B.fma_peak(True, 1 << 14)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_chosen, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded mass-action network and states; no dataset)",
            "config": {"workload": "massaction-13sp-27rx RKC, 1,048,576 systems/GPU, t in [0,1e-4], rtol 1e-6, atol 1e-12",
                       "nsys_per_gpu": w.nsys, "method": "rkc",
                       "form": "chosen: FP32 RHS, stages, step size, spectral radius and error norms, Kahan "
                               "state, remaining interval as an FP32 pair, FP64 coefficient tables, generated "
                               "network code, mapping chosen by ODE_MAP_AUTO",
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"independent batches x{world}"},
            "rhs_evals_per_s": float(np.sum(c_mixed["n_rhs"])) * world / (ms_chosen * 1e-3),
            "plain_fp64": None if not ms_plain else {
                "value": aggregate_rate(w.nsys, world, ms_plain), "ms_per_step": ms_plain,
                "rhs_evals_per_s": float(np.sum(c_plain["n_rhs"])) * world / (ms_plain * 1e-3),
                "achieved_tflops": achieved_plain, "frac_fp64_peak": achieved_plain / FP64_PEAK_TFLOPS,
                "frac_fp64_measured": achieved_plain / (peak64 / 1e3)},
            "speedup_chosen_vs_plain": ms_plain / ms_chosen if ms_plain else None,
            "mixed_spec_split": None if not ms_mixed64 else {
                "value": aggregate_rate(w.nsys, world, ms_mixed64), "ms_per_step": ms_mixed64,
                "form": "FP32 stages + Kahan state; FP64 time, step size, error-norm accumulation"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS,
                         "traffic": NCU_TRAFFIC_BYTES_PER_SYSTEM * w.nsys if amap == B.ODE_MAP_THREAD else None,
                         "traffic_source": "ncu dram__bytes_read+write of k_static on 262,144 systems, scaled by "
                                           "the system count (null when another kernel ran)",
                         "kernel": kname,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
                         "peak_measured_fma": peak32 / 1e3, "frac_of_measured": achieved / (peak32 / 1e3),
                         "flops_per_launch": flops_mixed},
            "fp64_fma_measured_tflops": peak64 / 1e3,
            "e2e": {"value": aggregate_rate(w.nsys, world, e2e_step), "unit": UNIT,
                    "h2d_bytes_per_step": int(w.y0.nbytes + w.params.nbytes), "d2h_bytes_per_step": int(w.y0.nbytes)},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "status_ok_frac": float(np.mean((c_mixed["status"] & 0xFF) == 0)),
        }
        if not args.no_cpu and c_plain is not None:
            out["cpu_baseline"], acc = cpu_baseline(w, args, y_mixed, y_plain, c_plain)
            out["accuracy_vs_oracle"] = acc
    if args.proposal_nsys > 0:
        prop = proposal_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["learned_proposal"] = prop
    if args.mixed_nsys > 0:
        mixed = mixed_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["mixed_batch"] = mixed
    if args.pleiades_nsys > 0:
        pl = pleiades_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["pleiades_rkck"] = pl
    if args.kinetics_nsys > 0:
        kn = kinetics_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["kinetics_ignition"] = kn
    if args.specrad_steps > 0:
        sr = specrad_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["specrad_modes"] = sr
    if args.split_steps > 0:
        split = split_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["global_steps"] = split
    if rank == 0:
        print(json.dumps(out), flush=True)
    B.release(h)
    if world > 1:
        dist.destroy_process_group()


def proposal_leg(args, B, torch, dev, stream, rank, world, barrier):
    """The learned proposal on the 4,194,304-system mass-action batch:
    trained on records the plain FP64 solver logs on held-out seeds (state
    features -> first step, spectral-radius bound, whole-integration cost),
    then the chosen form timed without it, with the proposed start, and
    with the proposed start plus the batch taken longest-first by the
    predicted cost (the proposal and ordering passes are inside the timed
    step).  For context, the order from the true costs of an earlier run on
    the same inputs bounds what any cost predictor can give."""
    import oracle as O
    t_start = time.perf_counter()
    wt = W.massaction(nsys=args.proposal_train, seed=1000 + rank)
    ht = B.register_workload(wt)
    log = torch.full((wt.nsys, wt.neq + 4), float("nan"), dtype=torch.float32, device=dev)
    B.integrate("rkc", ht, torch.from_numpy(wt.y0).to(dev), torch.from_numpy(wt.params).to(dev), wt.t0, wt.tend,
                wt.rtol, wt.atol, precision=B.ODE_PREC_FP64, log_xy=log, sync=True)
    B.release(ht)
    ok = torch.isfinite(log).all(dim=1)
    X, Y = log[ok, :wt.neq + 1].contiguous(), log[ok, wt.neq + 1:].contiguous()
    net = B.MLP(wt.neq + 1, seed=0)
    net.fit_normalization(X, Y)
    hist = net.train(X, Y, epochs=args.proposal_epochs, batch=4096, lr=2e-3, seed=0)
    t_train = time.perf_counter() - t_start
    del log, X, Y

    w = W.massaction(nsys=args.proposal_nsys, seed=4 + rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    yout = torch.empty_like(y0)
    CH = B.ODE_PREC_MIXED_LEAN
    B.prepare(h, "rkc", CH)
    true_cost = None

    def step(mode, counters=None):
        kw = {}
        if mode in ("with_proposal", "with_proposal_ordered"):
            h0, s0, c = net.propose(y0, p, stream=stream.cuda_stream, with_cost=True)
            kw = dict(h0=h0, sigma0=s0)
            if mode == "with_proposal_ordered":
                kw["cost"] = c
        elif mode == "ordered_by_true_cost":
            kw = dict(cost=true_cost)
        B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=yout, counters=counters, precision=CH,
                    mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream, **kw)

    res = {}
    for mode in ("without", "with_proposal", "with_proposal_ordered", "ordered_by_true_cost"):
        for _ in range(args.warmup):
            step(mode)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.proposal_steps):
            step(mode)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.proposal_steps
        cnt = B.counters_like(w.nsys, dev)
        step(mode, cnt)
        torch.cuda.synchronize()
        c = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        if mode == "without":
            true_cost = cnt.n_rhs.float()
        res[mode] = {
            "systems_per_s": w.nsys * world / (ms * 1e-3), "ms_per_step": ms,
            "reject_rate": float(np.sum(c["n_reject"]) / np.sum(c["n_accept"] + c["n_reject"])),
            "mean_rhs": float(np.mean(c["n_rhs"])), "mean_power_iterations": float(np.mean(c["n_specrad_iter"])),
            "proposal_used": float(np.mean((c["status"] & B.ODE_ST_PROPOSED) != 0)),
            "y_sample": yout[:, :2048].cpu().numpy()}
        if mode == "with_proposal_ordered":
            pred = np.log(net.propose(y0, p, with_cost=True)[2].cpu().numpy())
            res[mode]["log_cost_corr_pred_vs_true"] = float(np.corrcoef(pred, np.log(c["n_rhs"]))[0, 1])
    res["ordered_by_true_cost"]["note"] = ("upper bound: order from the n_rhs counters of an earlier run on the "
                                           "same inputs (the previous global step in operator splitting)")
    B.release(h)
    net.release()
    ref = O.integrate_workload(W.subset(w, np.arange(2048)))
    for k, r in res.items():
        e = (np.abs(r.pop("y_sample") - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
        r["err_vs_fp64_oracle_max"] = float(e.max())
        r["err_vs_fp64_oracle_p999"] = float(np.quantile(e, 0.999))
    res["config"] = {"nsys_per_gpu": w.nsys, "train_pairs": int(ok.sum().item()), "train_seeds": "1000+rank",
                     "eval_seed": "4+rank", "epochs": args.proposal_epochs, "batch": 4096, "final_train_loss": float(hist[-1]),
                     "train_seconds_incl_logging": t_train,
                     "network": "14 -> 64 -> 64 -> 3 SiLU (log h0, log sigma, log cost), BF16 weights, "
                                "FP32 accumulate"}
    res["speedup_with_proposal"] = res["without"]["ms_per_step"] / res["with_proposal"]["ms_per_step"]
    res["speedup_with_proposal_ordered"] = res["without"]["ms_per_step"] / res["with_proposal_ordered"]["ms_per_step"]
    return res


def pleiades_leg(args, B, torch, dev, stream, rank, world, barrier):
    """The paper's RKCK benchmark shape (Section 4.1): copies of a seven-body
    planar gravity problem (28 equations) with perturbed initial states,
    eps = 1e-10, t in [0, 1], plain FP64 (the tolerance is beyond FP32
    stages), one 8-lane team per system; against the oracle on the host
    cores."""
    import torch.distributed as dist
    import oracle as O
    w = W.pleiades(nsys=args.pleiades_nsys, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    y = torch.empty_like(y0)
    cnt = B.counters_like(w.nsys, dev)

    def step(counters=None):
        B.integrate("rkck", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=y, counters=counters,
                    precision=B.ODE_PREC_FP64, mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.pleiades_steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.pleiades_steps
    ms = max_over_ranks(ms, world, dev)
    step(cnt)
    torch.cuda.synchronize()
    c = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "status")}
    yg = y.cpu().numpy()
    B.release(h)
    # RHS: per body 6 flops per other body (differences, r2) + sqrt + 2 mult/div pairs; count
    # 20 flops per pair and direction as the algorithmic work, FP64
    n = w.neq // 4
    rhs_flops = 20 * n * (n - 1)
    flops = float(np.sum(c["n_rhs"])) * rhs_flops + float(np.sum(c["n_accept"] + c["n_reject"])) * 60 * w.neq
    sample = np.arange(min(w.nsys, 4096))
    t0 = time.perf_counter()
    ref = O.integrate_workload(W.subset(w, sample))
    cpu_s = time.perf_counter() - t0
    same = (c["n_accept"][sample] == ref.n_accept) & (c["n_reject"][sample] == ref.n_reject)
    e = (np.abs(yg[:, sample] - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
    return {"systems_per_s": w.nsys * world / (ms * 1e-3), "ms_per_step": ms,
            "mean_attempts": float(np.mean(c["n_accept"] + c["n_reject"])),
            "rhs_evals_per_s": float(np.sum(c["n_rhs"])) * world / (ms * 1e-3),
            "achieved_tflops_fp64": flops / (ms * 1e-3) / 1e12,
            "frac_fp64_peak": flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
            "status_ok_frac": float(np.mean(c["status"] == 0)),
            "parity_sample": {"systems": int(sample.size), "same_counts_frac": float(same.mean()),
                              "max_rel_err_same_counts": float(e[same].max()) if same.any() else None},
            "cpu_oracle_systems_per_s": sample.size / cpu_s, "cpu_cores": os.cpu_count(),
            "config": {"nsys_per_gpu": w.nsys, "bodies": n, "neq": w.neq, "eps": w.rtol,
                       "interval": [w.t0, w.tend], "perturbation": 1e-3,
                       "flops_model": "20 per ordered pair per evaluation + 60 per unknown per attempt"}}


def kinetics_leg(args, B, torch, dev, stream, rank, world, barrier):
    """The paper's RKC case shape (Section 4.2): constant-volume kinetics with
    a temperature equation on a synthetic 57-species, 766-reaction mechanism,
    10 global steps of 1e-6 s.  Plain FP64 (the paper's form) and the lean
    mixed form, with cold restarts (the paper's driver) and with warm
    RESTART carries; the CPU oracle on a bounded sample."""
    import torch.distributed as dist
    import oracle as O
    w = W.kinetics(nsys=args.kinetics_nsys, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    y = torch.empty_like(y0)
    carry = B.carry_like(w.neq, w.nsys, dev)
    cnt = B.counters_like(w.nsys, dev)
    edges = np.linspace(0.0, 1e-5, 11)

    def chain(prec, warm, total=None):
        for t_a, t_b in zip(edges[:-1], edges[1:]):
            kw = dict(carry=carry, carry_mode=B.ODE_CARRY_RESTART) if warm else {}
            B.integrate("rkc", h, y, p, float(t_a), float(t_b), w.rtol, w.atol, y_out=y, counters=cnt,
                        precision=prec, mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream, **kw)
            if total is not None:
                torch.cuda.synchronize()
                total += cnt.n_rhs.cpu().numpy()

    res = {}
    for pname, prec in (("fp64", B.ODE_PREC_FP64), ("lean", B.ODE_PREC_MIXED_LEAN)):
        for warm in (False, True):
            ms = []
            for rep in range(1 + args.kinetics_reps):
                y.copy_(y0)
                carry.zero_()
                torch.cuda.synchronize()
                barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                chain(prec, warm)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep > 0:
                    ms.append(e0.elapsed_time(e1))
            t = float(np.mean(ms))
            t = max_over_ranks(t, world, dev)
            y.copy_(y0)
            carry.zero_()
            total = np.zeros(w.nsys, np.int64)
            chain(prec, warm, total)
            res[f"{pname}_{'warm_restart' if warm else 'cold'}"] = {
                "systems_per_s": w.nsys * world / (t * 1e-3), "ms_per_chain": t, "mean_rhs": float(total.mean()),
                "y_sample": y[:, :256].cpu().numpy()}
    B.release(h)
    ws = W.subset(w, np.arange(256))
    ws.aux = w.aux
    m = O.model_for(ws)
    t0 = time.perf_counter()
    ys = ws.y0.copy()
    for t_a, t_b in zip(edges[:-1], edges[1:]):
        ys = O.integrate(m, 1, ys, ws.params, float(t_a), float(t_b), ws.rtol, ws.atol).y
    cpu_s = time.perf_counter() - t0
    for k, r in res.items():
        yy = r.pop("y_sample")
        e = (np.abs(yy - ys) / (np.abs(ys) + w.atol)).max(axis=0)
        r["err_vs_oracle_cold_chain_p999"] = float(np.quantile(e, 0.999))
    res["cpu_oracle_cold_chain"] = {"systems_per_s": 256 / cpu_s, "cores": os.cpu_count(), "sample": 256}
    res["config"] = {"nsys_per_gpu": w.nsys, "species": w.neq - 1, "reactions": w.aux["mechanism"].n_reactions,
                     "global_steps": 10, "dt": 1e-6, "rtol": w.rtol, "atol": w.atol,
                     "mapping": "one warp per system, rates and concentrations staged in shared memory"}
    return res


def specrad_leg(args, B, torch, dev, stream, rank, world, barrier):
    """The chosen form on the mass-action batch with each spectral-radius
    estimate: the Appendix's power method (the paper's), the Gershgorin
    bound instead of it, and the power method capped by the bound."""
    import torch.distributed as dist
    w = W.massaction(nsys=args.nsys, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    y = torch.empty_like(y0)
    cnt = B.counters_like(w.nsys, dev)
    CH = B.ODE_PREC_MIXED_LEAN
    B.prepare(h, "rkc", CH)
    res = {}
    ref = None
    for name, mode in (("power", B.ODE_SPECRAD_POWER), ("gershgorin", B.ODE_SPECRAD_GERSHGORIN),
                       ("power_capped", B.ODE_SPECRAD_POWER_CAPPED)):
        def step(counters=None):
            B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=y, counters=counters, precision=CH,
                        mapping=B.ODE_MAP_AUTO, specrad=mode, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.specrad_steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.specrad_steps
        ms = max_over_ranks(ms, world, dev)
        step(cnt)
        torch.cuda.synchronize()
        yy = y.cpu().numpy()
        if ref is None:
            ref = yy
        e = (np.abs(yy - ref) / (np.abs(ref) + w.atol)).max(axis=0)
        res[name] = {"systems_per_s": w.nsys * world / (ms * 1e-3), "ms_per_step": ms,
                     "mean_rhs": float(cnt.n_rhs.float().mean().item()),
                     "mean_power_iterations": float(cnt.n_specrad_iter.float().mean().item()),
                     "p999_diff_vs_power": float(np.quantile(e, 0.999))}
    B.release(h)
    return res


def split_leg(args, B, torch, dev, stream, rank, world, barrier):
    """The paper's outer loop (Section 3): the mass-action batch integrated
    over [0, 1e-4] as G global steps, one rkc_integrate call each, states
    resident on the device.  cold = every call restarts (the paper's
    driver); warm_continue / warm_restart = the controller state carried
    across calls (ode_opts.carry, carry modes CONTINUE / RESTART); *_ordered
    = also taking each call's systems longest-first by the previous call's
    n_rhs counters.  One repetition of all G calls is one timed step."""
    import torch.distributed as dist
    import oracle as O
    w = W.massaction(nsys=args.nsys, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    y = torch.empty_like(y0)
    carry = B.carry_like(w.neq, w.nsys, dev)
    cnt = B.counters_like(w.nsys, dev)
    CH = B.ODE_PREC_MIXED_LEAN
    B.prepare(h, "rkc", CH)
    edges = np.linspace(w.t0, w.tend, args.split_steps + 1)

    def chain(mode, total=None):
        for g, (t_a, t_b) in enumerate(zip(edges[:-1], edges[1:])):
            kw = {}
            if mode.startswith("warm"):
                kw["carry"] = carry
                kw["carry_mode"] = B.ODE_CARRY_RESTART if "restart" in mode else B.ODE_CARRY_CONTINUE
            if mode.endswith("ordered") and g > 0:
                kw["cost"] = cnt.n_rhs
            B.integrate("rkc", h, y, p, float(t_a), float(t_b), w.rtol, w.atol, y_out=y, counters=cnt,
                        precision=CH, mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream, **kw)
            if total is not None:
                torch.cuda.synchronize()
                total += cnt.n_rhs.cpu().numpy()

    res = {}
    MODES = ("cold", "cold_ordered", "warm_continue", "warm_restart", "warm_restart_ordered")
    for mode in MODES:
        ms = []
        for rep in range(1 + args.split_reps):   # the first repetition warms up (and tunes the mapping)
            y.copy_(y0)
            carry.zero_()
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            chain(mode)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                ms.append(e0.elapsed_time(e1))
        t = float(np.mean(ms))
        t = max_over_ranks(t, world, dev)
        # counts and the final state of one more chain
        y.copy_(y0)
        carry.zero_()
        total = np.zeros(w.nsys, np.int64)
        chain(mode, total)
        res[mode] = {"systems_per_s": w.nsys * world / (t * 1e-3), "ms_per_chain": t,
                     "mean_rhs": float(total.mean()), "y_sample": y[:, :2048].cpu().numpy()}
    B.release(h)
    # accuracy: the oracle's own chain (same mode of restart) and its single call, on 2048 systems
    ws = W.subset(w, np.arange(2048))
    m = O.model_for(ws)
    ref_single = O.integrate_workload(ws)
    ref_chain = {}
    for kind in ("cold", "continue", "restart"):
        ys, c = ws.y0.copy(), None
        for t_a, t_b in zip(edges[:-1], edges[1:]):
            r = O.integrate(m, 1, ys, ws.params, float(t_a), float(t_b), ws.rtol, ws.atol,
                            carry_in=c if kind != "cold" else None, carry_out=True,
                            carry_mode=O.CARRY_RESTART if kind == "restart" else O.CARRY_CONTINUE)
            ys, c = r.y, r.carry
        ref_chain[kind] = ys
    for mode, r in res.items():
        ys = r.pop("y_sample")
        rc = ref_chain["cold" if mode.startswith("cold") else ("restart" if "restart" in mode else "continue")]
        e_chain = (np.abs(ys - rc) / (np.abs(rc) + w.atol)).max(axis=0)
        e_single = (np.abs(ys - ref_single.y) / (np.abs(ref_single.y) + w.atol)).max(axis=0)
        r["err_vs_oracle_chain_p999"] = float(np.quantile(e_chain, 0.999))
        r["err_vs_single_call_p999"] = float(np.quantile(e_single, 0.999))
    res["speedup_vs_cold"] = {m: res["cold"]["ms_per_chain"] / res[m]["ms_per_chain"] for m in MODES}
    res["config"] = {"nsys_per_gpu": w.nsys, "global_steps": args.split_steps, "interval": [w.t0, w.tend],
                     "timed": f"{args.split_reps} repetitions of the whole chain after one warm-up repetition",
                     "precision": "mixed lean", "state": "device resident (the paper copies each global step)"}
    return res


def mixed_leg(args, B, torch, dev, stream, rank, world, barrier):
    """The ragged batch: 262,144 systems, half Brusselator grids of 1-128
    points (RKC, rtol 1e-5), half van der Pol chains of 1-64 oscillators
    (RKCK, rtol 1e-6), in one graph-captured plan; the autotuned shapes
    against the paper's fixed one-thread-per-system mapping."""
    b = W.mixed(nsys=args.mixed_nsys, seed=rank)
    hb = B.register(B.ODE_RHS_BRUSS1D, 256)
    hc = B.register(B.ODE_RHS_VDP_CHAIN, 128, coupling=b.coupling)
    handles = np.where(b.kind == B.ODE_RHS_BRUSS1D, hb, hc)
    devt = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    y0, prm = devt(b.y0), devt(b.param)
    t0, tend, rtol, atol = devt(b.t0), devt(b.tend), devt(b.rtol), devt(b.atol)
    y = torch.empty_like(y0)
    res = {}
    for name, mapping in (("autotuned", B.ODE_MAP_AUTO), ("fixed_thread_per_system", B.ODE_MAP_THREAD)):
        plan = B.RaggedPlan(handles, b.method, b.neq, b.offset[:-1], y0, prm, t0, tend, rtol, atol, y_out=y,
                            precision=B.ODE_PREC_MIXED_LEAN, mapping=mapping, stream=stream.cuda_stream)
        for _ in range(1):
            plan.launch(stream.cuda_stream)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.mixed_steps):
            plan.launch(stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.mixed_steps
        res[name] = {"systems_per_s": b.nsys * world / (ms * 1e-3), "ms_per_step": ms,
                     "buckets": [{k: d[k] for k in ("family", "method", "size_class", "systems", "lanes",
                                                     "points_per_lane", "block", "mapping")} for d in plan.info()]}
        plan.destroy()
    B.release(hb)
    B.release(hc)
    res["speedup_autotuned_vs_fixed"] = res["fixed_thread_per_system"]["ms_per_step"] / res["autotuned"]["ms_per_step"]
    res["config"] = {"nsys_per_gpu": b.nsys, "unknowns_total": int(b.offset[-1]), "precision": "mixed lean",
                     "graph": "one CUDA graph launch per step (all buckets on parallel branches)"}
    return res


def cpu_baseline(w, args, y_mixed, y_plain, c_plain):
    """Time the oracle (as it stands) on a bounded sample of the same batch,
    and compare both GPU forms with it on that sample."""
    import oracle as O
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(123)
    probe = np.sort(rng.choice(w.nsys, 2048, replace=False))
    t0 = time.perf_counter()
    O.integrate_workload(W.subset(w, probe))
    rate = 2048 / (time.perf_counter() - t0)
    n = int(min(w.nsys, max(4096, rate * args.cpu_seconds)))
    idx = np.sort(rng.choice(w.nsys, n, replace=False))
    sub = W.subset(w, idx)
    t0 = time.perf_counter()
    ref = O.integrate_workload(sub)
    dt = time.perf_counter() - t0
    e_m = (np.abs(y_mixed[:, idx] - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
    e_p = (np.abs(y_plain[:, idx] - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
    same = (c_plain["n_accept"][idx] == ref.n_accept) & (c_plain["n_reject"][idx] == ref.n_reject)
    tol_units = (np.abs(y_mixed[:, idx] - ref.y) / (w.atol + w.rtol * np.abs(ref.y))).max(axis=0)
    base = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of {w.nsys} systems drawn uniformly (seed 123), full interval, all host cores"}
    acc = {"sample": n, "chosen_max_rel_err": float(e_m.max()), "chosen_p999_rel_err": float(np.quantile(e_m, 0.999)),
           "chosen_median_rel_err": float(np.median(e_m)),
           "chosen_max_err_in_tolerances": float(tol_units.max()),
           "chosen_p999_err_in_tolerances": float(np.quantile(tol_units, 0.999)),
           "plain_max_rel_err_same_counts": float(e_p[same].max()) if same.any() else None,
           "plain_same_counts_frac": float(same.mean())}
    # both forms against an independent tight reference (RKCK, rtol 1e-12) on
    # a small sample: the FP32 stages' error next to the method's own
    k = min(1024, n)
    sub_k = W.subset(w, idx[:k])
    tight = O.integrate(O.model_for(sub_k), 0, sub_k.y0, sub_k.params, sub_k.t0, sub_k.tend, 1e-12, 1e-18)
    e_ct = (np.abs(y_mixed[:, idx[:k]] - tight.y) / (np.abs(tight.y) + w.atol)).max(axis=0)
    e_ot = (np.abs(ref.y[:, :k] - tight.y) / (np.abs(tight.y) + w.atol)).max(axis=0)
    acc["vs_tight_reference"] = {"sample": k, "reference": "oracle RKCK rtol 1e-12 atol 1e-18",
                                 "chosen_max": float(e_ct.max()), "chosen_median": float(np.median(e_ct)),
                                 "fp64_oracle_max": float(e_ot.max()), "fp64_oracle_median": float(np.median(e_ot))}
    return base, acc


# ------------------------------------------------------------ reference arm

def run_reference(args):
    """The oracle (the paper's algorithm restated in plain C, FP64) timed on
    the host cores, each step a bounded slice of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    w = W.massaction(nsys=args.nsys, seed=0)
    cores = os.cpu_count() or 1
    per = args.ref_sample
    times = []
    for k in range(args.warmup + args.steps):
        idx = np.arange(k * per, (k + 1) * per) % w.nsys
        sub = W.subset(w, idx)
        t0 = time.perf_counter()
        O.integrate_workload(sub)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = float(np.mean(times)) * 1e3
    value = per / (ms * 1e-3)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "massaction-13sp-27rx RKC, t in [0,1e-4], rtol 1e-6, atol 1e-12",
                      "sample_per_step": per},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{per} consecutive systems per step of the {w.nsys}-system batch"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nsys", type=int, default=NSYS)
    ap.add_argument("--plain-steps", type=int, default=3, help="0 skips the plain FP64 and specified-split legs")
    ap.add_argument("--mapping", choices=["auto", "thread", "queue"], default="auto",
                    help="mapping of the main leg (fix it under a profiler, whose overhead distorts the "
                         "timing runs of auto)")
    ap.add_argument("--block", type=int, default=0, help="block size of the main leg (0: tuned / default)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-sample", type=int, default=16384)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--proposal-nsys", type=int, default=1 << 22, help="0 skips the learned-proposal leg")
    ap.add_argument("--proposal-train", type=int, default=1 << 20)
    ap.add_argument("--proposal-steps", type=int, default=3)
    ap.add_argument("--proposal-epochs", type=int, default=24)
    ap.add_argument("--mixed-nsys", type=int, default=262144, help="0 skips the ragged-batch leg")
    ap.add_argument("--mixed-steps", type=int, default=3)
    ap.add_argument("--specrad-steps", type=int, default=2, help="timed steps per spectral-radius mode (0 skips)")
    ap.add_argument("--pleiades-nsys", type=int, default=262144, help="n-body RKCK leg batch (0 skips)")
    ap.add_argument("--kinetics-nsys", type=int, default=16384, help="kinetics leg batch (0 skips)")
    ap.add_argument("--kinetics-reps", type=int, default=1)
    ap.add_argument("--pleiades-steps", type=int, default=3)
    ap.add_argument("--split-steps", type=int, default=10, help="global steps of the outer-loop leg (0 skips it)")
    ap.add_argument("--split-reps", type=int, default=2)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # at least three untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
