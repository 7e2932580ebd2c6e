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
# The chosen form must reach this final-state error against the FP64 oracle
# (p99.9 over systems of max_i |y - y_ref| / (|y_ref| + atol)) at this
# multiple of the plain FP64 form's throughput.
TARGET_P999, TARGET_SPEEDUP = 1e-5, 2.0
# nominal ALU peaks from unit counts and the maximum SM clock: FP32 128 lanes
# x 2 flops per SM per clock (the SM count read from the device); FP64 the
# part's rated 1.25 TFLOP/s
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = 1.25


def fp32_peak_tflops(sm_count: int) -> float:
    return sm_count * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20

# The precision forms of rkc_integrate (ODE_PREC_*), their kernels and the
# arithmetic each computes in.
FORMS = {"f2_lean_learned": 4, "f2_lean": 4, "f2_learned": 3, "f2": 3, "mixed_lean": 2, "mixed_spec_split": 1,
         "plain_fp64": 0}
# forms whose step also runs the learned proposal: the network's pre-pass
# (spectral-radius bound and cost per system, the Euler trial still setting
# the first step) and the longest-first order by the predicted cost
LEARNED_FORMS = {"f2_lean_learned", "f2_learned"}
# the precision form underneath (what the other legs run when they take the
# headline's precision without its proposal)
BASE_FORM = {"f2_lean_learned": "f2_lean", "f2_learned": "f2"}
# our kernel launches per step: the integration kernel; for the generated
# two-float forms the rate-constant prologue; for the learned forms the
# proposal pre-pass and the four kernels of the cost order
LAUNCHES = {"f2_lean_learned": 7, "f2_lean": 2, "f2_learned": 7, "f2": 2, "mixed_lean": 1, "mixed_spec_split": 1,
            "plain_fp64": 1}
FORM_KERNELS = {"f2_lean_learned": "RkcF2<JitMass, false>", "f2_lean": "RkcF2<JitMass, false>",
                "f2_learned": "RkcF2<JitMass, true>", "f2": "RkcF2<JitMass, true>",
                "mixed_lean": "RkcMixed<JitMass, false>", "mixed_spec_split": "RkcMixed<JitMass, true>",
                "plain_fp64": "RkcF64<JitMass>"}
FORM_DTYPES = {"f2_lean_learned": "f32x2", "f2_lean": "f32x2", "f2_learned": "f32x2+f64", "f2": "f32x2+f64", "mixed_lean": "f32", "mixed_spec_split": "f32+f64",
               "plain_fp64": "f64"}
FORM_TEXT = {
    "f2_lean_learned": "the two-float form (f2_lean) with the learned proposal: a BF16 network's pre-pass gives "
                       "each system's initial spectral-radius bound and predicted cost, and the batch runs "
                       "longest-first by that cost (network trained before timing on held-out seeds)",
    "f2_learned": "the two-float form with FP64 bookkeeping (f2: the specified split's FP64 time, step size and "
                  "error-norm reduction) with the learned proposal, as f2_lean_learned",
    "f2_lean": "two-float (FP32 pair, ~48-bit) state, stages, evaluation points and RHS; FP32 step size, spectral "
               "radius and error norm; remaining interval as an FP32 pair; FP64-built coefficients as pairs",
    "f2": "two-float state, stages, evaluation points and RHS; FP64 time, step size, spectral radius and error-norm "
          "accumulation; FP64-built coefficients as pairs",
    "mixed_lean": "FP32 RHS, stages, step size, spectral radius and error norms; Kahan-compensated FP32 state; "
                  "remaining interval as an FP32 pair",
    "mixed_spec_split": "FP32 RHS and stages, Kahan-compensated FP32 state; FP64 time, step size and error-norm "
                        "accumulation (the split as the target specifies it)",
    "plain_fp64": "every operation in FP64 (the paper's form; bitwise equal to the oracle)"}
# DRAM bytes (read + write) per system of each form's generated kernel, from
# one ncu capture of k_static on 262,144 systems of this workload; traffic
# grows with the number of systems (each state is read once, written once).
# mixed_lean: 29.883 MB read + 0.899 MB written.  f2_lean_learned (the
# kernel with the block-wide step-end hold; it reads its systems through the
# predicted-cost order, so each 8-byte state access is a 32-byte sector of
# its own; it also reads the rate table of the prologue): 439.148 MB read +
# 66.671 MB written.
NCU_TRAFFIC_BYTES_PER_SYSTEM = {"mixed_lean": (29.88288e6 + 0.89856e6) / 262144,
                                "f2_lean_learned": (439.148032e6 + 66.67136e6) / 262144}
# FP32 pipe use of the chosen kernel from the same capture (ncu --set full)
NCU_PIPE_CONTEXT = {"f2_lean_learned": {
    "fma_pipe_cycles_active": 0.540, "issue_active": 0.670, "fp32_thread_inst_per_method_flop": 3.5,
    # 506.2 G FADD + 2 x 138.2 G FFMA + 50.7 G FMUL thread instructions on 262,144 systems
    "fp32_flops_executed_per_system": 833.3e9 / 262144,
    "source": "ncu --set full of k_static<RkcF2> on 262,144 systems of this workload, 128-thread blocks, "
              "block-wide step-end hold (summary under profiles/)"}}
NCU_TRAFFIC_SOURCE = ("ncu dram__bytes_read+write of k_static on 262,144 systems, scaled by the system count "
                      "(null when another kernel ran or no capture of this kernel exists)")


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
    """Algorithmic flops of one right-hand side (an FMA counts 2).
    Mass-action: per reaction (|R| - 1) products of concentrations, one
    product with k_j and 2 (|R| + |P|) for the stoichiometric scatter
    updates, i.e. 3 |R| + 2 |P|.  Van der Pol: 5.  Brusselator: 17 per grid
    point."""
    if w.kind == W.RHS_MASSACTION:
        n = w.network
        return int(np.sum(3 * n.n_reac + 2 * n.n_prod))
    if w.kind == W.RHS_VDP:
        return 5
    if w.kind == W.RHS_BRUSS1D:
        return 17 * (w.neq // 2)
    raise ValueError(f"no flop model for kind {w.kind}")


def rkc_flops(w: W.Workload, n_acc, n_rej, n_rhs, n_sr) -> float:
    """Algorithmic flops of RKC runs from the per-system counters: every RHS
    evaluation, plus per m-stage attempt N (2 + 9 (m - 1) + 11) vector flops
    and 15 (m - 1) for the stage coefficients, per power iteration 6 N and
    5 N for the initial step."""
    N = w.neq
    A = n_acc.astype(np.float64) + n_rej
    sum_m = n_rhs.astype(np.float64) - n_sr - 2.0      # minus F(t0) and the initial trial step
    vec = N * (13.0 * A + 9.0 * (sum_m - A)) + 15.0 * (sum_m - A) + 6.0 * N * n_sr + 5.0 * N
    return float(np.sum(n_rhs.astype(np.float64) * rhs_flops(w) + vec))


def rkck_flops(w: W.Workload, n_acc, n_rej) -> float:
    """Algorithmic flops of RKCK runs: per attempt six RHS evaluations and
    60 N vector flops (stage sums, the fifth-order solution, the error
    vector, its scaling and maximum)."""
    A = n_acc.astype(np.float64) + n_rej
    return float(np.sum(A * (6.0 * rhs_flops(w) + 60.0 * w.neq)))


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

def map_text(B, h, prec, mapping, block):
    """The kernel and block size a form's calls ran with (ODE_MAP_AUTO's
    cached choice unless the mapping is fixed)."""
    if mapping != B.ODE_MAP_AUTO:
        return ("thread" if mapping == B.ODE_MAP_THREAD else "queue") + f", block {block or 128}"
    m, b, tuned = B.mapping_info(h, "rkc", prec, block_size=block)
    return ("thread" if m == B.ODE_MAP_THREAD else "queue") + f", block {b}" + ("" if tuned else " (default)")


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

    # the learned proposal's network (trained before any timing, on held-out seeds)
    net, net_info = None, None
    if args.chosen in LEARNED_FORMS or args.plain_steps > 0 or args.proposal_nsys > 0:
        net, net_info = train_proposal(args, B, torch, dev, rank)
    no_h0 = torch.full((w.nsys,), float("nan"), dtype=torch.float32, device=dev)

    def step(name, counters=None, y_in=None, p_in=None, y_res=None):
        y_in = y0 if y_in is None else y_in
        p_in = p if p_in is None else p_in
        kw = {}
        if name in LEARNED_FORMS:
            # the network's bound replaces the initial power method (the Euler
            # trial still sets the first step); its cost orders the batch
            _, s0, c = net.propose(y_in, p_in, stream=stream.cuda_stream, with_cost=True)
            kw = dict(h0=no_h0, sigma0=s0, cost=c)
        B.integrate("rkc", h, y_in, p_in, w.t0, w.tend, w.rtol, w.atol, y_out=yout if y_res is None else y_res,
                    counters=counters, precision=FORMS[name], mapping=MAPPING, block_size=args.block,
                    stream=stream.cuda_stream, **kw)

    CHOSEN = FORMS[args.chosen]
    for prec in set(FORMS.values()):
        B.prepare(h, "rkc", prec)       # generated network kernels compiled before any timing

    def timed(name, steps, warmup):
        for _ in range(warmup):
            step(name)
        torch.cuda.synchronize()
        evs = []
        barrier()
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()                       # L2 flush between timed iterations
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(name)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        total = sum(ms)
        total = max_over_ranks(total, world, dev)
        return total / steps, ms

    def counted(name):
        step(name, cnt)
        torch.cuda.synchronize()
        c = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        return c, yout.cpu().numpy()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None

    # chosen form: timed with the clock sampler running
    with ClockSampler(gpu_id) as clk:
        ms_chosen, per_step = timed(args.chosen, args.steps, args.warmup)
    clocks = clk.summary()
    runs = {}
    c_ch, y_ch = counted(args.chosen)
    runs[args.chosen] = {"ms": ms_chosen, "c": c_ch, "y": y_ch}
    # the learned form's pre-pass alone (the proposal kernel), so that the
    # integration kernel's share of the step is known
    ms_prepass = 0.0
    if args.chosen in LEARNED_FORMS:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            net.propose(y0, p, stream=stream.cuda_stream, with_cost=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_prepass = e0.elapsed_time(e1) / args.steps
    if args.plain_steps > 0:
        # every other form on the same inputs
        for name in FORMS:
            if name == args.chosen:
                continue
            ms, _ = timed(name, args.plain_steps, 1)
            c, y = counted(name)
            runs[name] = {"ms": ms, "c": c, "y": y}

    # the kernel the chosen form ran (ODE_MAP_AUTO's choice unless --mapping fixes it)
    amap, ablock, _ = B.mapping_info(h, "rkc", CHOSEN, block_size=args.block)
    if MAPPING != B.ODE_MAP_AUTO:
        amap, ablock = MAPPING, (args.block or 128)
    kname = ("k_static" if amap == B.ODE_MAP_THREAD else "k_queue") + \
        f"<{FORM_KERNELS[args.chosen]}> (generated network code; block {ablock})"

    # end to end through the C ABI with pinned host buffers
    hy0 = torch.from_numpy(w.y0).pin_memory()
    hp = torch.from_numpy(w.params).pin_memory()
    hy = torch.empty_like(hy0).pin_memory()
    e2e_ms = []
    dy0, dp, dy = torch.empty_like(y0), torch.empty_like(p), torch.empty_like(y0)
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.chosen in LEARNED_FORMS:
            # the proposal needs device arrays: pinned host -> device, the
            # step, device -> pinned host, all inside the timed region
            dy0.copy_(hy0, non_blocking=True)
            dp.copy_(hp, non_blocking=True)
            step(args.chosen, y_in=dy0, p_in=dp, y_res=dy)
            hy.copy_(dy, non_blocking=True)
            torch.cuda.synchronize()
        else:
            B.integrate("rkc", h, hy0.numpy(), hp.numpy(), w.t0, w.tend, w.rtol, w.atol, y_out=hy.numpy(),
                        precision=CHOSEN, mapping=MAPPING, block_size=args.block)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_step = float(np.mean(e2e_ms))
    e2e_step = max_over_ranks(e2e_step, world, dev)

    value = aggregate_rate(w.nsys, world, ms_chosen)
    flops = {k: rkc_flops(w, r["c"]["n_accept"], r["c"]["n_reject"], r["c"]["n_rhs"], r["c"]["n_specrad_iter"])
             for k, r in runs.items()}
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak32_nominal = fp32_peak_tflops(sm_count)

    out = {}
    if rank == 0:
        peak32, _ = B.fma_peak(False, 1 << 20)
        peak64, _ = B.fma_peak(True, 1 << 14)
        peak32, peak64 = peak32 / 1e3, peak64 / 1e3
        # the integration kernel's time: the step less the learned pre-pass
        # (the rate-constant prologue and the order kernels, ~1 % of the
        # step, stay inside: a lower bound on the kernel's rate)
        ms_kernel = ms_chosen - ms_prepass
        achieved = flops[args.chosen] / (ms_kernel * 1e-3) / 1e12
        two_float = args.chosen.startswith("f2")
        ms_plain = runs["plain_fp64"]["ms"] if "plain_fp64" in runs else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_chosen, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPES[args.chosen],
            "data": "synthetic (seeded mass-action network and states; no dataset)",
            "config": {"workload": f"massaction-13sp-27rx RKC, {w.nsys:,} systems/GPU, t in [0,1e-4], rtol 1e-6, atol 1e-12",
                       "nsys_per_gpu": w.nsys, "method": "rkc", "form": FORM_TEXT[args.chosen],
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"independent batches x{world}"},
            "rhs_evals_per_s": float(np.sum(runs[args.chosen]["c"]["n_rhs"])) * world / (ms_chosen * 1e-3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak32_nominal, "unit": "TFLOP/s",
                         "frac": achieved / peak32_nominal,
                         "traffic": (NCU_TRAFFIC_BYTES_PER_SYSTEM[args.chosen] * w.nsys
                                     if amap == B.ODE_MAP_THREAD and args.chosen in NCU_TRAFFIC_BYTES_PER_SYSTEM else None),
                         "traffic_source": NCU_TRAFFIC_SOURCE,
                         "kernel": kname,
                         "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flops x 2070 MHz (FP32 pipe, the one "
                                        "the kernel runs on)",
                         "peak_measured_fma": peak32, "frac_of_measured": achieved / peak32,
                         "flops_per_launch": flops[args.chosen],
                         "kernel_ms": ms_kernel, "prepass_ms": ms_prepass,
                         "flops_model": "method flops (3|R| + 2|P| per mass-action evaluation, N (13 + 9 (m - 1)) + "
                                        "15 (m - 1) per attempt, 6 N per power iteration, 5 N for the start)"},
            "fp64_fma_measured_tflops": peak64, "fp32_fma_measured_tflops": peak32,
            "e2e": {"value": aggregate_rate(w.nsys, world, e2e_step), "unit": UNIT,
                    "h2d_bytes_per_step": int(w.y0.nbytes + w.params.nbytes), "d2h_bytes_per_step": int(w.y0.nbytes)},
            "gpu_launches": args.steps * LAUNCHES[args.chosen],
            "clocks": clocks,
            "status_ok_frac": float(np.mean((runs[args.chosen]["c"]["status"] & 0xFF) == 0)),
        }
        if two_float:
            # the two-float form computes the FP64 method's arithmetic to ~48 bits on the FP32 pipe:
            # its method flops against the FP64 pipe's peak (above 1: beyond any FP64 kernel)
            out["roofline"]["method_tflops_vs_fp64_peak"] = {
                "achieved": achieved, "peak_rated": FP64_PEAK_TFLOPS, "peak_measured_fma": peak64,
                "frac_rated": achieved / FP64_PEAK_TFLOPS, "frac_measured": achieved / peak64}
        if args.chosen in NCU_PIPE_CONTEXT and amap == B.ODE_MAP_THREAD:
            # each method flop is several FP32 instructions in two-float
            # arithmetic: the kernel's own use of the FP32 pipe, from its
            # ncu capture (context for frac, not a timing)
            ctx = dict(NCU_PIPE_CONTEXT[args.chosen])
            # the FP32 flops the kernel executes (FMA = 2, from the capture's
            # instruction mix, per system) at the live kernel time
            ex = ctx["fp32_flops_executed_per_system"] * w.nsys / (ms_kernel * 1e-3) / 1e12
            ctx["fp32_flops_executed_tflops"] = ex
            ctx["fp32_flops_executed_frac"] = ex / peak32_nominal
            out["roofline"]["ncu_pipe_context"] = ctx
        forms = {}
        for name, r in runs.items():
            fl = flops[name]
            ach = fl / (r["ms"] * 1e-3) / 1e12
            peak_kind = "fp64" if name == "plain_fp64" else "fp32"
            forms[name] = {"value": aggregate_rate(w.nsys, world, r["ms"]), "ms_per_step": r["ms"],
                           "rhs_evals_per_s": float(np.sum(r["c"]["n_rhs"])) * world / (r["ms"] * 1e-3),
                           "achieved_tflops": ach,
                           "frac_peak": ach / (FP64_PEAK_TFLOPS if peak_kind == "fp64" else peak32_nominal),
                           "frac_peak_measured": ach / (peak64 if peak_kind == "fp64" else peak32),
                           "peak": peak_kind, "form": FORM_TEXT[name],
                           "speedup_vs_plain": (ms_plain / r["ms"]) if ms_plain else None,
                           "mapping": map_text(B, h, FORMS[name], MAPPING, args.block),
                           "status_ok_frac": float(np.mean((r["c"]["status"] & 0xFF) == 0))}
        out["forms"] = forms
        if ms_plain:
            out["plain_fp64"] = forms["plain_fp64"]
            out["speedup_chosen_vs_plain"] = ms_plain / ms_chosen
        if not args.no_cpu and "plain_fp64" in runs:
            out["cpu_baseline"], acc = cpu_baseline(w, args, runs)
            out["accuracy_vs_oracle"] = acc
            for name in forms:
                forms[name]["err_vs_fp64_oracle_p999"] = acc["forms"][name]["p999_rel_err"]
                forms[name]["err_vs_fp64_oracle_max"] = acc["forms"][name]["max_rel_err"]
                forms[name]["meets_target"] = bool(
                    acc["forms"][name]["p999_rel_err"] <= TARGET_P999 and
                    (name == "plain_fp64" or (forms[name]["speedup_vs_plain"] or 0.0) >= TARGET_SPEEDUP))
            qual = [n for n in forms if n != "plain_fp64" and forms[n]["meets_target"]]
            out["target"] = {"bar": f"p99.9 error <= {TARGET_P999:g} vs the FP64 oracle at >= {TARGET_SPEEDUP:g}x "
                                    "the plain FP64 form's systems/s",
                             "chosen": args.chosen, "chosen_meets": forms[args.chosen]["meets_target"],
                             "fastest_qualifying": max(qual, key=lambda n: forms[n]["value"]) if qual else None}
    if args.stoich_reps > 0 and rank == 0:
        lean = runs.get("mixed_lean")
        out["stoich_tensor_cores"] = stoich_leg(args, B, float(np.mean(lean["c"]["n_rhs"])) if lean else None,
                                                lean["ms"] if lean else None)
    if args.c0_steps > 0:
        c0 = c0_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["c0_vdp_rkck"] = c0
    if args.c1_steps > 0:
        c1 = c1_leg(args, B, torch, dev, stream, rank, world, barrier)
        if rank == 0:
            out["c1_bruss_rkc"] = c1
    if rank == 0 and net_info is not None:
        out["proposal_network"] = {"train_pairs": net_info["pairs"], "train_sigma_records": net_info["sigma_records"],
                                   "train_seconds_incl_logging": net_info["seconds"],
                                   "final_train_loss": float(net_info["hist"][-1]), "train_seeds": "1000+rank",
                                   "note": "trained once before any timing; used by the learned forms and the "
                                           "learned_proposal leg"}
    if args.proposal_nsys > 0:
        prop = proposal_leg(args, B, torch, dev, stream, rank, world, barrier, net, net_info)
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
    if net is not None:
        net.release()
    if world > 1:
        dist.destroy_process_group()


def train_proposal(args, B, torch, dev, rank):
    """The learned proposal's network, trained before any timing on records
    the plain FP64 solver logs on held-out seeds (first-step records: state
    features -> first step, spectral-radius bound, whole-integration cost;
    spectral-radius records along the trajectories: state features -> bound)."""
    t_start = time.perf_counter()
    wt = W.massaction(nsys=args.proposal_train, seed=1000 + rank)
    ht = B.register_workload(wt)
    log = torch.full((wt.nsys, wt.neq + 4), float("nan"), dtype=torch.float32, device=dev)
    lsr = torch.full((wt.nsys, args.proposal_sr_records, wt.neq + 2), float("nan"), dtype=torch.float32, device=dev)
    B.integrate("rkc", ht, torch.from_numpy(wt.y0).to(dev), torch.from_numpy(wt.params).to(dev), wt.t0, wt.tend,
                wt.rtol, wt.atol, precision=B.ODE_PREC_FP64, log_xy=log, log_sr=lsr,
                log_sr_every=args.proposal_sr_every, sync=True)
    B.release(ht)
    ok = torch.isfinite(log).all(dim=1)
    # first-step records (all three targets) and spectral-radius records
    # (sigma only: the other targets NaN, which the training skips)
    r = lsr.reshape(-1, wt.neq + 2)
    r = r[torch.isfinite(r).all(dim=1)]
    Y2 = torch.full((r.shape[0], 3), float("nan"), dtype=torch.float32, device=dev)
    Y2[:, 1] = r[:, wt.neq + 1]
    X = torch.cat([log[ok, :wt.neq + 1], r[:, :wt.neq + 1]]).contiguous()
    Y = torch.cat([log[ok, wt.neq + 1:], Y2]).contiguous()
    info = {"pairs": int(ok.sum().item()), "sigma_records": int(r.shape[0])}
    del lsr, r, Y2
    net = B.MLP(wt.neq + 1, seed=0)
    net.fit_normalization(X, Y)
    info["hist"] = net.train(X, Y, epochs=args.proposal_epochs, batch=4096, lr=2e-3, seed=0)
    torch.cuda.synchronize()
    info["seconds"] = time.perf_counter() - t_start
    return net, info


def proposal_leg(args, B, torch, dev, stream, rank, world, barrier, net, info):
    """The learned proposal on the 4,194,304-system mass-action batch:
    trained on records the plain FP64 solver logs on held-out seeds (state
    features -> first step, spectral-radius bound, whole-integration cost;
    and state features -> spectral-radius bound at later estimates), then
    the chosen form timed without it, with the proposed spectral radius
    (the Euler trial still sets the first step), with the proposed start
    (spectral radius and first step), with the network evaluated in the
    kernel at every spectral-radius point (with_sigma_every), and each of
    these with the batch taken longest-first by the predicted cost (the
    proposal and ordering passes are inside the timed step); every mode's
    error against the FP64 oracle on a sample.  For context, the order from
    the true costs of an earlier run on the same inputs bounds what any
    cost predictor can give."""
    import oracle as O
    t_train, n_sr_records, hist, n_pairs = info["seconds"], info["sigma_records"], info["hist"], info["pairs"]

    w = W.massaction(nsys=args.proposal_nsys, seed=4 + rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    yout = torch.empty_like(y0)
    CH = FORMS[args.chosen]
    B.prepare(h, "rkc", CH)
    true_cost = None

    no_h0 = torch.full((w.nsys,), float("nan"), dtype=torch.float32, device=dev)

    def step(mode, counters=None):
        kw = {}
        if mode.startswith("with_sigma_every"):
            # the network in the kernel at every spectral-radius point
            kw = dict(mlp=net)
            if mode.endswith("_ordered"):
                kw["cost"] = net.propose(y0, p, stream=stream.cuda_stream, with_cost=True)[2]
        elif mode.startswith("with_"):
            h0, s0, c = net.propose(y0, p, stream=stream.cuda_stream, with_cost=True)
            # with_sigma*: only the spectral radius (the Euler trial sets h0)
            kw = dict(h0=no_h0 if mode.startswith("with_sigma") else h0, sigma0=s0)
            if mode.endswith("_ordered"):
                kw["cost"] = c
        elif mode == "ordered_by_true_cost":
            kw = dict(cost=true_cost)
        B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=yout, counters=counters, precision=CH,
                    mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream, **kw)

    res = {}
    MODES = ("without", "with_sigma", "with_sigma_ordered", "with_proposal", "with_proposal_ordered",
             "with_sigma_every", "with_sigma_every_ordered", "ordered_by_true_cost")
    for mode in MODES:
        for _ in range(1):
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
            "y_sample": yout[:, :args.proposal_sample].cpu().numpy()}
        if mode == "with_proposal_ordered":
            pred = np.log(net.propose(y0, p, with_cost=True)[2].cpu().numpy())
            res[mode]["log_cost_corr_pred_vs_true"] = float(np.corrcoef(pred, np.log(c["n_rhs"]))[0, 1])
    res["ordered_by_true_cost"]["note"] = ("upper bound: order from the n_rhs counters of an earlier run on the "
                                           "same inputs (the previous global step in operator splitting)")
    B.release(h)
    ref = O.integrate_workload(W.subset(w, np.arange(args.proposal_sample)))
    for k, r in res.items():
        e = (np.abs(r.pop("y_sample") - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
        r["err_vs_fp64_oracle_max"] = float(e.max())
        r["err_vs_fp64_oracle_p999"] = float(np.quantile(e, 0.999))
        r["err_vs_fp64_oracle_median"] = float(np.median(e))
        r["meets_target"] = bool(r["err_vs_fp64_oracle_p999"] <= TARGET_P999)
    qual = [k for k in MODES if res[k]["meets_target"] and k != "ordered_by_true_cost"]
    res["fastest_within_target"] = max(qual, key=lambda k: res[k]["systems_per_s"]) if qual else None
    res["config"] = {"nsys_per_gpu": w.nsys, "train_pairs": n_pairs,
                     "train_sigma_records": n_sr_records,
                     "sigma_records_per_system": f"estimates 0, {args.proposal_sr_every}, ... (at most "
                                                 f"{args.proposal_sr_records})",
                     "train_seeds": "1000+rank",
                     "eval_seed": "4+rank", "epochs": args.proposal_epochs, "batch": 4096, "final_train_loss": float(hist[-1]),
                     "train_seconds_incl_logging": t_train,
                     "network": "14 -> 64 -> 64 -> 3 SiLU (log h0, log sigma, log cost), BF16 weights, "
                                "FP32 accumulate"}
    for k in MODES[1:]:
        res["speedup_" + k] = res["without"]["ms_per_step"] / res[k]["ms_per_step"]
    res["config"]["form"] = FORM_TEXT[BASE_FORM.get(args.chosen, args.chosen)]
    res["config"]["oracle_sample"] = args.proposal_sample
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
    """The chosen form's precision (without the learned proposal) on the
    mass-action batch with each spectral-radius estimate: the Appendix's power method (the paper's), the Gershgorin
    bound instead of it, and the power method capped by the bound."""
    import torch.distributed as dist
    w = W.massaction(nsys=args.nsys, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    y = torch.empty_like(y0)
    cnt = B.counters_like(w.nsys, dev)
    CH = FORMS[args.chosen]
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
    CH = FORMS[args.chosen]
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
                     "precision": FORM_TEXT[BASE_FORM.get(args.chosen, args.chosen)],
                     "state": "device resident (the paper copies each global step)"}
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
    res, y_runs = {}, {}
    # the FP32 lean plan autotuned and with the paper's fixed mapping; the
    # two-float plan (grids by two-float RKC, chains by two-float RKCK) and
    # the plain FP64 plan, both autotuned
    for name, mapping, prec in (("autotuned", B.ODE_MAP_AUTO, B.ODE_PREC_MIXED_LEAN),
                                ("fixed_thread_per_system", B.ODE_MAP_THREAD, B.ODE_PREC_MIXED_LEAN),
                                ("two_float_autotuned", B.ODE_MAP_AUTO, B.ODE_PREC_F2_LEAN),
                                ("fp64_autotuned", B.ODE_MAP_AUTO, B.ODE_PREC_FP64)):
        plan = B.RaggedPlan(handles, b.method, b.neq, b.offset[:-1], y0, prm, t0, tend, rtol, atol, y_out=y,
                            precision=prec, mapping=mapping, stream=stream.cuda_stream)
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
        if name != "fixed_thread_per_system":
            torch.cuda.synchronize()
            y_runs[name] = y.cpu().numpy()
    B.release(hb)
    B.release(hc)
    res["speedup_autotuned_vs_fixed"] = res["fixed_thread_per_system"]["ms_per_step"] / res["autotuned"]["ms_per_step"]
    res["speedup_two_float_vs_fp64"] = res["fp64_autotuned"]["ms_per_step"] / res["two_float_autotuned"]["ms_per_step"]
    res["config"] = {"nsys_per_gpu": b.nsys, "unknowns_total": int(b.offset[-1]),
                     "precision": "mixed lean (autotuned, fixed_thread_per_system); two-float RKC for the grids and "
                                  "two-float RKCK for the chains, FP32 scalars (two_float_autotuned); plain FP64 "
                                  "(fp64_autotuned)",
                     "graph": "one CUDA graph launch per step (all buckets on parallel branches)"}
    if rank == 0 and not args.no_cpu:
        # the error against the FP64 oracle on a sample (half grids, half chains)
        import oracle as O
        rng = np.random.default_rng(7)
        idx = np.sort(rng.choice(b.nsys, args.mixed_sample, replace=False))
        sub = W.mixed_subset(b, idx)
        t0 = time.perf_counter()
        ref = O.integrate_mixed(sub)
        cpu_s = time.perf_counter() - t0
        acc = {"sample": int(idx.size), "cpu_oracle_systems_per_s": idx.size / cpu_s, "cores": os.cpu_count()}
        for run_name, y_run in y_runs.items():
            per = {}
            for fam, kind in (("brusselator_rkc", W.RHS_BRUSS1D), ("vdp_chain_rkck", W.RHS_VDP_CHAIN)):
                e = []
                for k, i in enumerate(idx):
                    if b.kind[i] != kind:
                        continue
                    yg = y_run[b.offset[i]:b.offset[i] + b.neq[i]]
                    yr = ref.y[sub.offset[k]:sub.offset[k] + sub.neq[k]]
                    e.append(float(np.max(np.abs(yg - yr) / (np.abs(yr) + b.atol[i]))))
                e = np.array(e)
                per[fam] = {"systems": int(e.size), "median_rel_err": float(np.median(e)),
                            "p999_rel_err": float(np.quantile(e, 0.999)), "max_rel_err": float(e.max())}
            if run_name == "autotuned":
                acc.update(per)   # the lean plan's figures, at the top level as before
            else:
                acc[run_name] = per
        res["accuracy_vs_oracle"] = acc
    return res


def stoich_leg(args, B, mean_rhs, lean_ms):
    """The tensor-core question for the one contraction of the mass-action
    right-hand side, f = N r (Section 4.2's omega_i sums), measured on the
    benchmark network: the sparse FP32 form the generated integrators use
    against a warp-level TF32 tensor-core product with the rates split into
    two TF32 words (FP32-class accuracy), each timed over `reps` products
    per system minus a launch with none.  The per-step effect on the FP32
    lean form follows from its evaluations per system (mean_rhs) and its
    measured step (lean_ms, 1,048,576 systems)."""
    w = W.massaction(nsys=8, seed=0)
    h = B.register_workload(w)
    n, reps = args.stoich_nsys, args.stoich_reps
    res = {}
    for name, v in (("sparse_fp32", 0), ("tensor_tf32x2", 1)):
        t0, _ = B.stoich_bench(h, v, n, 0)
        t1, err = B.stoich_bench(h, v, n, reps)
        per = (t1 - t0) / reps
        res[name] = {"ms_per_product_over_batch": per, "ns_per_system_product": per * 1e6 / n,
                     "launch_ms_with_products": t1, "launch_ms_without": t0,
                     "max_err_vs_fp64_per_sum_of_terms": err}
    B.release(h)
    sp, tc = res["sparse_fp32"]["ms_per_product_over_batch"], res["tensor_tf32x2"]["ms_per_product_over_batch"]
    res["tensor_over_sparse_time"] = tc / sp
    if mean_rhs and lean_ms:
        delta = (tc - sp) * mean_rhs * (NSYS / n)
        res["lean_step_1m"] = {"measured_ms": lean_ms, "products_per_step_ms_sparse": sp * mean_rhs * (NSYS / n),
                               "estimated_ms_with_tensor_product": lean_ms + delta}
    res["config"] = {"nsys": n, "reps": reps, "network": "seed-0 mass-action, 13 species x 27 reactions",
                     "rates": "synthetic, log-uniform in [1e-8, 1e4]",
                     "tensor": "mma.sync m16n8k8 TF32 (leading + trailing TF32 words of the rates, exact integer "
                               "coefficients), FP32 accumulation; rates staged through shared memory into the "
                               "A-fragment layout, results back to one row per lane"}
    return res


def timed_calls(torch, stream, fn, steps, warmup, barrier):
    """Mean milliseconds of fn() over `steps` calls after `warmup` untimed
    ones (CUDA events on the launching stream)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def c0_leg(args, B, torch, dev, stream, rank, world, barrier):
    """Configuration c0: van der Pol systems by the plain FP64 RKCK (the
    paper's RKCK path; mu log-uniform in [0.1, 10], t in [0, 20], rtol 1e-6,
    atol 1e-9).  The configured 4096 systems fill 32 blocks of 128 threads
    (a fifth of the SMs), so a 1,048,576-system batch of the same
    distribution is timed too.  Step counts and final states against the
    oracle (all 4096 systems; a sample of the large batch), the oracle timed
    on the host cores on the same systems.  Beside the plain form, the
    two-float RKCK (FP32 scalars) on the same systems, with its error."""
    import oracle as O
    res = {}
    for nsys in (4096, args.c0_big):
        w = W.vdp(nsys, seed=rank)
        h = B.register_workload(w)
        y0 = torch.from_numpy(w.y0).to(dev)
        p = torch.from_numpy(w.params).to(dev)
        y = torch.empty_like(y0)
        cnt = B.counters_like(w.nsys, dev)
        runs = {}
        for form, prec in (("plain_fp64", B.ODE_PREC_FP64), ("two_float", B.ODE_PREC_F2_LEAN)):
            def call(counters=None):
                B.integrate("rkck", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=y, counters=counters,
                            precision=prec, mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream)

            ms = timed_calls(torch, stream, call, args.c0_steps, args.warmup, barrier)
            ms = max_over_ranks(ms, world, dev)
            call(cnt)
            torch.cuda.synchronize()
            c = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "status")}
            runs[form] = (ms, c, y.cpu().numpy(), B.mapping_info(h, "rkck", prec))
        B.release(h)
        ms, c, yg, mapping = runs["plain_fp64"]
        fl = rkck_flops(w, c["n_accept"], c["n_reject"])
        r = {"systems_per_s": w.nsys * world / (ms * 1e-3), "ms_per_step": ms,
             "rhs_evals_per_s": float(np.sum(c["n_rhs"])) * world / (ms * 1e-3),
             "mean_attempts": float(np.mean(c["n_accept"] + c["n_reject"])),
             "achieved_tflops_fp64": fl / (ms * 1e-3) / 1e12,
             "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
             "mapping_block_tuned": list(mapping)}
        ms2, c2, y2, mapping2 = runs["two_float"]
        r["two_float"] = {"systems_per_s": w.nsys * world / (ms2 * 1e-3), "ms_per_step": ms2,
                          "speedup_vs_plain": ms / ms2, "mapping_block_tuned": list(mapping2),
                          "status_ok_frac": float(np.mean((c2["status"] & 0xFF) == 0))}
        if rank == 0 and not args.no_cpu:
            if nsys <= 4096:
                idx = np.arange(nsys)
                t0 = time.perf_counter()
                ref = O.integrate_workload(w)
                rate = nsys / (time.perf_counter() - t0)
            else:
                idx, ref, rate = oracle_sample(w, args, seed=5)
            same = (c["n_accept"][idx] == ref.n_accept) & (c["n_reject"][idx] == ref.n_reject)
            e = (np.abs(yg[:, idx] - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
            r["parity"] = {"systems": int(idx.size), "same_counts_frac": float(same.mean()),
                           "max_rel_err_same_counts": float(e[same].max()) if same.any() else None,
                           "max_rel_err": float(e.max()),
                           "status_equal": bool(np.array_equal(c["status"][idx], ref.status))}
            r["cpu_oracle"] = {"systems_per_s": rate, "cores": os.cpu_count(), "sample": int(idx.size)}
            same2 = (c2["n_accept"][idx] == ref.n_accept) & (c2["n_reject"][idx] == ref.n_reject)
            e2 = (np.abs(y2[:, idx] - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
            r["two_float"]["err_vs_fp64_oracle"] = {
                "systems": int(idx.size), "median_rel_err": float(np.median(e2)),
                "p999_rel_err": float(np.quantile(e2, 0.999)), "max_rel_err": float(e2.max()),
                "same_counts_frac": float(same2.mean())}
        res[f"nsys_{nsys}"] = r
    res["config"] = {"method": "rkck", "precision": "plain FP64; two_float: two-float RKCK with FP32 scalars",
                     "rtol": 1e-6, "atol": 1e-9, "interval": [0.0, 20.0],
                     "flops_model": "6 evaluations x 5 flops + 60 N per attempt"}
    return res


def c1_leg(args, B, torch, dev, stream, rank, world, barrier):
    """Configuration c1: 1D Brusselator grids of 32 points (64 unknowns,
    one warp per system), RKC, rtol 1e-5, atol 1e-8, t in [0, 10], 65,536
    systems: the plain FP64 form against FP32 stages with FP64 bookkeeping
    (the configured comparison), with the lean and two-float forms beside
    them; error against the oracle on a sample, the oracle timed on it."""
    w = W.bruss(args.c1_nsys, n=32, seed=rank)
    h = B.register_workload(w)
    y0 = torch.from_numpy(w.y0).to(dev)
    p = torch.from_numpy(w.params).to(dev)
    y = torch.empty_like(y0)
    cnt = B.counters_like(w.nsys, dev)
    runs = {}
    for name in ("plain_fp64", "mixed_spec_split", "mixed_lean", "f2", "f2_lean"):
        prec = FORMS[name]

        def call(counters=None):
            B.integrate("rkc", h, y0, p, w.t0, w.tend, w.rtol, w.atol, y_out=y, counters=counters,
                        precision=prec, mapping=B.ODE_MAP_AUTO, stream=stream.cuda_stream)

        ms = timed_calls(torch, stream, call, args.c1_steps, 1, barrier)
        ms = max_over_ranks(ms, world, dev)
        call(cnt)
        torch.cuda.synchronize()
        c = {k: getattr(cnt, k).cpu().numpy() for k in ("n_accept", "n_reject", "n_rhs", "n_specrad_iter", "status")}
        runs[name] = {"ms": ms, "c": c, "y": y.cpu().numpy()}
    B.release(h)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    res = {}
    for name, r in runs.items():
        fl = rkc_flops(w, r["c"]["n_accept"], r["c"]["n_reject"], r["c"]["n_rhs"], r["c"]["n_specrad_iter"])
        ach = fl / (r["ms"] * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS if name == "plain_fp64" else fp32_peak_tflops(sm_count)
        res[name] = {"systems_per_s": w.nsys * world / (r["ms"] * 1e-3), "ms_per_step": r["ms"],
                     "rhs_evals_per_s": float(np.sum(r["c"]["n_rhs"])) * world / (r["ms"] * 1e-3),
                     "mean_rhs": float(np.mean(r["c"]["n_rhs"])), "achieved_tflops": ach,
                     "frac_peak": ach / peak, "peak": "fp64" if name == "plain_fp64" else "fp32",
                     "speedup_vs_plain": runs["plain_fp64"]["ms"] / r["ms"],
                     "status_ok_frac": float(np.mean((r["c"]["status"] & 0xFF) == 0))}
    if rank == 0 and not args.no_cpu:
        idx, ref, rate = oracle_sample(w, args, seed=11, min_n=1024)
        for name, r in runs.items():
            st = err_stats(r["y"][:, idx], ref.y, w.atol, w.rtol)
            same = (r["c"]["n_accept"][idx] == ref.n_accept) & (r["c"]["n_reject"][idx] == ref.n_reject)
            st["same_counts_frac"] = float(same.mean())
            res[name]["err_vs_fp64_oracle"] = st
        res["cpu_oracle"] = {"systems_per_s": rate, "cores": os.cpu_count(), "sample": int(idx.size)}
    res["config"] = {"nsys_per_gpu": w.nsys, "grid_points": 32, "neq": w.neq, "rtol": w.rtol, "atol": w.atol,
                     "interval": [w.t0, w.tend], "mapping": "one warp per system (ODE_MAP_AUTO block)",
                     "flops_model": "17 per grid point per evaluation; RKC vector terms as the main leg"}
    return res


def err_stats(y, ref_y, atol, rtol):
    """Per-system final-state error against the oracle: max_i |y - y_ref| /
    (|y_ref| + atol), summarised over the systems, and in tolerance units."""
    e = (np.abs(y - ref_y) / (np.abs(ref_y) + atol)).max(axis=0)
    tu = (np.abs(y - ref_y) / (atol + rtol * np.abs(ref_y))).max(axis=0)
    return {"median_rel_err": float(np.median(e)), "p999_rel_err": float(np.quantile(e, 0.999)),
            "max_rel_err": float(e.max()), "p999_err_in_tolerances": float(np.quantile(tu, 0.999))}


def oracle_sample(w, args, seed=123, min_n=4096):
    """Time the oracle (as it stands, all host cores) on a uniformly drawn
    sample of the batch sized for about args.cpu_seconds."""
    import oracle as O
    rng = np.random.default_rng(seed)
    probe = np.sort(rng.choice(w.nsys, min(2048, w.nsys), replace=False))
    t0 = time.perf_counter()
    O.integrate_workload(W.subset(w, probe))
    rate = probe.size / (time.perf_counter() - t0)
    n = int(min(w.nsys, max(min_n, rate * args.cpu_seconds)))
    idx = np.sort(rng.choice(w.nsys, n, replace=False))
    t0 = time.perf_counter()
    ref = O.integrate_workload(W.subset(w, idx))
    return idx, ref, n / (time.perf_counter() - t0)


def cpu_baseline(w, args, runs):
    """The oracle timed on a bounded sample of the same batch, and every GPU
    form compared with it on that sample."""
    import oracle as O
    cores = os.cpu_count() or 1
    idx, ref, rate = oracle_sample(w, args)
    n = idx.size
    base = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of {w.nsys} systems drawn uniformly (seed 123), full interval, all host cores"}
    acc = {"sample": n, "forms": {}}
    for name, r in runs.items():
        st = err_stats(r["y"][:, idx], ref.y, w.atol, w.rtol)
        same = (r["c"]["n_accept"][idx] == ref.n_accept) & (r["c"]["n_reject"][idx] == ref.n_reject)
        st["same_counts_frac"] = float(same.mean())
        if name == "plain_fp64":
            e = (np.abs(r["y"][:, idx] - ref.y) / (np.abs(ref.y) + w.atol)).max(axis=0)
            st["max_rel_err_same_counts"] = float(e[same].max()) if same.any() else None
        acc["forms"][name] = st
    # every form against an independent tight reference (RKCK, rtol 1e-12)
    # on a small sample: the forms' rounding next to the method's own error
    k = min(1024, n)
    sub_k = W.subset(w, idx[:k])
    tight = O.integrate(O.model_for(sub_k), 0, sub_k.y0, sub_k.params, sub_k.t0, sub_k.tend, 1e-12, 1e-18)
    vt = {"sample": k, "reference": "oracle RKCK rtol 1e-12 atol 1e-18"}
    e_ot = (np.abs(ref.y[:, :k] - tight.y) / (np.abs(tight.y) + w.atol)).max(axis=0)
    vt["fp64_oracle"] = {"max": float(e_ot.max()), "median": float(np.median(e_ot))}
    for name, r in runs.items():
        e = (np.abs(r["y"][:, idx[:k]] - tight.y) / (np.abs(tight.y) + w.atol)).max(axis=0)
        vt[name] = {"max": float(e.max()), "median": float(np.median(e))}
    acc["vs_tight_reference"] = vt
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
    ap.add_argument("--plain-steps", type=int, default=3, help="timed steps of the forms other than the chosen one "
                                                               "(0 skips them)")
    ap.add_argument("--chosen", choices=sorted(FORMS), default="f2_lean_learned",
                    help="the headline form (the fastest one that meets the accuracy target, as measured)")
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
    ap.add_argument("--proposal-sr-records", type=int, default=4,
                    help="spectral-radius training records per system (estimates 0, k, 2k, ...)")
    ap.add_argument("--proposal-sr-every", type=int, default=10)
    ap.add_argument("--proposal-sample", type=int, default=8192, help="systems of the leg compared with the oracle")
    ap.add_argument("--mixed-nsys", type=int, default=262144, help="0 skips the ragged-batch leg")
    ap.add_argument("--mixed-steps", type=int, default=3)
    ap.add_argument("--mixed-sample", type=int, default=1024, help="ragged systems compared with the oracle")
    ap.add_argument("--c0-steps", type=int, default=3, help="timed steps of the van der Pol RKCK leg (0 skips)")
    ap.add_argument("--c0-big", type=int, default=1 << 20, help="systems of the weak-scaled van der Pol batch")
    ap.add_argument("--c1-steps", type=int, default=2, help="timed steps per form of the Brusselator leg (0 skips)")
    ap.add_argument("--c1-nsys", type=int, default=65536)
    ap.add_argument("--stoich-reps", type=int, default=64, help="products per system of the tensor-core leg (0 skips)")
    ap.add_argument("--stoich-nsys", type=int, default=1 << 20)
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
