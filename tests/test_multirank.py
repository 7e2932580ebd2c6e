"""The benchmark's multi-process host logic on CPU: two ranks over gloo.

Every rank integrates its own batch (seed = rank) with no exchange on the
data path; the only collectives are the barrier and the maximum of the step
times, which sets the whole-job rate (units of all ranks over the slowest
rank's time).  Without a GPU this checks the cross-rank maximum, the
aggregate rate and the distinct per-rank batches in two gloo processes, and
launches the reference arm through torch.distributed.run with two ranks:
rank 0 alone runs and prints one JSON line, rank 1 exits 0 without output.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_1611_02274_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, wsz, _ = bench.dist_env()
        mine = 10.0 + 7.0 * r                      # this rank's step time, ms
        slowest = bench.max_over_ranks(mine, wsz, "cpu")
        w = W.massaction(nsys=64, seed=r)          # each rank its own batch
        dist.barrier()
        q.put((r, wsz, slowest, float(np.sum(w.y0[0])), float(np.sum(w.params)),
               bench.aggregate_rate(w.nsys, wsz, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, m0, y0, p0, a0), (r1, w1, m1, y1, p1, a1) = got
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert m0 == m1 == 17.0                         # both ranks see the slower rank's time
    assert a0 == a1 == 64 * 2 / 17.0e-3             # all ranks' systems over that time
    assert y0 != y1 and p0 != p1                    # seeds differ: distinct batches
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5   # one rank: no collective


def test_reference_arm_under_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--steps", "1", "--warmup", "3", "--nsys", "4096", "--ref-sample", "32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["value"] == d["value"]
