"""The benchmark's algorithmic flop model, the numerator of its roofline
figure, on a hand-built network: one mass-action evaluation costs |R|
multiplications per reaction (rate constant times each reactant
occurrence) plus one accumulation per reactant and product occurrence;
the RKC total is linear in the per-system counters and charges every
evaluation that price."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1611_02274_gb300 import workloads as W  # noqa: E402


def tiny_network():
    # A -> B, A + B -> C, 2A -> B + C
    return W.Network(3, np.array([1, 2, 2], np.int32), np.array([[0, -1], [0, 1], [0, 0]], np.int32),
                     np.array([1, 1, 2], np.int32), np.array([[1, -1], [2, -1], [1, 2]], np.int32),
                     np.zeros(3), np.zeros(3), np.zeros(3))


def test_rhs_flops_counts_the_mass_action_law():
    w = W.Workload("tiny", W.RHS_MASSACTION, W.METHOD_RKC, 1, 3, np.ones((3, 1)), np.ones((1, 1)),
                   0.0, 1.0, 1e-6, 1e-12, network=tiny_network())
    # k C_A, then -r to A, +r to B                  : 1 + 2 (1 + 1) = 5
    # k C_A C_B, then -r to A and B, +r to C        : 2 + 2 (2 + 1) = 8
    # k C_A C_A, then -r twice to A, +r to B and C  : 2 + 2 (2 + 2) = 10
    # (each scatter update a multiply-add with the stoichiometric sign: 2 flops)
    assert bench.rhs_flops(w) == 5 + 8 + 10


def test_rkc_flops_is_linear_in_the_counters_and_prices_each_evaluation():
    w = W.massaction(nsys=4, seed=0)
    rng = np.random.default_rng(0)
    acc = rng.integers(500, 1500, 4)
    rej = rng.integers(0, 3, 4)
    sr = rng.integers(10, 90, 4)
    rhs = 2 + sr + 2 * (acc + rej)                      # m = 2 on every attempt
    total = bench.rkc_flops(w, acc, rej, rhs, sr)
    per = [bench.rkc_flops(w, acc[i:i + 1], rej[i:i + 1], rhs[i:i + 1], sr[i:i + 1]) for i in range(4)]
    assert total == sum(per)                             # a sum over systems
    one_more = bench.rkc_flops(w, acc[:1], rej[:1], rhs[:1] + 1, sr[:1] + 1)   # one more power iteration
    assert one_more - per[0] == bench.rhs_flops(w) + 6 * w.neq
    # one more accepted two-stage step: two evaluations, N (2 + 9 + 11) vector flops, 15 coefficient flops
    one_step = bench.rkc_flops(w, acc[:1] + 1, rej[:1], rhs[:1] + 2, sr[:1])
    assert one_step - per[0] == 2 * bench.rhs_flops(w) + 22 * w.neq + 15


def test_seed0_network_flops():
    # the benchmark network: 45 reactant and 38 product occurrences
    w = W.massaction(nsys=1, seed=0)
    assert int(w.network.n_reac.sum()) == 45 and int(w.network.n_prod.sum()) == 38
    assert bench.rhs_flops(w) == 3 * 45 + 2 * 38


def test_rkck_and_other_families():
    v = W.vdp(2)
    assert bench.rhs_flops(v) == 5
    assert bench.rkck_flops(v, np.array([10]), np.array([2])) == 12 * (6 * 5 + 60 * 2)
    assert bench.rhs_flops(W.bruss(2, n=32)) == 17 * 32


def test_aggregate_rate_is_all_ranks_units_over_the_slowest_time():
    assert bench.aggregate_rate(1 << 20, 1, 52.0) == (1 << 20) / 0.052
    assert bench.aggregate_rate(1 << 20, 8, 52.0) == 8 * (1 << 20) / 0.052


def test_every_precision_form_is_described_everywhere():
    # each form the bench times has its precision code, kernel, dtype,
    # launch count and description; the learned forms name the form
    # underneath them, which has the same precision code
    for table in (bench.FORM_KERNELS, bench.FORM_DTYPES, bench.LAUNCHES, bench.FORM_TEXT):
        assert set(bench.FORMS) <= set(table)
    for name in bench.LEARNED_FORMS:
        base = bench.BASE_FORM[name]
        assert bench.FORMS[name] == bench.FORMS[base]
        assert bench.FORM_KERNELS[name] == bench.FORM_KERNELS[base]
        # proposal pre-pass, four cost-order kernels, rate prologue, integration
        assert bench.LAUNCHES[name] == bench.LAUNCHES[base] + 5
    assert bench.FORMS["plain_fp64"] == 0


def test_ncu_context_of_the_chosen_form_is_self_consistent():
    # the executed FP32 flops per system and the instructions per method
    # flop come from one capture of 262,144 systems
    ctx = bench.NCU_PIPE_CONTEXT["f2_lean_learned"]
    assert 0.0 < ctx["fma_pipe_cycles_active"] <= ctx["issue_active"] <= 1.0
    flops_262k = ctx["fp32_flops_executed_per_system"] * 262144
    # FP32 flops (FMA = 2) exceed the FP32 instructions, which exceed the method flops
    assert flops_262k > ctx["fp32_thread_inst_per_method_flop"] * 197.86e9 > 197.86e9
