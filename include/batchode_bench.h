/*
 * batchode_bench.h -- measurement helpers exported by libbatchode.so.
 *
 * Not part of the integration path.  The roofline of the integrators is an
 * ALU roofline (FP64 pipe for the plain form, FP32 pipe for the mixed and
 * two-float forms); bode_fma_peak measures the issue-limited FMA throughput
 * of the current device so that achieved FLOP/s can be quoted as a
 * fraction of it, and bode_stoich_bench measures whether the tensor cores
 * pay for the one contraction a right-hand side contains.
 */
#ifndef BATCHODE_BENCH_H
#define BATCHODE_BENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runs independent fused multiply-add chains on every SM of the current
 * device (fp64 != 0: double, else float) for `iters` iterations per chain
 * and writes the achieved GFLOP/s (2 flops per FMA) and the kernel time.
 * Synchronous.  Returns 0, or ODE_ERR_CUDA / ODE_ERR_ARG (iters < 1). */
int bode_fma_peak(int fp64, int32_t iters, double* gflops, double* ms);

/* The stoichiometry product of a registered mass-action network (rhs, a
 * handle from ode_rhs_register; at most 16 species and 32 reactions),
 * f = N r for synthetic rates r of nsys systems (a multiple of 128, at
 * most 2^26), repeated `reps` times per system, timed as one launch:
 * variant 0 the sparse FP32 form of the generated integrators (one add per
 * nonzero coefficient occurrence), variant 1 the warp-level tensor-core
 * form (mma.sync m16n8k8, TF32 operands with the rates split into two TF32
 * words, FP32 accumulation).  Writes the launch time; with reps > 0 and
 * max_err non-NULL also the largest error of the results against an FP64
 * evaluation, relative to the sum of |terms| of each species (every
 * reactant and product occurrence, as the sums are accumulated).  Synchronous;
 * compiles the kernels with NVRTC at first use and allocates its own
 * buffers.  Returns 0, or ODE_ERR_ARG / ODE_ERR_HANDLE / ODE_ERR_UNSUPPORTED
 * (NVRTC missing, network too large) / ODE_ERR_CUDA.  Section 4.2 gives the
 * omega_i sums this product forms. */
int bode_stoich_bench(int32_t rhs, int32_t variant, int64_t nsys, int32_t reps, double* ms, double* max_err);

#ifdef __cplusplus
}
#endif

#endif /* BATCHODE_BENCH_H */
