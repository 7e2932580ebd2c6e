/*
 * batchode_bench.h -- measurement helpers exported by libbatchode.so.
 *
 * Not part of the integration path.  The roofline of the integrators is an
 * ALU roofline (FP64 pipe for the plain form, FP32 pipe for the mixed
 * form); these entry points measure the issue-limited FMA throughput of the
 * current device so that achieved FLOP/s can be quoted as a fraction of it.
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

#ifdef __cplusplus
}
#endif

#endif /* BATCHODE_BENCH_H */
