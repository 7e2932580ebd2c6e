// kernels.cuh -- the batched kernels that drive the per-system integrators
// (device code only; also compiled at run time for generated right-hand sides).
#pragma once
#include "common.cuh"
#include "team.cuh"

// Launch bounds: at most BODE_MAX_THREADS threads per block and, when
// BODE_MIN_BLOCKS > 1, a register budget that keeps that many blocks resident
// per SM (the run-time compiled kernels take both from tuning options).
#ifndef BODE_MAX_THREADS
#define BODE_MAX_THREADS 256
#endif
#ifndef BODE_MIN_BLOCKS
#define BODE_MIN_BLOCKS 1
#endif
// Block lockstep of the one-launch mapping (run-time compiled kernels):
// 0 -- each warp loops on its own; 1 -- the warps of a block take their
// iterations together (a block-wide vote ends the loop); 2 -- as 1, and the
// step-end hold waits for every system of the block, so the block's warps
// also run the same phase of the step.
#ifndef BODE_LOCKSTEP
#define BODE_LOCKSTEP 0
#endif

namespace bode {

// Dynamic shared memory of the methods (and models) that keep data there:
// Method::SMEM_FLOATS floats per thread, launched with SMEM_FLOATS *
// blockDim floats.  bind_smem receives the block's base and blockDim; a
// per-thread column starts at base + threadIdx.x with stride blockDim, a
// per-team region is carved from the base by the team's index.
extern __shared__ __align__(16) float bode_dyn_smem[];

template <class Method>
__device__ __forceinline__ void bind_method_smem(Method& m) {
    if constexpr (Method::SMEM_FLOATS > 0) m.bind_smem(bode_dyn_smem, (int)blockDim.x);
}

// Step-end hold (methods with a variable stage count, Method::kStepSync):
// a system whose stages are done and whose next evaluation closes the step
// (F_{n+1}, then the error test and the next step's set-up) waits while
// any system of the warp is still in its stages.  The step-closing work
// then runs once for all lanes that reached it, instead of once per lane
// in different iterations; the price is idle evaluation slots of the lanes
// with fewer stages.  Every iteration in which a lane is in its stages
// advances that lane, so the hold always ends.  The arithmetic of each
// system is unchanged.
template <class Method, int LOCK = 0>
__device__ __forceinline__ bool step_hold(const Method& m, bool live) {
    if constexpr (Method::kStepSync && Method::W < 32) {
        const bool staging = LOCK == 2 ? __syncthreads_or(live && m.in_stages()) != 0
                                       : __any_sync(0xffffffffu, live && m.in_stages());
        return live && staging && m.at_step_end();
    } else {
        return false;
    }
}

// In-kernel proposal network (methods with kWarpPropose): a warp-wide
// evaluation for the lanes at a spectral-radius point, before the warp's
// next right-hand-side evaluation.  Every lane calls.
template <class M, class = void>
struct WarpPropose {
    static constexpr bool value = false;
};
template <class M>
struct WarpPropose<M, void_t_<decltype(M::kWarpPropose)>> {
    static constexpr bool value = M::kWarpPropose;
};
template <class Method>
__device__ __forceinline__ void warp_propose(Method& m, const BatchArgs& a, const Team<Method::W>& tm, bool live,
                                             int64_t i) {
    if constexpr (WarpPropose<Method>::value) m.propose_warp(a, tm, live, i);
}

// Register budget of a method's kernels: Method::kMaxRegs when it declares
// one, else 255 (the launch bounds alone decide).  Every block size stays
// launchable (168 registers x 256 threads fit in an SM's register file).
template <class M, class = void>
struct KernelRegs {
    static constexpr int value = 255;
};
template <class M>
struct KernelRegs<M, void_t_<decltype(M::kMaxRegs)>> {
    static constexpr int value = M::kMaxRegs;
};

// One system per team, one launch over the batch (the paper's intDriver
// mapping when the team is one thread), grid rounded up.  Each iteration
// evaluates the right-hand side once, at the point the system's phase needs.
// Lanes past the end of the batch stay in the loop (inactive) so that the
// warp votes see every lane.
template <class Method, class Ctx>
__global__ void __launch_bounds__(BODE_MAX_THREADS, BODE_MIN_BLOCKS) __maxnreg__(KernelRegs<Method>::value) k_static(const BatchArgs a, const __grid_constant__ Ctx ctx) {
    constexpr int W = Method::W, P = Method::P;
    using R = typename Method::R;
    const Team<W> tm = Team<W>::make();
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const bool in_range = k < a.nsys;  // team-uniform
    Method m;
    bind_method_smem(m);
    int64_t i = 0;
    if (in_range) {
        i = a.sys_of(k);
        m.init(a, ctx, tm, i);
    }
    R x[P], f[P];
    if constexpr (Method::kStepSync && W < 32) {
        for (;;) {
            const bool live = in_range && !m.done();
            if constexpr (BODE_LOCKSTEP > 0) {
                if (!__syncthreads_or(live)) break;  // every thread of the block takes part
            } else {
                if (!__any_sync(0xffffffffu, live)) break;
            }
            warp_propose(m, a, tm, live, i);                      // every lane takes part
            const bool hold = step_hold<Method, BODE_LOCKSTEP>(m, live);  // a vote: every lane takes part
            if (live && !hold) {
                R tx;
                m.point(x, tx);
                m.sys.rhs(tm, tx, x, f);
                m.consume(a, tm, x, f);
            }
        }
    } else if (in_range) {  // one team per warp, or a fixed stage count: nothing to hold for
        while (!m.done()) {
            R tx;
            m.point(x, tx);
            m.sys.rhs(tm, tx, x, f);
            m.consume(a, tm, x, f);
        }
    }
    if (in_range) m.store(a, tm, i);
}

// Persistent kernel: each team pulls a system index from the queue cursor;
// every iteration of the loop evaluates the right-hand side once for every
// live team of the warp, at one call site, whatever phase each system is
// in.  A team whose system finishes stores it and pulls the next one before
// the next evaluation, so no lane idles while a slow neighbour finishes
// (the divergence tail of the static mapping).  The only inter-thread
// interaction is the atomic cursor.
template <class Method, class Ctx>
__global__ void __launch_bounds__(BODE_MAX_THREADS, BODE_MIN_BLOCKS) __maxnreg__(KernelRegs<Method>::value) k_queue(const BatchArgs a, const __grid_constant__ Ctx ctx) {
    constexpr int W = Method::W, P = Method::P;
    using R = typename Method::R;
    const Team<W> tm = Team<W>::make();
    Method m;
    bind_method_smem(m);
    int64_t i = 0;
    bool live = false;
    // pull systems until one needs work (a zero-length interval finishes at init)
    auto next = [&]() {
        for (;;) {
            unsigned long long v = 0;
            if (tm.lane == 0) v = atomicAdd(a.cursor, 1ull);
            const int64_t k = (int64_t)tm.bcast(v, 0);
            live = k < a.nsys;
            if (!live) return;
            i = a.sys_of(k);
            m.init(a, ctx, tm, i);
            if (!m.done()) return;
            m.store(a, tm, i);
        }
    };
    next();
    R x[P], f[P];
    // The evaluation loop runs until a system of the warp finishes; the
    // switch to the next systems runs outside it, before the next
    // evaluation (the same order of events as switching inside it).  Kept
    // apart, the loop does not carry the register demand of the set-up code:
    // with the switch inside, the compiler spilled the method's state around
    // it in every iteration.
    while (__any_sync(0xffffffffu, live)) {
        bool fin = false;
        for (;;) {
            warp_propose(m, a, tm, live, i);       // every lane takes part
            const bool hold = step_hold(m, live);  // a warp vote: every lane takes part
            if (live && !hold) {
                R tx;
                m.point(x, tx);
                m.sys.rhs(tm, tx, x, f);
                fin = m.consume(a, tm, x, f);
            }
            if (__any_sync(0xffffffffu, fin)) break;
        }
        if (fin) {
            m.store(a, tm, i);
            next();
        }
    }
}

}  // namespace bode
