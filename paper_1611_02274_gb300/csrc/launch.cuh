// launch.cuh -- batched kernels over the per-system state machines and the
// host-side launcher they share.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "team.cuh"

namespace bode {

// Registered right-hand side (host copy).
struct RhsEntry {
    int32_t kind;
    int32_t neq;
    int32_t n_params;
    MassActionNet net;
    double bruss_A, bruss_B, bruss_ubc, bruss_vbc;
    double coupling;
};

// Launch configuration resolved by the API layer.
struct LaunchCfg {
    int mapping;     // ODE_MAP_THREAD or ODE_MAP_QUEUE
    int block;       // threads per block
    int team;        // requested lanes per system (0 = family default)
    int sm_count;
    cudaStream_t stream;
};

// One system per team, one launch over the batch (the paper's intDriver
// mapping when the team is one thread), grid rounded up.  Each iteration
// evaluates the right-hand side once, at the point the system's phase needs.
template <class Method, class Ctx>
__global__ void __launch_bounds__(256) k_static(const BatchArgs a, const __grid_constant__ Ctx ctx) {
    constexpr int W = Method::W, P = Method::P;
    using R = typename Method::R;
    const Team<W> tm = Team<W>::make();
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    if (i >= a.nsys) return;  // team-uniform
    Method m;
    m.init(a, ctx, tm, i);
    R x[P], f[P];
    while (!m.done()) {
        R tx;
        m.point(x, tx);
        m.sys.rhs(tm, tx, x, f);
        m.consume(a, tm, f);
    }
    m.store(a, tm, i);
}

// Persistent kernel: each team pulls a system index from the queue cursor;
// every iteration of the loop evaluates the right-hand side once for every
// live team of the warp, at one call site, whatever phase each system is
// in.  A team whose system finishes stores it and pulls the next one before
// the next evaluation, so no lane idles while a slow neighbour finishes
// (the divergence tail of the static mapping).  The only inter-thread
// interaction is the atomic cursor.
template <class Method, class Ctx>
__global__ void __launch_bounds__(256) k_queue(const BatchArgs a, const __grid_constant__ Ctx ctx) {
    constexpr int W = Method::W, P = Method::P;
    using R = typename Method::R;
    const Team<W> tm = Team<W>::make();
    Method m;
    int64_t i = 0;
    bool live = false;
    // pull systems until one needs work (a zero-length interval finishes at init)
    auto next = [&]() {
        for (;;) {
            unsigned long long v = 0;
            if (tm.lane == 0) v = atomicAdd(a.cursor, 1ull);
            i = (int64_t)tm.bcast(v, 0);
            live = i < a.nsys;
            if (!live) return;
            m.init(a, ctx, tm, i);
            if (!m.done()) return;
            m.store(a, tm, i);
        }
    };
    next();
    R x[P], f[P];
    while (__any_sync(0xffffffffu, live)) {
        if (live) {
            R tx;
            m.point(x, tx);
            m.sys.rhs(tm, tx, x, f);
            if (m.consume(a, tm, f)) {
                m.store(a, tm, i);
                next();
            }
        }
    }
}

template <class Method, class Ctx>
cudaError_t launch_method(const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c) {
    constexpr int W = Method::W;
    const int block = c.block;
    const int64_t threads = a.nsys * W;
    if (c.mapping == ODE_MAP_QUEUE) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_queue<Method, Ctx>, block, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        int64_t grid = (int64_t)per_sm * c.sm_count;
        const int64_t need = (threads + block - 1) / block;
        if (grid > need) grid = need;
        k_queue<Method, Ctx><<<(unsigned)grid, block, 0, c.stream>>>(a, ctx);
    } else {
        const int64_t grid = (threads + block - 1) / block;
        k_static<Method, Ctx><<<(unsigned)grid, block, 0, c.stream>>>(a, ctx);
    }
    return cudaGetLastError();
}

enum { kMethodRkck = 0, kMethodRkc = 1 };

// Per-family dispatch (defined in k_*.cu).  Each sets *ok = false when the
// family / size / precision / mapping combination is not built.
cudaError_t launch_vdp(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_mass(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_bruss(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);

// Builds the RKC stage-coefficient tables on the current device.
cudaError_t build_rkc_tables(double* tab64, float4* tab32, int mmax, cudaStream_t s);

}  // namespace bode
