// launch.cuh -- batched kernels over the per-system state machines and the
// host-side launcher they share.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.cuh"
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
    double masses[kMaxBodies];
    KinDevice kin;          // device mechanism (ODE_RHS_KINETICS), freed at release
    void* kin_alloc;        // the one device allocation behind kin
};

// Launch configuration resolved by the API layer.
struct LaunchCfg {
    int mapping;     // ODE_MAP_THREAD or ODE_MAP_QUEUE
    int block;       // threads per block
    int team;        // requested lanes per system (0 = family default)
    int sm_count;
    cudaStream_t stream;
};

template <class Method, class Ctx>
cudaError_t launch_method(const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c) {
    constexpr int W = Method::W;
    const int block = c.block;
    const size_t smem = sizeof(float) * Method::SMEM_FLOATS * (size_t)block;
    const int64_t threads = a.nsys * W;
    if (smem > 48 * 1024) {  // above the default dynamic shared-memory limit: opt in
        cudaError_t e = cudaFuncSetAttribute(k_static<Method, Ctx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_queue<Method, Ctx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (c.mapping == ODE_MAP_QUEUE) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_queue<Method, Ctx>, block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        int64_t grid = (int64_t)per_sm * c.sm_count;
        const int64_t need = (threads + block - 1) / block;
        if (grid > need) grid = need;
        BatchArgs q = a;
        q.warp_sched = 1;
        k_queue<Method, Ctx><<<(unsigned)grid, block, smem, c.stream>>>(q, ctx);
    } else {
        const int64_t grid = (threads + block - 1) / block;
        k_static<Method, Ctx><<<(unsigned)grid, block, smem, c.stream>>>(a, ctx);
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
cudaError_t launch_nbody(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_kinetics(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);

// Builds the RKC stage-coefficient tables on the current device.
cudaError_t build_rkc_tables(double* tab64, float4* tab32, int mmax, cudaStream_t s);

}  // namespace bode
