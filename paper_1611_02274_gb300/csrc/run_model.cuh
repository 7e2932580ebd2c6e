// run_model.cuh -- instantiate the integrator forms for one model.
#pragma once
#include "integrators.cuh"
#include "launch.cuh"
#include "rhs.cuh"

namespace bode {

// one precision only (lets a family split its kernels over translation units)
template <class Model, int PREC, class Ctx>
cudaError_t run_model_prec(int method, const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c) {
    if constexpr (PREC == ODE_PREC_FP64) {
        if (method == kMethodRkck) return launch_method<RkckF64<Model>>(a, ctx, c);
        return launch_method<RkcF64<Model>>(a, ctx, c);
    } else if constexpr (PREC == ODE_PREC_MIXED) {
        if (method == kMethodRkck) return launch_method<RkckMixed<Model, true>>(a, ctx, c);
        return launch_method<RkcMixed<Model, true>>(a, ctx, c);
    } else {
        if (method == kMethodRkck) return launch_method<RkckMixed<Model, false>>(a, ctx, c);
        return launch_method<RkcMixed<Model, false>>(a, ctx, c);
    }
}

// both mixed modes (FP64 or compensated FP32 error-norm accumulation)
template <class Model, class Ctx>
cudaError_t run_model_mixed(int method, int prec, const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c) {
    if (prec == ODE_PREC_MIXED) return run_model_prec<Model, ODE_PREC_MIXED>(method, a, ctx, c);
    return run_model_prec<Model, ODE_PREC_MIXED_LEAN>(method, a, ctx, c);
}

// two-float forms: the variant with the warp-level code (M1) for the work
// queue and the in-kernel network, where the model supports it; otherwise
// the plain variant (M0)
template <class M0, class M1, class Ctx>
cudaError_t launch_f2(const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c) {
    if constexpr (M1::kWarpPropose) {
        if (a.mlp != nullptr || c.mapping == ODE_MAP_QUEUE) return launch_method<M1>(a, ctx, c);
    }
    return launch_method<M0>(a, ctx, c);
}

// two-float forms: RKC, and RKCK where a unit builds it (RKCK = true)
template <class Model, bool RKCK = false, class Ctx>
cudaError_t run_model_f2(int method, int prec, const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c, bool* ok) {
    if (method == kMethodRkck) {
        *ok = RKCK;
        if constexpr (RKCK) {
            if (prec == ODE_PREC_F2) return launch_method<RkckF2<Model, true>>(a, ctx, c);
            return launch_method<RkckF2<Model, false>>(a, ctx, c);
        }
        return cudaSuccess;
    }
    *ok = true;
    if (prec == ODE_PREC_F2) return launch_f2<RkcF2<Model, true, false>, RkcF2<Model, true, true>>(a, ctx, c);
    return launch_f2<RkcF2<Model, false, false>, RkcF2<Model, false, true>>(a, ctx, c);
}

template <class Model, class Ctx>
cudaError_t run_model(int method, int prec, const BatchArgs& a, const Ctx& ctx, const LaunchCfg& c) {
    if (method == kMethodRkck) {
        if (prec == ODE_PREC_FP64) return launch_method<RkckF64<Model>>(a, ctx, c);
        return launch_method<RkckMixed<Model>>(a, ctx, c);
    }
    if (prec == ODE_PREC_FP64) return launch_method<RkcF64<Model>>(a, ctx, c);
    return launch_method<RkcMixed<Model>>(a, ctx, c);
}

inline GridCtx grid_ctx(const RhsEntry& r) {
    return GridCtx{r.bruss_A, r.bruss_B, r.bruss_ubc, r.bruss_vbc, r.coupling};
}

inline NbodyCtx nbody_ctx(const RhsEntry& r) {
    NbodyCtx c;
    for (int b = 0; b < kMaxBodies; ++b) c.m[b] = b < r.neq / 4 ? r.masses[b] : 0.0;
    return c;
}

}  // namespace bode
