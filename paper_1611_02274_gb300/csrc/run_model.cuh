// run_model.cuh -- instantiate the four integrator forms for one model.
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
    } else {
        if (method == kMethodRkck) return launch_method<RkckMixed<Model>>(a, ctx, c);
        return launch_method<RkcMixed<Model>>(a, ctx, c);
    }
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

}  // namespace bode
