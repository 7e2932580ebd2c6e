// k_nbody_f64.cu -- planar n-body kernels (one body per lane: teams of 8
// or 16 lanes per system); plain FP64 form; compiled without multiply-add
// contraction.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_nbody_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    const NbodyCtx ctx = nbody_ctx(r);
    if (r.neq <= 32) return run_model_prec<NbodyModel<8>, ODE_PREC_FP64>(method, a, ctx, c);
    if (r.neq <= 64) return run_model_prec<NbodyModel<16>, ODE_PREC_FP64>(method, a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
