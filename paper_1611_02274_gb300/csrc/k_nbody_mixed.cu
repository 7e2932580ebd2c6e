// k_nbody_mixed.cu -- planar n-body kernels (one body per lane: teams of 8
// or 16 lanes per system); mixed FP32/FP64 forms.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_nbody_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    const NbodyCtx ctx = nbody_ctx(r);
    if (r.neq <= 32) return run_model_mixed<NbodyModel<8>>(method, prec, a, ctx, c);
    if (r.neq <= 64) return run_model_mixed<NbodyModel<16>>(method, prec, a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
