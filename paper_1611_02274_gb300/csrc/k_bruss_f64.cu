// k_bruss_f64.cu -- Brusselator kernels, one warp per system (grid point g = q * 32 + lane);
// plain FP64 form; compiled without multiply-add contraction.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_bruss_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    (void)r;
    if (r.neq <= 64) return run_model_prec<BrussModel<32, 1>, ODE_PREC_FP64>(method, a, grid_ctx(r), c);
    if (r.neq <= 256) return run_model_prec<BrussModel<32, 4>, ODE_PREC_FP64>(method, a, grid_ctx(r), c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
