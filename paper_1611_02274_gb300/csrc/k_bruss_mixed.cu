// k_bruss_mixed.cu -- Brusselator kernels, one warp per system (grid point g = q * 32 + lane);
// mixed FP32/FP64 form.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_bruss_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    (void)r;
    if (r.neq <= 64) return run_model_mixed<BrussModel<32, 1>>(method, prec, a, grid_ctx(r), c);
    if (r.neq <= 256) return run_model_mixed<BrussModel<32, 4>>(method, prec, a, grid_ctx(r), c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
