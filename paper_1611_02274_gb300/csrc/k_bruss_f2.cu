// k_bruss_f2.cu -- Brusselator RKC kernels, one warp per system (grid point
// g = q * 32 + lane); two-float forms.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_bruss_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (r.neq <= 64) return run_model_f2<BrussModel<32, 1>>(method, prec, a, grid_ctx(r), c, ok);
    if (r.neq <= 256) return run_model_f2<BrussModel<32, 4>>(method, prec, a, grid_ctx(r), c, ok);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
