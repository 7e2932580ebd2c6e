// k_chain_f2.cu -- coupled van der Pol chain kernels, one warp per system
// (oscillator g = q * 32 + lane); two-float forms, RKCK and RKC.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_chain_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (r.neq <= 64) return run_model_f2<ChainModel<32, 1>, true>(method, prec, a, grid_ctx(r), c, ok);
    if (r.neq <= 128) return run_model_f2<ChainModel<32, 2>, true>(method, prec, a, grid_ctx(r), c, ok);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
