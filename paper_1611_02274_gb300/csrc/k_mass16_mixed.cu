// k_mass16_mixed.cu -- mass-action kernels for networks of <= 16 species and <= 32 reactions
// (one thread per system, reaction loop unrolled);
// mixed FP32/FP64 form.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_mass16_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    return run_model_mixed<MassActionModel<16, 32>>(method, prec, a, r.net, c);
}

}  // namespace bode
