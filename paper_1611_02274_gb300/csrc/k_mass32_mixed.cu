// k_mass32_mixed.cu -- mass-action kernels for networks of <= 32 species and <= 64 reactions
// (one thread per system, reaction loop not unrolled);
// mixed FP32/FP64 form.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_mass32_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    return run_model_mixed<MassActionModel<32, 64>>(method, prec, a, r.net, c);
}

}  // namespace bode
