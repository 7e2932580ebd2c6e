// k_mass16_f64.cu -- mass-action kernels for networks of <= 16 species and <= 32 reactions
// (one thread per system, reaction loop unrolled);
// plain FP64 form; compiled without multiply-add contraction.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_mass16_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    return run_model_prec<MassActionModel<16, 32>, ODE_PREC_FP64>(method, a, r.net, c);
}

}  // namespace bode
