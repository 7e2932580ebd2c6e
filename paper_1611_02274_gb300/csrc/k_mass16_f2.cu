// k_mass16_f2.cu -- mass-action RKC kernels for networks of <= 16 species and
// <= 32 reactions (one thread per system, reaction loop unrolled); two-float
// forms.  Generated network code (jit.cu) takes precedence where NVRTC is present.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_mass16_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    return run_model_f2<MassActionModel<16, 32>>(method, prec, a, r.net, c, ok);
}

}  // namespace bode
