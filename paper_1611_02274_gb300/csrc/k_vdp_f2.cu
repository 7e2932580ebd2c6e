// k_vdp_f2.cu -- van der Pol kernels (one thread per system); two-float forms,
// RKCK and RKC.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_vdp_f2(int method, int prec, const RhsEntry&, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    return run_model_f2<VdpModel, true>(method, prec, a, NoCtx{}, c, ok);
}

}  // namespace bode
