// k_vdp_mixed.cu -- van der Pol kernels (one thread per system);
// mixed FP32/FP64 form.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_vdp_mixed(int method, int prec, const RhsEntry&, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    return run_model_mixed<VdpModel>(method, prec, a, NoCtx{}, c);
}

}  // namespace bode
