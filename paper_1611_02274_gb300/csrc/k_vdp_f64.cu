// k_vdp_f64.cu -- van der Pol kernels (one thread per system);
// plain FP64 form; compiled without multiply-add contraction.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_vdp_f64(int method, const RhsEntry&, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = true;
    return run_model_prec<VdpModel, ODE_PREC_FP64>(method, a, NoCtx{}, c);
}

}  // namespace bode
