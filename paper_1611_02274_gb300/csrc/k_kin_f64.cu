// k_kin_f64.cu -- constant-volume kinetics kernels (one warp per system,
// rate constants and concentrations staged in shared memory); plain FP64
// form; compiled without multiply-add contraction.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_kin_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = r.neq <= 64;
    if (!*ok) return cudaSuccess;
    return run_model_prec<KinModel<32>, ODE_PREC_FP64>(method, a, KinCtx{r.kin}, c);
}

}  // namespace bode
