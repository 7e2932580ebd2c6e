// k_kin_mixed.cu -- constant-volume kinetics kernels (one warp per system,
// rate constants and concentrations staged in shared memory); mixed
// FP32/FP64 forms.
#include "run_model.cuh"

namespace bode {

cudaError_t launch_kin_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    *ok = r.neq <= 64;
    if (!*ok) return cudaSuccess;
    return run_model_mixed<KinModel<32>>(method, prec, a, KinCtx{r.kin}, c);
}

}  // namespace bode
