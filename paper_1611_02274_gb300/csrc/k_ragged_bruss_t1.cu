// k_ragged_bruss_t1.cu -- extra team shapes of the bruss family for the ragged
// scheduler's autotuner (lean mixed form, RKC).
#include "run_model.cuh"

namespace bode {

cudaError_t launch_bruss_shape_t1(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok) {
    *ok = true;
    if (team == 1 && g == 4) return launch_method<RkcMixed<BrussModel<1, 4>, false>>(a, ctx, c);
    if (team == 1 && g == 128) return launch_method<RkcMixed<BrussModel<1, 128>, false>>(a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
