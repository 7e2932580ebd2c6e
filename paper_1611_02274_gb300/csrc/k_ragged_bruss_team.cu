// k_ragged_bruss_team.cu -- extra team shapes of the bruss family for the ragged
// scheduler's autotuner (lean mixed form, RKC).
#include "run_model.cuh"

namespace bode {

cudaError_t launch_bruss_shape_team(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok) {
    *ok = true;
    if (team == 8 && g == 1) return launch_method<RkcMixed<BrussModel<8, 1>, false>>(a, ctx, c);
    if (team == 16 && g == 1) return launch_method<RkcMixed<BrussModel<16, 1>, false>>(a, ctx, c);
    if (team == 32 && g == 2) return launch_method<RkcMixed<BrussModel<32, 2>, false>>(a, ctx, c);
    if (team == 32 && g == 3) return launch_method<RkcMixed<BrussModel<32, 3>, false>>(a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
