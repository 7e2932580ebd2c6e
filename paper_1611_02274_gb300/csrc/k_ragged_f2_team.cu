// k_ragged_f2_team.cu -- 8- and 16-lane team shapes of the two-float forms
// for the ragged scheduler's small size classes (two-float RKC for
// Brusselator grids of up to 16 points, two-float RKCK and RKC for chains of
// up to 16 oscillators; FP32 scalars, ODE_PREC_F2_LEAN).
#include "run_model.cuh"

namespace bode {

cudaError_t launch_bruss_shape_f2(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok) {
    *ok = true;
    if (team == 8 && g == 1) return launch_method<RkcF2<BrussModel<8, 1>, false, false>>(a, ctx, c);
    if (team == 16 && g == 1) return launch_method<RkcF2<BrussModel<16, 1>, false, false>>(a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

cudaError_t launch_chain_shape_f2(int method, int team, int g, const BatchArgs& a, const GridCtx& ctx,
                                  const LaunchCfg& c, bool* ok) {
    *ok = true;
    if (method == kMethodRkck) {
        if (team == 8 && g == 1) return launch_method<RkckF2<ChainModel<8, 1>, false>>(a, ctx, c);
        if (team == 16 && g == 1) return launch_method<RkckF2<ChainModel<16, 1>, false>>(a, ctx, c);
    } else {
        if (team == 8 && g == 1) return launch_method<RkcF2<ChainModel<8, 1>, false, false>>(a, ctx, c);
        if (team == 16 && g == 1) return launch_method<RkcF2<ChainModel<16, 1>, false, false>>(a, ctx, c);
    }
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
