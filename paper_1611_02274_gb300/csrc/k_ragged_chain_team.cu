// k_ragged_chain_team.cu -- extra team shapes of the chain family for the ragged
// scheduler's autotuner (lean mixed form, RKCK).
#include "run_model.cuh"

namespace bode {

cudaError_t launch_chain_shape_team(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok) {
    *ok = true;
    if (team == 8 && g == 1) return launch_method<RkckMixed<ChainModel<8, 1>, false>>(a, ctx, c);
    if (team == 16 && g == 1) return launch_method<RkckMixed<ChainModel<16, 1>, false>>(a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
