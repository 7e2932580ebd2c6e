// k_ragged_chain_t1.cu -- extra team shapes of the chain family for the ragged
// scheduler's autotuner (lean mixed form, RKCK).
#include "run_model.cuh"

namespace bode {

cudaError_t launch_chain_shape_t1(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok) {
    *ok = true;
    if (team == 1 && g == 4) return launch_method<RkckMixed<ChainModel<1, 4>, false>>(a, ctx, c);
    if (team == 1 && g == 64) return launch_method<RkckMixed<ChainModel<1, 64>, false>>(a, ctx, c);
    *ok = false;
    return cudaSuccess;
}

}  // namespace bode
