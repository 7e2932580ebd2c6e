// dispatch.cu -- route a call to the kernels of its family, size and precision.
#include "launch.cuh"

namespace bode {

cudaError_t launch_vdp_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_vdp_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_mass16_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_mass16_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_mass32_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_mass32_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_bruss_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_bruss_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_nbody_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_kin_f64(int method, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_kin_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_nbody_mixed(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_vdp_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_mass16_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_bruss_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain_f2(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok);

namespace {
inline bool f64(int prec) { return prec == ODE_PREC_FP64; }
// families without two-float kernels
inline cudaError_t none(bool* ok) {
    *ok = false;
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_vdp(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (prec_is_f2(prec)) return launch_vdp_f2(method, prec, r, a, c, ok);
    return f64(prec) ? launch_vdp_f64(method, r, a, c, ok) : launch_vdp_mixed(method, prec, r, a, c, ok);
}

cudaError_t launch_mass(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (prec_is_f2(prec))
        return r.net.n_species <= 16 && r.net.n_reactions <= 32 ? launch_mass16_f2(method, prec, r, a, c, ok) : none(ok);
    if (r.net.n_species <= 16 && r.net.n_reactions <= 32)
        return f64(prec) ? launch_mass16_f64(method, r, a, c, ok) : launch_mass16_mixed(method, prec, r, a, c, ok);
    return f64(prec) ? launch_mass32_f64(method, r, a, c, ok) : launch_mass32_mixed(method, prec, r, a, c, ok);
}

cudaError_t launch_bruss(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (prec_is_f2(prec)) return launch_bruss_f2(method, prec, r, a, c, ok);
    return f64(prec) ? launch_bruss_f64(method, r, a, c, ok) : launch_bruss_mixed(method, prec, r, a, c, ok);
}

cudaError_t launch_chain(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (prec_is_f2(prec)) return launch_chain_f2(method, prec, r, a, c, ok);
    return f64(prec) ? launch_chain_f64(method, r, a, c, ok) : launch_chain_mixed(method, prec, r, a, c, ok);
}

cudaError_t launch_nbody(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (prec_is_f2(prec)) return none(ok);
    return f64(prec) ? launch_nbody_f64(method, r, a, c, ok) : launch_nbody_mixed(method, prec, r, a, c, ok);
}

cudaError_t launch_kinetics(int method, int prec, const RhsEntry& r, const BatchArgs& a, const LaunchCfg& c, bool* ok) {
    if (prec_is_f2(prec)) return none(ok);
    return f64(prec) ? launch_kin_f64(method, r, a, c, ok) : launch_kin_mixed(method, prec, r, a, c, ok);
}

}  // namespace bode
