// common.cuh -- shared device definitions of the batched integrators.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "batchode.h"

namespace bode {

// An integer the optimiser cannot see through.  A loop that writes only the
// element whose index equals a run-time value would otherwise be rewritten
// as one indexed store, and an indexed store forces the whole per-system
// state object out of registers into local memory.
__device__ __forceinline__ int opaque(int x) {
    asm("" : "+r"(x));
    return x;
}

// Constants of the paper's listings (Section 3.1 constants, Section 3.2).
constexpr double kUround = 2.22e-16;
constexpr double kSafety = 0.9;
constexpr double kPgrow = -0.2;
constexpr double kPshrnk = -0.25;
constexpr double kErrcon = 1.89e-4;
constexpr double kTiny = 1.0e-30;
constexpr double kP1 = 0.1;  // factor-of-ten limit on step decreases (P1 of the listings)
constexpr int kSpecradItmax = 50;
constexpr int kSpecradEvery = 25;

constexpr int kMaxReactions = 64;
constexpr int kMaxSpecies = 32;

// One registered mass-action network, passed to kernels by value (lives in
// the kernel-parameter constant bank, so warp-uniform reads broadcast).
struct MassActionNet {
    int32_t n_species;
    int32_t n_reactions;
    double kmin, kmax;
    int8_t n_reac[kMaxReactions];
    int8_t n_prod[kMaxReactions];
    int8_t reac[kMaxReactions][2];
    int8_t prod[kMaxReactions][2];
    double log10A[kMaxReactions];
    double beta[kMaxReactions];
    double Ea[kMaxReactions];
};

// Compile-time type choice (the run-time compiler has no <type_traits>).
template <bool B, class T, class F>
struct Pick {
    using type = T;
};
template <class T, class F>
struct Pick<false, T, F> {
    using type = F;
};

// Floats of shared memory per thread that the mixed RKC integrator keeps its
// power-method vector in (one-thread systems of at most 32 unknowns; larger
// or multi-lane systems keep it in registers).  The row is rounded up to an
// odd length so that a warp's rows fall in distinct banks.
__host__ __device__ constexpr int rkc_mixed_smem_floats(int lanes, int per_lane) {
    return (lanes == 1 && per_lane <= 32) ? (per_lane | 1) : 0;
}
// The same for the two-float RKC integrator: leading words in [0, P),
// trailing words in [P, 2P), the row rounded up to an odd length.
__host__ __device__ constexpr int rkc_f2_smem_floats(int lanes, int per_lane) {
    return (lanes == 1 && per_lane <= 32) ? ((2 * per_lane) | 1) : 0;
}

// Two-float forms (ODE_PREC_F2, ODE_PREC_F2_LEAN).
__host__ __device__ constexpr bool prec_is_f2(int prec) { return prec == 3 || prec == 4; }

// Warm-restart carry words (see batchode.h): valid flag, time reached, h,
// sigma, h_old, err_old, accepted-step count, count at the last
// spectral-radius estimate, rejected flag; then the eigenvector.
enum : int {
    kCarryValid = 0, kCarryT, kCarryH, kCarrySigma, kCarryHold, kCarryErrOld, kCarryNumStep, kCarrySrStep,
    kCarryRejected, kCarryFixed
};

// Bodies of the largest registered n-body system.
constexpr int kMaxBodies = 16;

// Largest kinetics mechanism: species (neq = S + 1 <= 64) and reactions.
constexpr int kKinMaxSpecies = 63;
constexpr int kKinMaxReactions = 1024;

// A kinetics mechanism on the device (owned by the registry).  inc_off /
// inc list, per species, the reactions it takes part in, one entry per
// occurrence, ordered by j and reactants first (the order the oracle
// accumulates omega_i in).  Each entry packs what the rate-of-progress
// product needs, one field per instruction to extract: bits 0-9 the reaction
// j, bit 10 is_product, bits 16-21 its first reactant species, bits 24-29
// the second (kKinOne when it has one reactant: the staged concentrations
// keep 1 there, and the product's extra factor 1 is exact).
// The FP32 section serves the mixed forms: per reaction (log2(10) log10 A,
// beta, Ea log2(e), 0), so that k = 2^(x + beta log2 T - z / T); per species
// (a0, a1, a2, a3) and (R_gas / W, W, 1 / W, 0).
struct KinDevice {
    int S, R;
    double kmin, kmax;
    const double* W;        // [S]
    const double* thermo;   // [S][4]
    const double* log10A;   // [R]
    const double* beta;
    const double* Ea;
    const int* inc_off;     // [S + 1]
    const int* inc;         // [inc_off[S]]
    const float4* rate32;   // [R]
    const float4* thermo32; // [S][2]
    // omega schedule: lane l of a team sums the incidence lists of species
    // sched[k * 32 + l], k < sched_k (-1: none), assigned longest list
    // first to the least-loaded lane, so the lanes' loops are about equal
    const int* sched;       // [sched_k][32]
    int sched_k;
};

// staged-concentration slot that holds 1 (species indices stop at 62)
constexpr int kKinOne = 63;

__host__ __device__ constexpr int kin_inc_word(int j, bool is_product, int r0, int r1) {
    return j | (is_product ? 1 << 10 : 0) | (r0 << 16) | (r1 << 24);
}

// Detection idiom helper (member traits of models and methods).
template <class...>
using void_t_ = void;

// Kernel context of right-hand sides that need none.
struct NoCtx {};

struct BrussConst {
    double A, B, ubc, vbc;
};

// Everything one batched launch needs besides the model.
struct MlpPacked;  // mlp_warp.cuh

struct BatchArgs {
    int64_t nsys;
    int32_t neq;
    int32_t max_attempts;
    const double* y0;
    const double* params;
    double* y_out;
    double t0, tend, rtol, atol;
    int32_t* n_accept;
    int32_t* n_reject;
    int32_t* n_rhs;
    int32_t* n_specrad;
    int32_t* status;
    // persistent mapping: work-queue cursor (zeroed before the launch)
    unsigned long long* cursor;
    // RKC stage coefficients for m = 2..rkc_tab_max (entry (m, j), j = 1..m,
    // at index m (m - 1) / 2 - 1 + j - 1): FP64 {1 - mu - nu, mu, nu, mu~,
    // gamma~, c, lo} and FP32 {mu, nu, mu~, gamma~}, where the FP32 words
    // are the leading words of the two-float coefficients and lo (the FP64
    // entry's last 16 bytes) holds their four trailing words
    const double* rkc_tab64;
    const float4* rkc_tab32;
    int32_t rkc_tab_max;
    // optional proposals (mixed RKC) and training log (plain RKC)
    const float* h0;
    const float* sigma0;
    float* log_xy;
    // optional training log of the spectral-radius estimates (plain RKC):
    // estimate q of a system (q = 0 at the start) with q % log_sr_every == 0
    // goes to record q / log_sr_every if below log_sr_records
    float* log_sr;
    int32_t log_sr_every, log_sr_records;
    // optional proposal network evaluated in-kernel at every spectral-radius
    // point (two-float RKC, one thread per system; mlp_warp.cuh)
    const MlpPacked* mlp;
    // ragged batches: the queue holds nsys entries index[k] (global system
    // numbers); system i's state starts at offset[i] (components contiguous)
    // and has neq_arr[i] unknowns and its own interval and tolerances.
    const int32_t* index;
    const int64_t* offset;
    const int32_t* neq_arr;
    const double* t0_arr;
    const double* tend_arr;
    const double* rtol_arr;
    const double* atol_arr;
    // uniform layout: stride between consecutive components of a system in
    // y0 (ld_in) and y_out (ld_out); 0 means nsys.  A run on the first k
    // systems of a batch (mapping autotuning) keeps the batch's input stride
    // and writes a k-system output.
    int64_t ld_in, ld_out;
    // warm-restart state, in and out (uniform batches; NULL = none): word w
    // of system i at carry[i + nsys w], layout as in batchode.h
    double* carry;
    int32_t carry_mode;  // ODE_CARRY_CONTINUE / ODE_CARRY_RESTART
    int32_t specrad;     // ODE_SPECRAD_POWER / _GERSHGORIN / _POWER_CAPPED (RKC)
    // set by the launcher for the work-queue kernel: methods that keep a
    // warp's spectral-radius points together (two-float RKC) count the
    // schedule per system and let lanes join each other's estimates
    int32_t warp_sched;
    // optional per-system constants of the right-hand side computed before
    // the integration kernel (generated mass-action networks, two-float
    // forms: rate constants as pairs, constant j of system i at
    // pre_consts[j * pre_stride + i]); NULL = computed at each system's set-up
    const void* pre_consts;
    int64_t pre_stride;

    __host__ __device__ int64_t sys_of(int64_t k) const { return index ? (int64_t)index[k] : k; }
    __host__ __device__ int64_t cidx(int64_t i, int w) const { return i + nsys * (int64_t)w; }
    __host__ __device__ int64_t yidx(int64_t i, int c) const {
        return offset ? offset[i] + c : i + (ld_in ? ld_in : nsys) * (int64_t)c;
    }
    __host__ __device__ int64_t yidx_out(int64_t i, int c) const {
        return offset ? offset[i] + c : i + (ld_out ? ld_out : nsys) * (int64_t)c;
    }
    __host__ __device__ int neq_of(int64_t i) const { return neq_arr ? neq_arr[i] : neq; }
    __host__ __device__ double t0_of(int64_t i) const { return t0_arr ? t0_arr[i] : t0; }
    __host__ __device__ double tend_of(int64_t i) const { return tend_arr ? tend_arr[i] : tend; }
    __host__ __device__ double rtol_of(int64_t i) const { return rtol_arr ? rtol_arr[i] : rtol; }
    __host__ __device__ double atol_of(int64_t i) const { return atol_arr ? atol_arr[i] : atol; }
};

__host__ __device__ inline int rkc_tab_index(int m, int j) { return m * (m - 1) / 2 - 1 + (j - 1); }

}  // namespace bode
