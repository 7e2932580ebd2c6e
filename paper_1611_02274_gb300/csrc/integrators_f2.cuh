// integrators_f2.cuh -- RKC (Section 2.2, rkcDriver of Section 3.2 with the
// Appendix power method) with the state, the stages, the evaluation points
// and the right-hand side in two-float arithmetic (f2.cuh).
//
// Why: at rtol 1e-6 the RKC error estimate of Eq. E:rmsE is a difference of
// terms of size h f that cancel down to ~rtol |y|.  With FP32 evaluation
// points and right-hand sides, their rounding (~6e-8 relative) shows up in
// the estimate as noise of several percent; the step-size rule of
// Eqs. dtnp1 / rkc-f turns that noise into a different step sequence, and
// the final state drifts from the FP64 solution by up to ~1e-5 relative.
// Two-float words carry ~48 bits, so the estimate -- and with it the step
// sequence -- follows the FP64 method; the arithmetic stays on the FP32
// pipe, which on this GPU is 64 times faster than the FP64 pipe.
//
// Scalars: step size, spectral radius and error norm in FP32 (their own
// rounding perturbs the step sequence by ~1e-7 relative, far below the
// controller's sensitivity), the remaining interval as an FP32 pair; with
// BK64 the time, step size and spectral radius are FP64 and the error norm
// is accumulated in FP64 (time and step-size bookkeeping in FP64).
// Chebyshev coefficients come from the FP64-built table as two-float pairs.
// The power method runs in two-float arithmetic with the FP64 perturbation
// size sqrt(uround) (the difference quotient keeps ~7 digits).
#pragma once

#include "f2.cuh"
#include "mlp_warp.cuh"

namespace bode {

// sqrt(2.22e-16): the power method's relative perturbation (Appendix)
constexpr float kSqrtUround = 1.4899664e-8f;

// Floats of shared memory per thread a system asks for to hold its
// constants (Sys::CONST_SMEM, 0 if it declares none).
template <class S, class = void>
struct ConstSmem {
    static constexpr int value = 0;
};
template <class S>
struct ConstSmem<S, void_t_<decltype(S::CONST_SMEM)>> {
    static constexpr int value = S::CONST_SMEM;
};

// Systems whose constants may come precomputed (Sys::kPreConsts, load_pre).
template <class S, class = void>
struct PreConsts {
    static constexpr bool value = false;
};
template <class S>
struct PreConsts<S, void_t_<decltype(S::kPreConsts)>> {
    static constexpr bool value = S::kPreConsts;
};

// NET: the variant with the warp-level code of the in-kernel network and of
// the joined spectral-radius estimates (the work queue, ode_opts.mlp); the
// plain variant, for the one-launch mapping without a network, leaves that
// code out of its evaluation loop, whose instructions are fetched every
// iteration.
template <class Model, bool BK64 = false, bool NET = false>
struct RkcF2 {
    static constexpr bool kStepSync = true;  // variable stage count: hold at the step end
    static constexpr int W = Model::W, P = Model::PER;
    // the proposal network at the spectral-radius points (one thread per
    // system, up to 32 components + the parameter)
    using R = F2;
    using TM = Team<W>;
    using HT = typename Pick<BK64, double, float>::type;
    typename Model::template Sys<F2> sys;
    F2 Fn[P], d1[P];  // d_j = w_j - y_n (d_0 = 0); y_n and d_{j-2} below
    static constexpr int V_SMEM = rkc_f2_smem_floats(W, P);
    // the system's constants, one row per thread after the V rows (an even
    // offset: 8-byte aligned pairs, since blocks are a multiple of 32 threads)
    static constexpr int C_SMEM = ConstSmem<typename Model::template Sys<F2>>::value;
    // d_{j-2}, needed only from the third stage on: for one-thread systems a
    // row of pairs in shared memory (an odd number of pairs per row), so a
    // two-stage step -- the common case at tight tolerances -- touches it
    // never and holds no registers for it
    static constexpr int D2_SMEM = (W == 1 && P <= 32) ? 2 * (P | 1) : 0;
    // the state y_n, read at the evaluation points, the error weights and
    // the accept only: for one-thread systems a shared-memory row too, so
    // that no state pair stays live across the right-hand-side evaluation
    static constexpr int Y_SMEM = (W == 1 && P <= 32) ? 2 * (P | 1) : 0;
    static constexpr int SMEM_FLOATS = V_SMEM + C_SMEM + D2_SMEM + Y_SMEM + ModelSmem<Model>::value;
    // the proposal network at the spectral-radius points (one thread per
    // system with rows in shared memory: up to 32 components + the
    // parameter, the BF16 features staged in the d_{j-2} row)
    static constexpr int kMlpKs = (P + 1 + 15) / 16;
    static constexpr bool kWarpPropose = NET && W == 1 && P <= 32 && D2_SMEM >= 8 * kMlpKs && Y_SMEM > 0;
    static constexpr int kJoin = 12;  // steps before its point a system joins a warp's network evaluation
    mutable F2 vreg[V_SMEM ? 1 : P];
    mutable F2 d2reg[D2_SMEM ? 1 : P];
    mutable F2 yreg[Y_SMEM ? 1 : P];
    float* vs;
    F2* d2s;
    F2* ys;
    __device__ void bind_smem(float* base, int stride) {
        vs = base + threadIdx.x * V_SMEM;  // this thread's row
        if constexpr (C_SMEM > 0) sys.bind_consts(base + V_SMEM * stride + threadIdx.x * C_SMEM);
        if constexpr (D2_SMEM > 0)
            d2s = reinterpret_cast<F2*>(base + (V_SMEM + C_SMEM) * stride + threadIdx.x * D2_SMEM);
        if constexpr (Y_SMEM > 0)
            ys = reinterpret_cast<F2*>(base + (V_SMEM + C_SMEM + D2_SMEM) * stride + threadIdx.x * Y_SMEM);
        if constexpr (ModelSmem<Model>::value > 0)
            sys.bind(base + (V_SMEM + C_SMEM + D2_SMEM + Y_SMEM) * stride, stride);
    }
    __device__ F2 Yg(int s) const {
        if constexpr (Y_SMEM > 0)
            return ys[s];
        else
            return yreg[s];
    }
    __device__ void Ys(int s, F2 v) const {
        if constexpr (Y_SMEM > 0)
            ys[s] = v;
        else
            yreg[s] = v;
    }
    __device__ const F2* yp() const {
        if constexpr (Y_SMEM > 0)
            return ys;
        else
            return yreg;
    }
    __device__ F2 D2g(int s) const {
        if constexpr (D2_SMEM > 0)
            return d2s[s];
        else
            return d2reg[s];
    }
    __device__ void D2s(int s, F2 v) const {
        if constexpr (D2_SMEM > 0)
            d2s[s] = v;
        else
            d2reg[s] = v;
    }
    __device__ F2 Vg(int s) const {
        if constexpr (V_SMEM > 0)
            return F2(vs[s], vs[P + s]);
        else
            return vreg[s];
    }
    __device__ void Vs(int s, F2 v) const {
        if constexpr (V_SMEM > 0) {
            vs[s] = v.hi;
            vs[P + s] = v.lo;
        } else {
            vreg[s] = v;
        }
    }
    double t, tend;                   // BK64
    float remf, reml, tendf;          // FP32 scalars: remaining interval as a pair
    HT hmax, hmin, h, h_old, sigma;
    F2 hh;                            // the step size as a pair (exact for an FP32 h)
    float rtolf, atolf, c3_old, dynrm, sig;
    float4 chi, clo;                  // (mu_j, nu_j, mu~_j, gamma~_j), leading / trailing words
    CoefSource cs;
    int32_t n_acc, n_rej, n_rhs, n_sr, status, max_att, mmax, num_step, sr_step, n;
    int32_t phase, m, j, sr_iter;
    bool have_sigma, rejected, warm;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        if constexpr (PreConsts<typename Model::template Sys<F2>>::value) {
            if (a.pre_consts != nullptr)
                sys.load_pre(static_cast<const F2*>(a.pre_consts), i, a.pre_stride, a.neq_of(i));
            else
                sys.load(ctx, tm, a.params[i], a.neq_of(i));
        } else {
            sys.load(ctx, tm, a.params[i], a.neq_of(i));
        }
        n = a.neq_of(i);
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            Ys(s, F2(c >= 0 ? a.y0[a.yidx(i, c)] : 0.0));
        }
        t = a.t0_of(i);
        tend = a.tend_of(i);
        remf = (float)(tend - t);
        reml = (float)((tend - t) - (double)remf);
        tendf = (float)tend;
        rtolf = (float)a.rtol_of(i);
        atolf = (float)a.atol_of(i);
        mmax = (int)round(sqrt(a.rtol_of(i) / (10.0 * kUround)));
        if (mmax < 2) mmax = 2;
        hmax = (HT)fabs(tend - t);
        hmin = (HT)(10.0 * kUround * fmax(fabs(t), fabs(tend - t)));
        n_acc = n_rej = n_sr = status = 0;
        n_rhs = 1;
        max_att = a.max_attempts;
        h = h_old = sigma = (HT)0;
        c3_old = 0.0f;
        num_step = 0;
        sr_step = -1;
        have_sigma = rejected = false;
        warm = carry_warm(a, i);
        if (warm) {  // resume the controller and the spectral-radius schedule
            h = (HT)a.carry[a.cidx(i, kCarryH)];
            sigma = (HT)a.carry[a.cidx(i, kCarrySigma)];
            h_old = (HT)a.carry[a.cidx(i, kCarryHold)];
            c3_old = fpow((float)a.carry[a.cidx(i, kCarryErrOld)], 1.0f / 3.0f);
            num_step = (int)a.carry[a.cidx(i, kCarryNumStep)];
            sr_step = (int)a.carry[a.cidx(i, kCarrySrStep)];
            rejected = (int)a.carry[a.cidx(i, kCarryRejected)] != 0;
            have_sigma = true;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                const int c = sys.comp(tm, s);
                Vs(s, F2(c >= 0 ? a.carry[a.cidx(i, kCarryFixed + c)] : 0.0));
            }
            if (a.carry_mode == ODE_CARRY_RESTART) {
                num_step = 0;
                sr_step = -1;
                rejected = false;
            }
        } else if (a.h0 != nullptr) {
            // a proposed spectral radius replaces the initial power method; a
            // proposed step size beside it replaces the Euler trial as well
            // (without one the trial sets h); the first rejection returns the
            // system to the power method
            const float hp = a.h0[i], sp = a.sigma0[i];
            if (isfinite(sp) && sp > 0.0f) {
                if (isfinite(hp) && hp > 0.0f) {
                    h = (HT)hp < hmax ? (HT)hp : hmax;
                    h = h > hmin ? h : hmin;
                }
                sigma = (HT)sp;
                have_sigma = true;
                sr_step = 0;
                status |= ODE_ST_PROPOSED;
            }
        }
        phase = PH_F0;
    }
    __device__ bool done() const { return phase == PH_DONE; }
    __device__ bool in_stages() const { return phase == PH_STAGE; }
    __device__ bool at_step_end() const { return phase == PH_FINAL; }

    // sum of squares of the leading words (norms that only scale a vector)
    template <class X>
    __device__ float sumsq_hi(const TM& tm, X x_of) const {
        float acc = 0.0f;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s)
            if (sys.comp(tm, s) >= 0) {
                const float v = x_of(s);
                acc = fmaf(v, v, acc);
            }
        return tm.sum(acc);
    }

    __device__ void point(F2* x, F2& tx) const {
        if constexpr (BK64)
            tx = F2(t);
        else
            tx = F2(tendf - remf);
        switch (phase) {
        case PH_F0:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = Yg(s);
            break;
        case PH_SR:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = Vg(s);
            break;
        case PH_TRIAL:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = Yg(s) + hh * Fn[s];
            break;
        default:  // stages and F_{n+1}: w = y_n + d (left unnormalised: it feeds products)
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = add_lazy(Yg(s), d1[s]);
        }
    }

    __device__ bool consume(const BatchArgs& a, const TM& tm, const F2* x, const F2* f) {
        switch (phase) {
        case PH_F0:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                Fn[s] = f[s];
                if (!warm) Vs(s, f[s]);  // first eigenvector guess
            }
            loop_top(a, tm);
            break;
        case PH_SR: sr_consume(a, tm, f); break;
        case PH_TRIAL: trial_consume(a, tm, f); break;
        case PH_STAGE: stage_consume(f); break;
        default: final_consume(a, tm, x, f);
        }
        return done();
    }

    __device__ void loop_top(const BatchArgs& a, const TM& tm) {
        if constexpr (BK64) {
            if (!(t < tend)) {
                phase = PH_DONE;
                return;
            }
        } else {
            if (!(remf > 0.0f)) {
                phase = PH_DONE;
                return;
            }
        }
        if (n_acc + n_rej >= max_att) {
            status |= ODE_ST_MAX_ATTEMPTS;
            phase = PH_DONE;
            return;
        }
        if constexpr (BK64) {
            if (1.1 * h >= fabs(tend - t)) h = fabs(tend - t);
        } else {
            if (1.1f * h >= remf) h = remf;
        }
        if constexpr (kWarpPropose) {
            // with the network, or in the work queue, the schedule counts
            // from each system's last estimate, and a system within kJoin
            // steps of its point takes its estimate (the network's bound, or
            // the power method) when another lane of its warp does
            // (propose_warp): the warp's points then coincide, even where
            // the systems started at different times (work queue), so the
            // lanes stay in one phase of the step
            if ((a.mlp != nullptr || a.warp_sched) && a.specrad == ODE_SPECRAD_POWER) {
                if (!have_sigma || rejected || num_step - sr_step >= kSpecradEvery) {
                    if (!rejected) {  // never after a rejection: the power method
                        phase = PH_PROPOSE;
                        return;
                    }
                    sr_begin(tm);
                    return;
                }
                after_sr(a);
                return;
            }
        }
        if (!have_sigma || rejected || (num_step % kSpecradEvery == 0 && sr_step != num_step)) {
            if (a.specrad == ODE_SPECRAD_GERSHGORIN) {  // the bound replaces the power method
                sigma = (HT)to_double(sys.gershgorin(tm, yp()));
                have_sigma = true;
                sr_step = num_step;
                after_sr(a);
                return;
            }
            sr_begin(tm);
            return;
        }
        after_sr(a);
    }

    // Learned spectral-radius bound for the lanes at a spectral-radius point
    // (phase PH_PROPOSE), one warp-wide evaluation of the network on their
    // current states: features log max(|y_k|, 1e-30) and the parameter,
    // normalised.  The bound is taken when it is finite, positive, inside
    // the training box and at least half the system's previous bound;
    // otherwise the power method runs as without a network.  Lanes at the
    // start of a step within kJoin steps of their own point join the
    // evaluation (their step is set up again with the new bound; a joiner
    // whose bound fails the checks keeps its old one).  Every lane of the
    // warp calls (warp votes and mma.sync).
    __device__ void propose_warp(const BatchArgs& a, const TM& tm, bool live, int64_t i) {
        if constexpr (kWarpPropose) {
            const MlpPacked* __restrict__ net = a.mlp;
            if (net == nullptr && !a.warp_sched) return;
            const bool want = live && phase == PH_PROPOSE;
            if (!__any_sync(0xffffffffu, want)) return;
            const bool join = live && phase == PH_STAGE && j == 2 && have_sigma && !rejected &&
                              num_step - sr_step >= kSpecradEvery - kJoin && num_step != sr_step;
            if (net == nullptr) {  // the power method, started together
                if (want || join) sr_begin(tm);
                return;
            }
            const bool mine = want || join;
            const unsigned take = __ballot_sync(0xffffffffu, mine);
            // features into this lane's d_{j-2} row (unused at a step's
            // start) as BF16, zero up to 16 KS; a rolled loop (cold code)
            bool inside = true;
            if (mine) {
                uint16_t* fr = reinterpret_cast<uint16_t*>(d2s);
                const float par = (float)a.params[i];
#pragma unroll 1
                for (int k = 0; k < 16 * kMlpKs; ++k) {
                    float fx = 0.0f;
                    if (k <= n) {
                        const float raw = k < n ? __logf(fmaxf(fabsf(ys[k].hi), 1e-30f)) : par;
                        fx = (raw - net->x_mean[k]) * net->x_iscale[k];
                        inside = inside && raw >= net->x_lo[k] && raw <= net->x_hi[k];
                    }
                    fr[k] = to_bf16(fx);
                }
            }
            __syncwarp();
            float o0 = 0.0f, o1 = 0.0f;
            mlp_warp_eval<kMlpKs>(net, take, reinterpret_cast<const uint32_t*>(d2s), D2_SMEM, o0, o1);
            __syncwarp();  // every row read before a lane writes its row again
            if (!mine) return;
            const float sh = __expf(o1 * net->y_scale[1] + net->y_mean[1]);
            const bool ok = inside && isfinite(sh) && sh > 0.0f && !(have_sigma && sh < 0.5f * (float)sigma);
            if (!ok) {
                if (want) sr_begin(tm);
                return;
            }
            sigma = (HT)sh;
            have_sigma = true;
            sr_step = num_step;
            status |= ODE_ST_PROPOSED;
            if (want) {
                after_sr(a);
            } else {  // a joiner: the step's stage count and set-up again (from
                      // its step size as it stands: a cap the old bound set stays)
                stage_begin(a);
            }
        }
    }

    // power method (Appendix) with the FP64 perturbation size
    __device__ void sr_begin(const TM& tm) {
        const float nrm1 = sqrtf(sumsq_hi(tm, [&](int s) { return Yg(s).hi; }));
        const float nrm2 = sqrtf(sumsq_hi(tm, [&](int s) { return Vg(s).hi; }));
        if (nrm1 != 0.0f && nrm2 != 0.0f) {
            dynrm = nrm1 * kSqrtUround;
            const float sc = dynrm / nrm2;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, Yg(s) + Vg(s) * sc);
        } else if (nrm1 != 0.0f) {
            dynrm = nrm1 * kSqrtUround;
            const F2 sc(1.0 + (double)kSqrtUround);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, Yg(s) * sc);
        } else if (nrm2 != 0.0f) {
            dynrm = (float)kUround;
            const float sc = dynrm / nrm2;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, Vg(s) * sc);
        } else {
            dynrm = (float)kUround;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, F2(dynrm));
        }
        sig = 0.0f;
        sr_iter = 0;
        phase = PH_SR;
    }

    __device__ void sr_consume(const BatchArgs& a, const TM& tm, const F2* Fv) {
        sr_iter += 1;
        n_sr += 1;
        F2 df[P];
        float acc = 0.0f;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            df[s] = Fv[s] - Fn[s];
            if (sys.comp(tm, s) >= 0) acc = fmaf(df[s].hi, df[s].hi, acc);
        }
        const float d = sqrtf(tm.sum(acc));
        const float sig_prev = sig;
        sig = d / dynrm;
        if (sr_iter >= 2 && fabsf(sig - sig_prev) <= fmaxf(sig, 1.0f / (float)hmax) * 0.01f) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, Vg(s) - Yg(s));
            sr_end(a, tm);
            return;
        }
        if (d != 0.0f) {
            const float sc = dynrm / d;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, Yg(s) + df[s] * sc);
        } else {
            const int ind = sr_iter % n;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (opaque(sys.comp(tm, s)) == ind) Vs(s, Yg(s) - (Vg(s) - Yg(s)));
        }
        if (sr_iter == kSpecradItmax) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) Vs(s, Vg(s) - Yg(s));
            status |= ODE_ST_SPECRAD_NOCONV;
            sr_end(a, tm);
        }
    }

    __device__ void sr_end(const BatchArgs& a, const TM& tm) {
        sigma = (HT)1.2 * (HT)sig;
        if (a.specrad == ODE_SPECRAD_POWER_CAPPED) {
            const HT g = (HT)to_double(sys.gershgorin(tm, yp()));
            sigma = sigma < g ? sigma : g;
        }
        have_sigma = true;
        sr_step = num_step;
        after_sr(a);
    }

    __device__ void after_sr(const BatchArgs& a) {
        if (h < (HT)kUround) {
            h = hmax;
            if (sigma * h > (HT)1) h = (HT)1 / sigma;
            h = h > hmin ? h : hmin;
            hh = F2(h);
            phase = PH_TRIAL;
            return;
        }
        stage_begin(a);
    }

    // weighted sum of squares, FP64 (BK64) or FP32
    template <class E>
    __device__ HT weighted_ssq(const TM& tm, E e_of) const {
        HT acc = (HT)0;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s)
            if (sys.comp(tm, s) >= 0) {
                const float e = e_of(s);
                if constexpr (BK64)
                    acc = fma((double)e, (double)e, acc);
                else
                    acc = fmaf(e, e, acc);
            }
        return tm.sum(acc);
    }

    __device__ void trial_consume(const BatchArgs& a, const TM& tm, const F2* f) {
        n_rhs += 1;
        const HT ssq = weighted_ssq(tm, [&](int s) {
            return __fdividef(to_float(f[s] - Fn[s]), atolf + rtolf * fabsf(Yg(s).hi));
        });
        const HT est = h * sqrt(ssq / (HT)n);
        if ((HT)kP1 * h < hmax * sqrt(est)) {
            h = (HT)kP1 * h / sqrt(est);
            h = h > hmin ? h : hmin;
        } else {
            h = hmax;
        }
        stage_begin(a);
    }

    __device__ void stage_begin(const BatchArgs& a) {
        m = 1 + (int)sqrt((HT)1.54 * h * sigma + (HT)1);
        if (m > mmax) {
            m = mmax;
            h = (HT)(m * m - 1) / ((HT)1.54 * sigma);
        }
        hh = F2(h);
        cs.start(m, a);
        const F2 mut1h = cs.mut1f2() * hh;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) d1[s] = mul_lazy(mut1h, Fn[s]);  // a product: its pair stays near-normal
        j = 2;
        cs.stagef2(2, chi, clo);
        phase = PH_STAGE;
    }

    // d_j = mu_j d_{j-1} + nu_j d_{j-2} + mu~_j h f_{j-1} + gamma~_j h F_n
    // (at j = 2, d_0 = 0 and the nu term is an exact zero: skipped).  The
    // products and the three- or four-term sum are lazy and d_j stays
    // unnormalised: every use of it (the next evaluation point, the next
    // stage's products, the error estimate's separate words, the accepted
    // state's full sum) takes an unnormalised pair.  At j = 2, d_1 = mu~_1 h F_n,
    // so d_2 = (mu_2 mu~_1 + gamma~_2) h F_n + mu~_2 h f_1: the scalar
    // coefficient once per step, two products and one sum per component
    // (the two-stage step is the one every system takes at tight
    // tolerances).
    __device__ void stage_consume(const F2* f) {
        const F2 mu(chi.x, clo.x), nu(chi.y, clo.y);
        const F2 muth = F2(chi.z, clo.z) * hh;
        const bool keep = j < m;  // d_{j-1} is the next stage's d_{j-2}
        if (j == 2) {
            const F2 c2h = (mu * cs.mut1f2() + F2(chi.w, clo.w)) * hh;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                const F2 dj = add_lazy(mul_lazy(c2h, Fn[s]), mul_lazy(muth, f[s]));
                if (keep) D2s(s, d1[s]);
                d1[s] = dj;
            }
        } else {
            const F2 gth = F2(chi.w, clo.w) * hh;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                const F2 dj = add_lazy(
                    add_lazy(add_lazy(mul_lazy(mu, d1[s]), mul_lazy(nu, D2g(s))), mul_lazy(muth, f[s])),
                    mul_lazy(gth, Fn[s]));
                if (keep) D2s(s, d1[s]);
                d1[s] = dj;
            }
        }
        j += 1;
        if (j <= m)
            cs.stagef2(j, chi, clo);
        else
            phase = PH_FINAL;
    }

    // x = w_m (the point F_{n+1} was evaluated at), f = F_{n+1}.
    // Eq. E:rmsE's 0.8 (y_n - y_{n+1}) + 0.4 h (F_n + F_{n+1}) is computed as
    // 0.4 (h (F_n + F_{n+1}) - 2 d_m): the two terms cancel, so the leading
    // product h a is formed exactly (two_prod) and the difference taken
    // before the single rounding to FP32.
    __device__ void final_consume(const BatchArgs& a, const TM& tm, const F2* x, const F2* f) {
        n_rhs += m;
        const HT ms = weighted_ssq(tm, [&](int s) {
            const F2 sum = add_lazy(Fn[s], f[s]);  // feeds the product below: left unnormalised
            const float p = hh.hi * sum.hi;
            float e = fmaf(hh.hi, sum.hi, -p);
            e = fmaf(hh.hi, sum.lo, e);
            e = fmaf(hh.lo, sum.hi, e);
            const float D = fmaf(-2.0f, d1[s].hi, p) + fmaf(-2.0f, d1[s].lo, e);
            return __fdividef(0.4f * D, atolf + rtolf * fmaxf(fabsf(x[s].hi), fabsf(Yg(s).hi)));
        }) / (HT)n;  // err^2
        if (isnan(ms)) {
            n_rej += 1;
            status |= ODE_ST_NONFINITE;
            phase = PH_DONE;
            return;
        }
        const float err = sqrtf((float)ms);
        const float c3 = fpow(err, 1.0f / 3.0f);
        if (ms > (HT)1) {
            n_rej += 1;
            h = h * (HT)(0.8f / c3);
            rejected = true;
            if (h < hmin) {
                status |= ODE_ST_H_UNDERFLOW;
                phase = PH_DONE;
                return;
            }
            loop_top(a, tm);
            return;
        }
        n_acc += 1;
        rejected = false;
        num_step += 1;
        float fac = 10.0f;
        if (h_old < (HT)kUround) {
            if (0.8f < fac * c3) fac = 0.8f / c3;
        } else {
            const float temp1 = 0.8f * (float)h * c3_old;
            const float temp2 = (float)h_old * (c3 * c3);
            if (temp1 < fac * temp2) fac = temp1 / temp2;
        }
        c3_old = c3;
        h_old = h;
        if constexpr (BK64) {
            t = t + h;
        } else if (h >= remf * 0.999999f) {
            remf = reml = 0.0f;  // the step covered what was left
        } else {
            df_sub(remf, reml, h);
        }
        float chk = 0.0f;  // one finiteness test of a sum per system
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const F2 yn = Yg(s) + d1[s];
            Ys(s, yn);
            Fn[s] = f[s];
            chk += (sys.comp(tm, s) >= 0) ? yn.hi - yn.hi : 0.0f;
        }
        const bool bad = !(chk == 0.0f);
        h = h * (HT)fmaxf((float)kP1, fac);
        h = h < hmax ? h : hmax;
        h = h > hmin ? h : hmin;
        if (tm.any(bad)) {
            status |= ODE_ST_NONFINITE;
            phase = PH_DONE;
            return;
        }
        loop_top(a, tm);
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            if (c >= 0) a.y_out[a.yidx_out(i, c)] = to_double(Yg(s));
            if (a.carry != nullptr && c >= 0) a.carry[a.cidx(i, kCarryFixed + c)] = to_double(Vg(s));
        }
        if (a.carry != nullptr && tm.lane == 0) {
            const int st = status & 0xFF;
            const double t_end = BK64 ? t : tend - ((double)remf + (double)reml);
            carry_scalars(a, i, (st == ODE_ST_OK || st == ODE_ST_MAX_ATTEMPTS) && have_sigma, t_end, (double)h,
                          (double)sigma, (double)h_old, (double)c3_old * (double)c3_old * (double)c3_old, num_step,
                          sr_step, rejected);
        }
        if (tm.lane == 0) {
            if (a.n_accept) a.n_accept[i] = n_acc;
            if (a.n_reject) a.n_reject[i] = n_rej;
            if (a.n_rhs) a.n_rhs[i] = n_rhs + n_sr;
            if (a.n_specrad) a.n_specrad[i] = n_sr;
            if (a.status) a.status[i] = status;
        }
    }
};

// ============================================================ RKCK two-float
//
// RKCK (Section 2.1, rkckDriver of Section 3.2) with the state, the six stage
// increments k_i = h f_i, the evaluation points and the right-hand side in
// two-float arithmetic.  Why: the embedded error estimate sum_i (c_i - c*_i)
// k_i is a difference of fifth- and fourth-order solutions that cancels
// down to ~rtol |y|; for oscillators on a limit cycle, FP32 rounding of the
// stages moves the phase along the cycle, and the final states of the FP32
// forms drift from the FP64 method's by up to ~1e-2 relative over t in
// [0, 20].  The tableau's rationals (Table 1) enter as two-float pairs, so
// the step sequence follows the FP64 method's.
//
// Scalars: the step size and the error ratio in FP32 (the error is a
// max-norm of FP32-rounded components; the step-size factor by fpow), the
// remaining interval as an FP32 pair; with BK64 the time and the step size
// are FP64, as in RkckMixed's specified split.  All six stages run for
// every system in the same order, so the lanes of a warp stay at the same
// stage and the per-stage switches do not diverge.

// a double as the nearest two-float pair, at compile time
__host__ __device__ constexpr F2 f2c(double d) { return F2((float)d, (float)(d - (double)(float)d)); }

namespace ck2 {
constexpr F2 B21 = f2c(ck::B21);
constexpr F2 B31 = f2c(ck::B31), B32 = f2c(ck::B32);
constexpr F2 B41 = f2c(ck::B41), B42 = f2c(ck::B42), B43 = f2c(ck::B43);
constexpr F2 B51 = f2c(ck::B51), B52 = f2c(ck::B52), B53 = f2c(ck::B53), B54 = f2c(ck::B54);
constexpr F2 B61 = f2c(ck::B61), B62 = f2c(ck::B62), B63 = f2c(ck::B63), B64 = f2c(ck::B64), B65 = f2c(ck::B65);
constexpr F2 C1 = f2c(ck::C1), C3 = f2c(ck::C3), C4 = f2c(ck::C4), C6 = f2c(ck::C6);
constexpr F2 DC1 = f2c(ck::DC1), DC3 = f2c(ck::DC3), DC4 = f2c(ck::DC4), DC5 = f2c(ck::DC5), DC6 = f2c(ck::DC6);
}  // namespace ck2

template <class Model, bool BK64 = false>
struct RkckF2 {
    static constexpr bool kStepSync = false;  // fixed six stages: lanes stay aligned
    static constexpr int SMEM_FLOATS = ModelSmem<Model>::value;
    __device__ void bind_smem(float* base, int stride) {
        if constexpr (SMEM_FLOATS > 0) sys.bind(base, stride);
    }
    static constexpr int W = Model::W, P = Model::PER;
    using R = F2;
    using TM = Team<W>;
    using HT = typename Pick<BK64, double, float>::type;
    typename Model::template Sys<F2> sys;
    F2 y[P], k1[P], k2[P], k3[P], k4[P], k5[P];
    double t, tend;                          // BK64
    HT h, hmax;
    F2 hh;                                   // the step size as a pair
    float remf, reml, tendf, tabsf, deltaf, inv_rtolf;  // FP32 scalars: remaining interval remf + reml
    int32_t n_acc, n_rej, status, max_att, stage;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq_of(i));
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            y[s] = F2(c >= 0 ? a.y0[a.yidx(i, c)] : 0.0);
        }
        t = a.t0_of(i);
        tend = a.tend_of(i);
        hmax = (HT)fabs(tend - t);
        h = (HT)(0.5 * fabs(tend - t));
        if (carry_warm(a, i) && a.carry[a.cidx(i, kCarryH)] > 0.0) h = (HT)a.carry[a.cidx(i, kCarryH)];
        remf = (float)(tend - t);
        reml = (float)((tend - t) - (double)remf);
        tendf = (float)tend;
        tabsf = fabsf((float)t);
        // FP32 divisions: in the work queue each lane sets up its own
        // systems, so FP64 set-up code runs once per system, not per warp
        const float rtolf = (float)a.rtol_of(i);
        deltaf = a.atol_of(i) > 0.0 ? (float)a.atol_of(i) / rtolf : (float)kTiny;
        inv_rtolf = 1.0f / rtolf;
        n_acc = n_rej = status = 0;
        max_att = a.max_attempts;
        loop_top();
    }
    __device__ bool done() const { return stage == 0; }

    // top of the rkckDriver loop: finished?  attempt cap, then clamp h
    __device__ void loop_top() {
        stage = 0;
        if constexpr (BK64) {
            if (!(t < tend)) return;
        } else {
            if (!(remf > 0.0f)) return;
        }
        if (n_acc + n_rej >= max_att) {
            status = ODE_ST_MAX_ATTEMPTS;
            return;
        }
        if constexpr (BK64)
            h = fmin(tend - t, h);
        else
            h = fminf(remf, h);
        hh = F2(h);
        stage = 1;
    }

    // y + sum_j b_ij k_j, the point of stage i (products and sums lazy, the
    // point left unnormalised: it feeds the right-hand side's products)
    __device__ void point(F2* x, F2& tx) const {
        float tb;
        if constexpr (BK64)
            tb = (float)t;
        else
            tb = tendf - remf;
        const float hf = (float)h;
        switch (stage) {
        case 1:
            tx = F2(tb);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = y[s];
            break;
        case 2:
            tx = F2(tb + (float)ck::A2 * hf);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = add_lazy(y[s], mul_lazy(ck2::B21, k1[s]));
            break;
        case 3:
            tx = F2(tb + (float)ck::A3 * hf);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                x[s] = add_lazy(y[s], add_lazy(mul_lazy(ck2::B31, k1[s]), mul_lazy(ck2::B32, k2[s])));
            break;
        case 4:
            tx = F2(tb + (float)ck::A4 * hf);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                x[s] = add_lazy(y[s], add_lazy(add_lazy(mul_lazy(ck2::B41, k1[s]), mul_lazy(ck2::B42, k2[s])),
                                               mul_lazy(ck2::B43, k3[s])));
            break;
        case 5:
            tx = F2(tb + (float)ck::A5 * hf);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                x[s] = add_lazy(y[s], add_lazy(add_lazy(mul_lazy(ck2::B51, k1[s]), mul_lazy(ck2::B52, k2[s])),
                                               add_lazy(mul_lazy(ck2::B53, k3[s]), mul_lazy(ck2::B54, k4[s]))));
            break;
        default:
            tx = F2(tb + (float)ck::A6 * hf);
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                x[s] = add_lazy(y[s], add_lazy(add_lazy(add_lazy(mul_lazy(ck2::B61, k1[s]), mul_lazy(ck2::B62, k2[s])),
                                                        add_lazy(mul_lazy(ck2::B63, k3[s]), mul_lazy(ck2::B64, k4[s]))),
                                               mul_lazy(ck2::B65, k5[s])));
        }
    }

    __device__ bool consume(const BatchArgs&, const TM& tm, const F2*, const F2* f) {
        switch (stage) {
        case 1:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k1[s] = f[s] * hh;
            break;
        case 2:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k2[s] = f[s] * hh;
            break;
        case 3:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k3[s] = f[s] * hh;
            break;
        case 4:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k4[s] = f[s] * hh;
            break;
        case 5:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k5[s] = f[s] * hh;
            break;
        default:
            finish(tm, f);
            return done();
        }
        stage += 1;
        return false;
    }

    // fifth-order solution, embedded error (Section 2.1) and the step-size
    // rule of the listing
    __device__ void finish(const TM& tm, const F2* f) {
        F2 yt[P];
        float err = 0.0f;
        bool nan_flag = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const F2 k6 = f[s] * hh;
            const F2 incr = add_lazy(add_lazy(mul_lazy(ck2::C1, k1[s]), mul_lazy(ck2::C3, k3[s])),
                                     add_lazy(mul_lazy(ck2::C4, k4[s]), mul_lazy(ck2::C6, k6)));
            yt[s] = y[s] + incr;
            const float ye = to_float(add_lazy(add_lazy(add_lazy(mul_lazy(ck2::DC1, k1[s]), mul_lazy(ck2::DC3, k3[s])),
                                                        add_lazy(mul_lazy(ck2::DC4, k4[s]), mul_lazy(ck2::DC5, k5[s]))),
                                               mul_lazy(ck2::DC6, k6)));
            if (sys.comp(tm, s) >= 0) {
                if (isnan(ye) || isnan(yt[s].hi)) nan_flag = true;
                err = fmaxf(err, __fdividef(fabsf(ye), fabsf(y[s].hi) + fabsf(k1[s].hi) + deltaf));
            }
        }
        err = tm.max(err) * inv_rtolf;
        nan_flag = tm.any(nan_flag);
        if (err > 1.0f || isnan(err) || nan_flag) {
            n_rej += 1;
            if (isnan(err) || nan_flag)
                h = h * (HT)kP1;
            else
                h = h * (HT)fmaxf((float)kSafety * fpow(err, (float)kPshrnk), (float)kP1);
            bool underflow;
            if constexpr (BK64)
                underflow = h < 1.0e-20 || t + h == t;
            else
                underflow = h < 1.0e-20f || h <= tabsf * 2.2e-16f;
            if (underflow) {
                status = ODE_ST_H_UNDERFLOW;
                stage = 0;
                return;
            }
            loop_top();
            return;
        }
        n_acc += 1;
        if constexpr (BK64) {
            t = t + h;
        } else if (h >= remf * 0.999999f) {
            remf = reml = 0.0f;  // the step covered what was left
        } else {
            df_sub(remf, reml, h);
            tabsf = fabsf(tendf - remf);
        }
        const float fac = (err > (float)kErrcon) ? (float)kSafety * fpow(err, (float)kPgrow) : 5.0f;
        if constexpr (BK64)
            h = fmax(1.0e-20, fmin(hmax, h * (double)fac));
        else
            h = fmaxf(1.0e-20f, fminf(hmax, h * fac));
        bool bad = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            y[s] = yt[s];
            if (sys.comp(tm, s) >= 0 && !isfinite(yt[s].hi)) bad = true;
        }
        if (tm.any(bad)) {
            status = ODE_ST_NONFINITE;
            stage = 0;
            return;
        }
        loop_top();
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            if (c >= 0) a.y_out[a.yidx_out(i, c)] = to_double(y[s]);
            if (a.carry != nullptr && c >= 0) a.carry[a.cidx(i, kCarryFixed + c)] = 0.0;
        }
        if (a.carry != nullptr && tm.lane == 0) {
            const double t_end = BK64 ? t : tend - ((double)remf + (double)reml);
            carry_scalars(a, i, status == ODE_ST_OK || status == ODE_ST_MAX_ATTEMPTS, t_end, (double)h, 0.0, 0.0,
                          0.0, 0, 0, false);
        }
        if (tm.lane == 0) {
            if (a.n_accept) a.n_accept[i] = n_acc;
            if (a.n_reject) a.n_reject[i] = n_rej;
            if (a.n_rhs) a.n_rhs[i] = 6 * (n_acc + n_rej);
            if (a.n_specrad) a.n_specrad[i] = 0;
            if (a.status) a.status[i] = status;
        }
    }
};

}  // namespace bode
