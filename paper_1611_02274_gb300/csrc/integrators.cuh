// integrators.cuh -- per-system RKCK and RKC integrators as phase machines.
//
// One object integrates one system on one team of lanes (team.cuh).  The
// algorithms are the rkckDriver / rkcDriver listings of Section 3 (RKC with
// the Appendix power method), reorganised around the right-hand side: the
// driving kernel repeatedly asks point() where f must be evaluated next,
// evaluates f there at ONE call site, and hands the result to consume(),
// which performs everything up to the next evaluation and returns true when
// the system is finished.  Lanes whose systems are in different phases
// (power iteration, trial step, stage j, error estimate) therefore still
// execute the right-hand side -- the dominant cost -- together, the code
// holds one copy of it, and a persistent kernel can refill a team between
// any two evaluations.
//
// Two arithmetic forms:
//   *F64    the plain form: every operation in FP64 in the order of the
//           listings (these translation units are compiled without
//           multiply-add contraction, norms are summed in component order),
//           so results reproduce a sequential FP64 implementation bit for bit;
//   *Mixed  FP32 right-hand sides and stage arithmetic on an FP32 state with
//           a Kahan compensation term and the RKC Chebyshev coefficients
//           computed in FP64; with SPEC also time, step size, spectral radius
//           and the RKC error-norm accumulation in FP64, without it only the
//           time t (the lean split: FP64 only where rounding accumulates).
#pragma once
#include <cmath>

#include "common.cuh"
#include "rkc_coef.cuh"
#include "team.cuh"
#include "xmath.cuh"

namespace bode {

// Floats of shared memory per thread a model asks for (Model::SMEM_FLOATS,
// 0 if it declares none); the integrators add them to their own and hand
// the model its part through Sys::bind.
template <class M, class = void>
struct ModelSmem {
    static constexpr int value = 0;
};
template <class M>
struct ModelSmem<M, void_t_<decltype(M::SMEM_FLOATS)>> {
    static constexpr int value = M::SMEM_FLOATS;
};

// PH_PROPOSE: waiting for the warp's evaluation of the proposal network
// (two-float RKC with an in-kernel network, mlp_warp.cuh)
enum : int { PH_DONE = 0, PH_F0, PH_SR, PH_TRIAL, PH_STAGE, PH_FINAL, PH_PROPOSE };

// Kahan-compensated state update (hi, lo) += d.
__device__ __forceinline__ void kahan_add(float& hi, float& lo, float d) {
    const float y = d + lo;
    const float t = hi + y;
    lo = y - (t - hi);
    hi = t;
}

// Double-float subtraction (hi, lo) -= b: Knuth's two-sum of hi and -b gives
// the rounded difference and its exact error, which joins lo before a
// renormalisation.  Keeps a time interval to ~48 significant bits with FP32
// instructions only.
__device__ __forceinline__ void df_sub(float& hi, float& lo, float b) {
    const float s = hi - b;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) - (b + bb);
    const float l = lo + e;
    hi = s + l;
    lo = l - (hi - s);
}

// Warm-restart carry (the outer global-step loop of Section 3; layout in
// batchode.h).  carry_warm: a valid carry for system i.  carry_store: the
// scalars from team lane 0, v from every lane (slots past the system's
// size hold no component and are skipped); RKCK stores only its step size.
__device__ __forceinline__ bool carry_warm(const BatchArgs& a, int64_t i) {
    return a.carry != nullptr && a.carry[a.cidx(i, kCarryValid)] == 1.0;
}
__device__ __forceinline__ void carry_scalars(const BatchArgs& a, int64_t i, bool valid, double t, double h,
                                              double sigma, double h_old, double err_old, int num_step,
                                              int sr_step, bool rejected) {
    double* c = a.carry;
    c[a.cidx(i, kCarryValid)] = valid ? 1.0 : 0.0;
    c[a.cidx(i, kCarryT)] = t;
    c[a.cidx(i, kCarryH)] = h;
    c[a.cidx(i, kCarrySigma)] = sigma;
    c[a.cidx(i, kCarryHold)] = h_old;
    c[a.cidx(i, kCarryErrOld)] = err_old;
    c[a.cidx(i, kCarryNumStep)] = (double)num_step;
    c[a.cidx(i, kCarrySrStep)] = (double)sr_step;
    c[a.cidx(i, kCarryRejected)] = rejected ? 1.0 : 0.0;
}

// ================================================================ RKCK F64

template <class Model>
struct RkckF64 {
    static constexpr bool kStepSync = false;  // fixed six stages: lanes stay aligned
    static constexpr int SMEM_FLOATS = ModelSmem<Model>::value;
    __device__ void bind_smem(float* base, int stride) {
        if constexpr (SMEM_FLOATS > 0) sys.bind(base, stride);
    }
    static constexpr int W = Model::W, P = Model::PER;
    using R = double;
    using TM = Team<W>;
    typename Model::template Sys<double> sys;
    double y[P], k1[P], k2[P], k3[P], k4[P], k5[P];
    double t, tend, h, hmax, delta, rtol;
    int32_t n_acc, n_rej, status, max_att, stage;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq_of(i));
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            y[s] = c >= 0 ? a.y0[a.yidx(i, c)] : 0.0;
        }
        t = a.t0_of(i);
        tend = a.tend_of(i);
        rtol = a.rtol_of(i);
        hmax = fabs(tend - t);
        h = 0.5 * fabs(tend - t);
        if (carry_warm(a, i) && a.carry[a.cidx(i, kCarryH)] > 0.0) h = a.carry[a.cidx(i, kCarryH)];
        delta = (a.atol_of(i) > 0.0) ? a.atol_of(i) / a.rtol_of(i) : kTiny;
        n_acc = n_rej = status = 0;
        max_att = a.max_attempts;
        loop_top();
    }
    __device__ bool done() const { return stage == 0; }

    // top of the rkckDriver loop: finished?  attempt cap, then clamp h
    __device__ void loop_top() {
        stage = 0;
        if (!(t < tend)) return;
        if (n_acc + n_rej >= max_att) {
            status = ODE_ST_MAX_ATTEMPTS;
            return;
        }
        h = fmin(tend - t, h);
        stage = 1;
    }

    // k_i = h f(t + a_i h, y + sum_j b_ij k_j): the point of stage i
    __device__ void point(double* x, double& tx) const {
        switch (stage) {
        case 1:
            tx = t;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = y[s];
            break;
        case 2:
            tx = t + ck::A2 * h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = y[s] + ck::B21 * k1[s];
            break;
        case 3:
            tx = t + ck::A3 * h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = y[s] + ck::B31 * k1[s] + ck::B32 * k2[s];
            break;
        case 4:
            tx = t + ck::A4 * h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = y[s] + ck::B41 * k1[s] + ck::B42 * k2[s] + ck::B43 * k3[s];
            break;
        case 5:
            tx = t + ck::A5 * h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                x[s] = y[s] + ck::B51 * k1[s] + ck::B52 * k2[s] + ck::B53 * k3[s] + ck::B54 * k4[s];
            break;
        default:
            tx = t + ck::A6 * h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                x[s] = y[s] + ck::B61 * k1[s] + ck::B62 * k2[s] + ck::B63 * k3[s] + ck::B64 * k4[s] +
                       ck::B65 * k5[s];
        }
    }

    __device__ bool consume(const BatchArgs&, const TM& tm, const double*, const double* f) {
        switch (stage) {
        case 1:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k1[s] = h * f[s];
            break;
        case 2:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k2[s] = h * f[s];
            break;
        case 3:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k3[s] = h * f[s];
            break;
        case 4:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k4[s] = h * f[s];
            break;
        case 5:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) k5[s] = h * f[s];
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
    __device__ void finish(const TM& tm, const double* f) {
        double yt[P];
        double err = 0.0;
        bool nan_flag = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const double k6 = h * f[s];
            yt[s] = y[s] + ck::C1 * k1[s] + ck::C3 * k3[s] + ck::C4 * k4[s] + ck::C6 * k6;
            const double ye = ck::DC1 * k1[s] + ck::DC3 * k3[s] + ck::DC4 * k4[s] + ck::DC5 * k5[s] + ck::DC6 * k6;
            if (sys.comp(tm, s) >= 0) {
                if (isnan(ye)) nan_flag = true;
                err = fmax(err, fabs(ye) / (fabs(y[s]) + fabs(k1[s]) + delta));
            }
        }
        err = tm.max(err) / rtol;
        nan_flag = tm.any(nan_flag);
        if (err > 1.0 || isnan(err) || nan_flag) {
            n_rej += 1;
            if (isnan(err) || nan_flag)
                h = h * kP1;
            else
                h = fmax(kSafety * h * xm::pow_series(err, kPshrnk), kP1 * h);
            if (h < 1.0e-20 || t + h == t) {
                status = ODE_ST_H_UNDERFLOW;
                stage = 0;
                return;
            }
            loop_top();
            return;
        }
        n_acc += 1;
        t = t + h;
        if (err > kErrcon)
            h = kSafety * h * xm::pow_series(err, kPgrow);
        else
            h = h * 5.0;
        h = fmax(1.0e-20, fmin(hmax, h));
        bool bad = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            y[s] = yt[s];
            if (sys.comp(tm, s) >= 0 && !isfinite(yt[s])) bad = true;
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
            if (c >= 0) a.y_out[a.yidx_out(i, c)] = y[s];
            if (a.carry != nullptr && c >= 0) a.carry[a.cidx(i, kCarryFixed + c)] = 0.0;
        }
        if (a.carry != nullptr && tm.lane == 0)
            carry_scalars(a, i, status == ODE_ST_OK || status == ODE_ST_MAX_ATTEMPTS, t, h, 0.0, 0.0, 0.0, 0, 0, false);
        if (tm.lane == 0) {
            if (a.n_accept) a.n_accept[i] = n_acc;
            if (a.n_reject) a.n_reject[i] = n_rej;
            if (a.n_rhs) a.n_rhs[i] = 6 * (n_acc + n_rej);
            if (a.n_specrad) a.n_specrad[i] = 0;
            if (a.status) a.status[i] = status;
        }
    }
};

// ================================================================= RKC F64

template <class Model>
struct RkcF64 {
    static constexpr bool kStepSync = true;  // variable stage count: hold at the step end
    static constexpr int SMEM_FLOATS = ModelSmem<Model>::value;
    __device__ void bind_smem(float* base, int stride) {
        if constexpr (SMEM_FLOATS > 0) sys.bind(base, stride);
    }
    static constexpr int W = Model::W, P = Model::PER;
    using R = double;
    using TM = Team<W>;
    typename Model::template Sys<double> sys;
    double yn[P], Fn[P], v[P], w1[P], w2[P];  // w1 = w_{j-1}, w2 = w_{j-2}
    double t, tend, rtol, atol, hmax, hmin, h, h_old, err_old, sigma;
    double dynrm, sig;                          // power method in progress
    StageCoef cur;                              // coefficients of the current stage
    CoefSource cs;
    int32_t n_acc, n_rej, n_rhs, n_sr, status, max_att, mmax, num_step, sr_step, n;
    int32_t phase, m, j, sr_iter;
    bool have_sigma, rejected, warm;
    int64_t idx;    // system index (training logs)
    int32_t n_est;  // spectral-radius estimates so far (training log)

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq_of(i));
        n = a.neq_of(i);
        idx = i;
        n_est = 0;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            yn[s] = c >= 0 ? a.y0[a.yidx(i, c)] : 0.0;
        }
        t = a.t0_of(i);
        tend = a.tend_of(i);
        rtol = a.rtol_of(i);
        atol = a.atol_of(i);
        mmax = (int)round(sqrt(rtol / (10.0 * kUround)));
        if (mmax < 2) mmax = 2;
        hmax = fabs(tend - t);
        hmin = 10.0 * kUround * fmax(fabs(t), hmax);
        n_acc = n_rej = n_sr = status = 0;
        n_rhs = 1;
        max_att = a.max_attempts;
        h = h_old = err_old = sigma = 0.0;
        num_step = 0;
        sr_step = -1;
        have_sigma = rejected = false;
        warm = carry_warm(a, i);
        if (warm) {  // resume the controller and the spectral-radius schedule
            h = a.carry[a.cidx(i, kCarryH)];
            sigma = a.carry[a.cidx(i, kCarrySigma)];
            h_old = a.carry[a.cidx(i, kCarryHold)];
            err_old = a.carry[a.cidx(i, kCarryErrOld)];
            num_step = (int)a.carry[a.cidx(i, kCarryNumStep)];
            sr_step = (int)a.carry[a.cidx(i, kCarrySrStep)];
            rejected = (int)a.carry[a.cidx(i, kCarryRejected)] != 0;
            have_sigma = true;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                const int c = sys.comp(tm, s);
                v[s] = c >= 0 ? a.carry[a.cidx(i, kCarryFixed + c)] : 0.0;
            }
            if (a.carry_mode == ODE_CARRY_RESTART) {  // the spectral-radius schedule starts again
                num_step = 0;
                sr_step = -1;
                rejected = false;
            }
        }
        phase = PH_F0;  // F_n = f(t0, y0)
    }
    __device__ bool done() const { return phase == PH_DONE; }
    __device__ bool in_stages() const { return phase == PH_STAGE; }
    __device__ bool at_step_end() const { return phase == PH_FINAL; }

    __device__ double sumsq(const TM& tm, const double* x) const {
        double sq[P];
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) sq[s] = x[s] * x[s];
        return sys.ordered_sum(tm, sq);
    }

    __device__ void point(double* x, double& tx) const {
        switch (phase) {
        case PH_F0:
            tx = t;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = yn[s];
            break;
        case PH_SR:
            tx = t;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = v[s];
            break;
        case PH_TRIAL:
            tx = t + h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = yn[s] + h * Fn[s];
            break;
        case PH_STAGE:
            tx = t + cur.cprev * h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = w1[s];
            break;
        default:  // PH_FINAL: F_{n+1} at w_m
            tx = t + h;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = w1[s];
        }
    }

    __device__ bool consume(const BatchArgs& a, const TM& tm, const double*, const double* f) {
        switch (phase) {
        case PH_F0:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                Fn[s] = f[s];
                if (!warm) v[s] = f[s];  // first eigenvector guess
            }
            loop_top(a, tm);
            break;
        case PH_SR: sr_consume(a, tm, f); break;
        case PH_TRIAL: trial_consume(a, tm, f); break;
        case PH_STAGE: stage_consume(a, f); break;
        default: final_consume(a, tm, f);
        }
        return done();
    }

    // top of the rkcDriver loop
    __device__ void loop_top(const BatchArgs& a, const TM& tm) {
        if (!(t < tend)) {
            phase = PH_DONE;
            return;
        }
        if (n_acc + n_rej >= max_att) {
            status |= ODE_ST_MAX_ATTEMPTS;
            phase = PH_DONE;
            return;
        }
        if (1.1 * h >= fabs(tend - t)) h = fabs(tend - t);
        if (!have_sigma || rejected || (num_step % kSpecradEvery == 0 && sr_step != num_step)) {
            if (a.specrad == ODE_SPECRAD_GERSHGORIN) {  // the bound replaces the power method
                sigma = sys.gershgorin(tm, yn);
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

    // nonlinear power method (Appendix): perturb y along v by |y| sqrt(uround)
    __device__ void sr_begin(const TM& tm) {
        const double sq = sqrt(kUround);
        const double nrm1 = sqrt(sumsq(tm, yn)), nrm2 = sqrt(sumsq(tm, v));
        if (nrm1 != 0.0 && nrm2 != 0.0) {
            dynrm = nrm1 * sq;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = yn[s] + v[s] * (dynrm / nrm2);
        } else if (nrm1 != 0.0) {
            dynrm = nrm1 * sq;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = yn[s] * (1.0 + sq);
        } else if (nrm2 != 0.0) {
            dynrm = kUround;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = v[s] * (dynrm / nrm2);
        } else {
            dynrm = kUround;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = kUround;
        }
        sig = 0.0;
        sr_iter = 0;
        phase = PH_SR;
    }

    __device__ void sr_consume(const BatchArgs& a, const TM& tm, const double* Fv) {
        sr_iter += 1;
        n_sr += 1;
        double sq[P];
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) sq[s] = (Fv[s] - Fn[s]) * (Fv[s] - Fn[s]);
        const double d = sqrt(sys.ordered_sum(tm, sq));
        const double sig_prev = sig;
        sig = d / dynrm;
        if (sr_iter >= 2 && fabs(sig - sig_prev) <= fmax(sig, 1.0 / hmax) * 0.01) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = v[s] - yn[s];
            sr_end(a, tm);
            return;
        }
        if (d != 0.0) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = yn[s] + (Fv[s] - Fn[s]) * (dynrm / d);
        } else {
            const int ind = sr_iter % n;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (opaque(sys.comp(tm, s)) == ind) v[s] = yn[s] - (v[s] - yn[s]);
        }
        if (sr_iter == kSpecradItmax) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) v[s] = v[s] - yn[s];
            status |= ODE_ST_SPECRAD_NOCONV;
            sr_end(a, tm);
        }
    }

    __device__ void sr_end(const BatchArgs& a, const TM& tm) {
        sigma = 1.2 * sig;
        if (a.specrad == ODE_SPECRAD_POWER_CAPPED) sigma = fmin(sigma, sys.gershgorin(tm, yn));
        have_sigma = true;
        sr_step = num_step;
        if (a.log_sr != nullptr) write_sr_log(a, tm);
        n_est += 1;
        after_sr(a);
    }

    // training record of a spectral-radius estimate: features of the state
    // it was taken at, the parameter and log sigma (n + 2 floats), for the
    // estimates the log's stride selects
    __device__ void write_sr_log(const BatchArgs& a, const TM& tm) const {
        const int every = a.log_sr_every > 0 ? a.log_sr_every : 1;
        if (n_est % every != 0 || n_est / every >= a.log_sr_records) return;
        float* rec = a.log_sr + (idx * (int64_t)a.log_sr_records + n_est / every) * (int64_t)(n + 2);
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            if (c >= 0) rec[c] = (float)log(fmax(fabs(yn[s]), 1e-30));
        }
        if (tm.lane == 0) {
            rec[n] = (float)a.params[idx];
            rec[n + 1] = (float)log(sigma);
        }
    }

    __device__ void after_sr(const BatchArgs& a) {
        if (h < kUround) {
            // initial step: trial Euler step of size 1/sigma
            h = hmax;
            if (sigma * h > 1.0) h = 1.0 / sigma;
            h = fmax(h, hmin);
            phase = PH_TRIAL;
            return;
        }
        stage_begin(a);
    }

    __device__ void trial_consume(const BatchArgs& a, const TM& tm, const double* f) {
        n_rhs += 1;
        double sq[P];
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const double e = (f[s] - Fn[s]) / (atol + rtol * fabs(yn[s]));
            sq[s] = e * e;
        }
        const double est = h * sqrt(sys.ordered_sum(tm, sq) / (double)n);
        if (kP1 * h < hmax * sqrt(est))
            h = fmax(kP1 * h / sqrt(est), hmin);
        else
            h = hmax;
        stage_begin(a);
    }

    // stage count, then w_0 = y_n, w_1 = w_0 + mu~_1 h F_n (Eqs. E:rkc0, E:rkc1)
    __device__ void stage_begin(const BatchArgs& a) {
        m = 1 + (int)sqrt(1.54 * h * sigma + 1.0);
        if (m > mmax) {
            m = mmax;
            h = (double)(m * m - 1) / (1.54 * sigma);
        }
        cs.start(m, a);
        const double mut1 = cs.mut1();
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            w2[s] = yn[s];
            w1[s] = yn[s] + mut1 * h * Fn[s];
        }
        j = 2;
        cur = cs.stage64(2);
        phase = PH_STAGE;
    }

    // Eq. E:rkcj with f_{j-1} = f(t + c_{j-1} h, w_{j-1})
    __device__ void stage_consume(const BatchArgs&, const double* f) {
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const double wj = cur.cy * yn[s] + cur.mu * w1[s] + cur.nu * w2[s] + cur.mut * h * f[s] + cur.gt * h * Fn[s];
            w2[s] = w1[s];
            w1[s] = wj;
        }
        j += 1;
        if (j <= m)
            cur = cs.stage64(j);
        else
            phase = PH_FINAL;
    }

    // error estimate (Eq. E:rmsE) and the step-size rules (Eqs. dtnp1, rkc-f)
    __device__ void final_consume(const BatchArgs& a, const TM& tm, const double* f) {
        n_rhs += m;
        double sq[P];
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            double e = 0.8 * (yn[s] - w1[s]) + 0.4 * h * (Fn[s] + f[s]);
            e = e / (atol + rtol * fmax(fabs(w1[s]), fabs(yn[s])));
            sq[s] = e * e;
        }
        const double err = sqrt(sys.ordered_sum(tm, sq) / (double)n);
        if (isnan(err)) {
            n_rej += 1;
            status |= ODE_ST_NONFINITE;
            phase = PH_DONE;
            return;
        }
        if (err > 1.0) {
            n_rej += 1;
            h = 0.8 * h / xm::pow_series(err, 1.0 / 3.0);
            rejected = true;
            if (h < hmin) {
                status |= ODE_ST_H_UNDERFLOW;
                phase = PH_DONE;
                return;
            }
            loop_top(a, tm);
            return;
        }
        if (a.log_xy != nullptr && n_acc == 0) write_log(a, tm);
        n_acc += 1;
        rejected = false;
        t = t + h;
        num_step += 1;
        double fac = 10.0;
        if (h_old < kUround) {
            const double temp2 = xm::pow_series(err, 1.0 / 3.0);
            if (0.8 < fac * temp2) fac = 0.8 / temp2;
        } else {
            const double temp1 = 0.8 * h * xm::pow_series(err_old, 1.0 / 3.0);
            const double temp2 = h_old * xm::pow_series(err, 2.0 / 3.0);
            if (temp1 < fac * temp2) fac = temp1 / temp2;
        }
        err_old = err;
        h_old = h;
        bool bad = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            yn[s] = w1[s];
            Fn[s] = f[s];
            if (sys.comp(tm, s) >= 0 && !isfinite(w1[s])) bad = true;
        }
        h = h * fmax(kP1, fac);
        h = fmax(hmin, fmin(hmax, h));
        if (tm.any(bad)) {
            status |= ODE_ST_NONFINITE;
            phase = PH_DONE;
            return;
        }
        loop_top(a, tm);
    }

    // training record of the first accepted step: features of the initial
    // state, the parameter, log h and log sigma (row of n + 4 floats; the
    // last, log n_rhs, is written when the system finishes)
    __device__ void write_log(const BatchArgs& a, const TM& tm) const {
        float* rec = a.log_xy + idx * (int64_t)(n + 4);
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            if (c >= 0) rec[c] = (float)log(fmax(fabs(yn[s]), 1e-30));
        }
        if (tm.lane == 0) {
            rec[n] = (float)a.params[idx];
            rec[n + 1] = (float)log(h);
            rec[n + 2] = (float)log(sigma);
        }
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            if (c >= 0) a.y_out[a.yidx_out(i, c)] = yn[s];
            if (a.carry != nullptr && c >= 0) a.carry[a.cidx(i, kCarryFixed + c)] = v[s];
        }
        if (a.carry != nullptr && tm.lane == 0) {
            const int st = status & 0xFF;
            carry_scalars(a, i, (st == ODE_ST_OK || st == ODE_ST_MAX_ATTEMPTS) && have_sigma, t, h, sigma, h_old,
                          err_old, num_step, sr_step, rejected);
        }
        if (tm.lane == 0) {
            if (a.log_xy != nullptr && n_acc > 0) a.log_xy[idx * (int64_t)(n + 4) + n + 3] = (float)log((double)(n_rhs + n_sr));
            if (a.n_accept) a.n_accept[i] = n_acc;
            if (a.n_reject) a.n_reject[i] = n_rej;
            if (a.n_rhs) a.n_rhs[i] = n_rhs + n_sr;
            if (a.n_specrad) a.n_specrad[i] = n_sr;
            if (a.status) a.status[i] = status;
        }
    }
};

// ============================================================== RKCK mixed

// x^p for the step-size factors of the mixed forms (x >= 0): two special
// function unit operations, relative error ~1e-6 -- ample for a safety factor.
__device__ __forceinline__ float fpow(float x, float p) { return exp2f(p * __log2f(x)); }

// Compensated FP32 accumulation (Knuth's two-sum): the rounding error of each
// addition is collected in c, so s + c carries the sum to about one rounding.
struct SumF2 {
    float s = 0.0f, c = 0.0f;
    __device__ void add(float x) {
        const float t = s + x;
        const float bb = t - s;
        c += (s - (t - bb)) + (x - bb);
        s = t;
    }
};

// SPEC: the split as specified (ODE_PREC_MIXED): time and step size in FP64.
// Otherwise (ODE_PREC_MIXED_LEAN) only the time t is FP64; the step size is
// FP32 and a step that reaches the end of the interval lands on tend exactly.
template <class Model, bool SPEC = true>
struct RkckMixed {
    static constexpr bool kStepSync = false;  // fixed six stages: lanes stay aligned
    static constexpr int SMEM_FLOATS = ModelSmem<Model>::value;
    __device__ void bind_smem(float* base, int stride) {
        if constexpr (SMEM_FLOATS > 0) sys.bind(base, stride);
    }
    static constexpr int W = Model::W, P = Model::PER;
    using R = float;
    using TM = Team<W>;
    using HT = typename Pick<SPEC, double, float>::type;
    typename Model::template Sys<float> sys;
    float yh[P], yl[P], k1[P], k2[P], k3[P], k4[P], k5[P];
    double t, tend;
    HT h, hmax;
    float hf, remf, reml, tendf, tabsf, deltaf, inv_rtolf;  // lean: remaining interval remf + reml
    int32_t n_acc, n_rej, status, max_att, stage;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq_of(i));
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            const double y0 = c >= 0 ? a.y0[a.yidx(i, c)] : 0.0;
            yh[s] = (float)y0;
            yl[s] = (float)(y0 - (double)yh[s]);
            k1[s] = k2[s] = k3[s] = k4[s] = k5[s] = 0.0f;
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
        deltaf = (float)((a.atol_of(i) > 0.0) ? a.atol_of(i) / a.rtol_of(i) : kTiny);
        inv_rtolf = (float)(1.0 / a.rtol_of(i));
        n_acc = n_rej = status = 0;
        max_att = a.max_attempts;
        loop_top();
    }
    __device__ bool done() const { return stage == 0; }

    __device__ void loop_top() {
        stage = 0;
        if constexpr (SPEC) {
            if (!(t < tend)) return;
        } else {
            if (!(remf > 0.0f)) return;
        }
        if (n_acc + n_rej >= max_att) {
            status = ODE_ST_MAX_ATTEMPTS;
            return;
        }
        if constexpr (SPEC)
            h = fmin(tend - t, h);
        else
            h = fminf(remf, h);
        hf = (float)h;
        stage = 1;
    }

    // stage point y + sum_j b_ij k_j with a zero-padded row of Table 1, so
    // lanes at different stages run the same instructions
    __device__ void point(float* x, float& tx) const {
        float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f, b5 = 0.f;
        switch (stage) {
        case 2: b1 = (float)ck::B21; break;
        case 3: b1 = (float)ck::B31; b2 = (float)ck::B32; break;
        case 4: b1 = (float)ck::B41; b2 = (float)ck::B42; b3 = (float)ck::B43; break;
        case 5: b1 = (float)ck::B51; b2 = (float)ck::B52; b3 = (float)ck::B53; b4 = (float)ck::B54; break;
        case 6:
            b1 = (float)ck::B61; b2 = (float)ck::B62; b3 = (float)ck::B63; b4 = (float)ck::B64; b5 = (float)ck::B65;
            break;
        default: break;
        }
        if constexpr (SPEC)
            tx = (float)t;
        else
            tx = tendf - remf;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) x[s] = yh[s] + (b1 * k1[s] + b2 * k2[s] + b3 * k3[s] + b4 * k4[s] + b5 * k5[s]);
    }

    __device__ bool consume(const BatchArgs&, const TM& tm, const float*, const float* f) {
        if (stage == 6) {
            finish(tm, f);
            return done();
        }
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const float k = hf * f[s];
            k1[s] = stage == 1 ? k : k1[s];
            k2[s] = stage == 2 ? k : k2[s];
            k3[s] = stage == 3 ? k : k3[s];
            k4[s] = stage == 4 ? k : k4[s];
            k5[s] = stage == 5 ? k : k5[s];
        }
        stage += 1;
        return false;
    }

    __device__ void finish(const TM& tm, const float* f) {
        float incr[P];
        float err = 0.0f;
        bool nan_flag = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const float k6 = hf * f[s];
            incr[s] = (float)ck::C1 * k1[s] + (float)ck::C3 * k3[s] + (float)ck::C4 * k4[s] + (float)ck::C6 * k6;
            const float ye = (float)ck::DC1 * k1[s] + (float)ck::DC3 * k3[s] + (float)ck::DC4 * k4[s] +
                             (float)ck::DC5 * k5[s] + (float)ck::DC6 * k6;
            if (sys.comp(tm, s) >= 0) {
                if (isnan(ye) || isnan(incr[s])) nan_flag = true;
                err = fmaxf(err, __fdividef(fabsf(ye), fabsf(yh[s]) + fabsf(k1[s]) + deltaf));
            }
        }
        err = tm.max(err) * inv_rtolf;
        nan_flag = tm.any(nan_flag);
        if (err > 1.0f || isnan(err) || nan_flag) {
            n_rej += 1;
            if (isnan(err) || nan_flag) {
                h = h * (HT)kP1;
#pragma unroll(P <= 64 ? P : 4)
                for (int s = 0; s < P; ++s) k1[s] = k2[s] = k3[s] = k4[s] = k5[s] = 0.0f;
            } else {
                h = h * (HT)fmaxf((float)kSafety * fpow(err, (float)kPshrnk), (float)kP1);
            }
            bool underflow;
            if constexpr (SPEC)
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
        if constexpr (SPEC) {
            t = t + h;
        } else if (h >= remf * 0.999999f) {
            remf = reml = 0.0f;  // the step covered what was left
        } else {
            df_sub(remf, reml, h);
            tabsf = fabsf(tendf - remf);
        }
        const float fac = (err > (float)kErrcon) ? (float)kSafety * fpow(err, (float)kPgrow) : 5.0f;
        if constexpr (SPEC)
            h = fmax(1.0e-20, fmin(hmax, h * (double)fac));
        else
            h = fmaxf(1.0e-20f, fminf(hmax, h * fac));
        bool bad = false;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            kahan_add(yh[s], yl[s], incr[s]);
            if (sys.comp(tm, s) >= 0 && !isfinite(yh[s])) bad = true;
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
            if (c >= 0) a.y_out[a.yidx_out(i, c)] = (double)yh[s] + (double)yl[s];
            if (a.carry != nullptr && c >= 0) a.carry[a.cidx(i, kCarryFixed + c)] = 0.0;
        }
        if (a.carry != nullptr && tm.lane == 0) {
            const double t_end = SPEC ? (double)t : tend - ((double)remf + (double)reml);
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

// =============================================================== RKC mixed

// SPEC (ODE_PREC_MIXED): time, step size and spectral radius in FP64 and the
// weighted error norm accumulated in FP64, as specified.  Otherwise
// (ODE_PREC_MIXED_LEAN): only the time t in FP64; step size, spectral radius
// and norms in FP32.
template <class Model, bool SPEC = true>
struct RkcMixed {
    static constexpr bool kStepSync = true;  // variable stage count: hold at the step end
    static constexpr int W = Model::W, P = Model::PER;
    using R = float;
    using TM = Team<W>;
    using HT = typename Pick<SPEC, double, float>::type;
    typename Model::template Sys<float> sys;
    float yh[P], yl[P], Fn[P], d1[P], d2[P];  // d_j = w_j - y_n (d_0 = 0)
    // Power-method vector v: touched only in the rare power-method phases,
    // so for small one-thread systems it lives in shared memory, which frees
    // P registers for the state the stages use.  Each thread owns one row of
    // V_SMEM (odd) floats: element s sits at a constant offset from a single
    // base address, and the odd pitch puts a warp's 32 rows in 32 banks.
    static constexpr int V_SMEM = rkc_mixed_smem_floats(W, P);
    static constexpr int SMEM_FLOATS = V_SMEM + ModelSmem<Model>::value;
    // register budget of the kernels (255: the launch bounds alone decide).
    // Lean warp-team systems of >= 8 values per lane (the 129-256-unknown
    // Brusselator grids) otherwise take ~200 registers and 4 blocks of 64
    // per SM; at 168 they keep 6.
    static constexpr int kMaxRegs = (!SPEC && W == 32 && P >= 8) ? 168 : 255;
    mutable float vreg[V_SMEM ? 1 : P];
    float* vs;
    __device__ void bind_smem(float* base, int stride) {
        vs = base + threadIdx.x * V_SMEM;  // this thread's row
        if constexpr (ModelSmem<Model>::value > 0) sys.bind(base + V_SMEM * stride, stride);
    }
    __device__ float& V(int s) const {
        if constexpr (V_SMEM > 0)
            return vs[s];
        else
            return vreg[s];
    }
    double t, tend;
    HT hmax, hmin, h, h_old, sigma;
    float rtolf, atolf, c3_old, hf, remf, dynrm, sig, inv_nf;  // c3_old = err_old^(1/3)
    float reml, tendf;  // lean: remaining interval remf + reml, FP32 end time for f(t, y)
    float4 cur;  // (mu_j, nu_j, mu~_j, gamma~_j) of the current stage
    CoefSource cs;
    int32_t n_acc, n_rej, n_rhs, n_sr, status, max_att, mmax, num_step, sr_step, n;
    int32_t phase, m, j, sr_iter;
    bool have_sigma, rejected, warm;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq_of(i));
        n = a.neq_of(i);
        inv_nf = 1.0f / (float)n;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const int c = sys.comp(tm, s);
            const double y0 = c >= 0 ? a.y0[a.yidx(i, c)] : 0.0;
            yh[s] = (float)y0;
            yl[s] = (float)(y0 - (double)yh[s]);
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
                V(s) = c >= 0 ? (float)a.carry[a.cidx(i, kCarryFixed + c)] : 0.0f;
            }
            if (a.carry_mode == ODE_CARRY_RESTART) {  // the spectral-radius schedule starts again
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

    template <class X>
    __device__ float sumsq(const TM& tm, X x_of) const {
        float acc = 0.0f;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s)
            if (sys.comp(tm, s) >= 0) acc = acc + x_of(s) * x_of(s);
        return tm.sum(acc);
    }

    __device__ void point(float* x, float& tx) const {
        if constexpr (SPEC)
            tx = (float)t;
        else
            tx = tendf - remf;
        switch (phase) {
        case PH_F0:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = yh[s];
            break;
        case PH_SR:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = V(s);
            break;
        case PH_TRIAL:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) x[s] = yh[s] + hf * Fn[s];
            break;
        default:  // stages and F_{n+1}: w = y_n + d
            if constexpr (SPEC) {
#pragma unroll(P <= 64 ? P : 4)
                for (int s = 0; s < P; ++s) x[s] = yh[s] + (yl[s] + d1[s]);
            } else {  // lean: the compensation word is below half an ulp of yh, so it moves no point
#pragma unroll(P <= 64 ? P : 4)
                for (int s = 0; s < P; ++s) x[s] = yh[s] + d1[s];
            }
        }
    }

    __device__ bool consume(const BatchArgs& a, const TM& tm, const float* x, const float* f) {
        switch (phase) {
        case PH_F0:
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) {
                Fn[s] = f[s];
                if (!warm) V(s) = f[s];  // first eigenvector guess
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
        if constexpr (SPEC) {
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
        if constexpr (SPEC) {
            if (1.1 * h >= fabs(tend - t)) h = fabs(tend - t);
        } else {
            if (1.1f * h >= remf) h = remf;
        }
        if (!have_sigma || rejected || (num_step % kSpecradEvery == 0 && sr_step != num_step)) {
            if (a.specrad == ODE_SPECRAD_GERSHGORIN) {  // the bound replaces the power method
                sigma = (HT)sys.gershgorin(tm, yh);
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

    // power method in FP32, perturbation scaled by the FP32 sqrt(uround)
    __device__ void sr_begin(const TM& tm) {
        const float nrm1 = sqrtf(sumsq(tm, [&](int s) { return yh[s]; }));
        const float nrm2 = sqrtf(sumsq(tm, [&](int s) { return V(s); }));
        if (nrm1 != 0.0f && nrm2 != 0.0f) {
            dynrm = nrm1 * kSqrtUroundF;
            const float sc = dynrm / nrm2;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = yh[s] + V(s) * sc;
        } else if (nrm1 != 0.0f) {
            dynrm = nrm1 * kSqrtUroundF;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = yh[s] * (1.0f + kSqrtUroundF);
        } else if (nrm2 != 0.0f) {
            dynrm = kSqrtUroundF;
            const float sc = dynrm / nrm2;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = V(s) * sc;
        } else {
            dynrm = kSqrtUroundF;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = kSqrtUroundF;
        }
        sig = 0.0f;
        sr_iter = 0;
        phase = PH_SR;
    }

    __device__ void sr_consume(const BatchArgs& a, const TM& tm, const float* Fv) {
        sr_iter += 1;
        n_sr += 1;
        float acc = 0.0f;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s)
            if (sys.comp(tm, s) >= 0) acc = acc + (Fv[s] - Fn[s]) * (Fv[s] - Fn[s]);
        const float d = sqrtf(tm.sum(acc));
        const float sig_prev = sig;
        sig = d / dynrm;
        if (sr_iter >= 2 && fabsf(sig - sig_prev) <= fmaxf(sig, 1.0f / (float)hmax) * 0.01f) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = V(s) - yh[s];
            sr_end(a, tm);
            return;
        }
        if (d != 0.0f) {
            const float sc = dynrm / d;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = yh[s] + (Fv[s] - Fn[s]) * sc;
        } else {
            const int ind = sr_iter % n;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (opaque(sys.comp(tm, s)) == ind) V(s) = yh[s] - (V(s) - yh[s]);
        }
        if (sr_iter == kSpecradItmax) {
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s) V(s) = V(s) - yh[s];
            status |= ODE_ST_SPECRAD_NOCONV;
            sr_end(a, tm);
        }
    }

    __device__ void sr_end(const BatchArgs& a, const TM& tm) {
        sigma = (HT)1.2 * (HT)sig;
        if (a.specrad == ODE_SPECRAD_POWER_CAPPED) {
            const HT g = (HT)sys.gershgorin(tm, yh);
            if constexpr (SPEC)
                sigma = fmin(sigma, g);
            else
                sigma = fminf(sigma, g);
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
            hf = (float)h;
            phase = PH_TRIAL;
            return;
        }
        stage_begin(a);
    }

    // weighted sum of squares of e, FP64 (SPEC) or compensated FP32
    template <class E>
    __device__ double weighted_ssq(const TM& tm, E e_of) const {
        if constexpr (SPEC) {
            double acc = 0.0;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (sys.comp(tm, s) >= 0) {
                    const float e = e_of(s);
                    acc = fma((double)e, (double)e, acc);
                }
            return tm.sum(acc);
        } else {
            SumF2 acc;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (sys.comp(tm, s) >= 0) {
                    const float e = e_of(s);
                    acc.add(e * e);
                }
            return (double)(tm.sum(acc.s) + tm.sum(acc.c));
        }
    }

    __device__ void trial_consume(const BatchArgs& a, const TM& tm, const float* f) {
        n_rhs += 1;
        if constexpr (SPEC) {
            const double ssq = weighted_ssq(tm, [&](int s) {
                return (f[s] - Fn[s]) / (atolf + rtolf * fabsf(yh[s]));
            });
            const double est = h * sqrt(ssq / (double)n);
            if (kP1 * h < hmax * sqrt(est))
                h = fmax(kP1 * h / sqrt(est), hmin);
            else
                h = hmax;
        } else {
            float acc = 0.0f;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (sys.comp(tm, s) >= 0) {
                    const float e = __fdividef(f[s] - Fn[s], atolf + rtolf * fabsf(yh[s]));
                    acc = fmaf(e, e, acc);
                }
            const float est = h * sqrtf(tm.sum(acc) * inv_nf);
            if ((float)kP1 * h < hmax * sqrtf(est))
                h = fmaxf((float)kP1 * h / sqrtf(est), hmin);
            else
                h = hmax;
        }
        stage_begin(a);
    }

    __device__ void stage_begin(const BatchArgs& a) {
        if constexpr (SPEC)
            m = 1 + (int)sqrtf((float)(1.54 * h * sigma) + 1.0f);
        else
            m = 1 + (int)sqrtf(1.54f * h * sigma + 1.0f);
        if (m > mmax) {
            m = mmax;
            h = (HT)(m * m - 1) / ((HT)1.54 * sigma);
        }
        hf = (float)h;
        cs.start(m, a);
        float mut1h;
        if constexpr (SPEC)
            mut1h = (float)cs.mut1() * hf;
        else
            mut1h = cs.mut1f() * hf;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            d2[s] = 0.0f;
            d1[s] = mut1h * Fn[s];
        }
        j = 2;
        cur = cs.stage32(2);
        phase = PH_STAGE;
    }

    // d_j = mu_j d_{j-1} + nu_j d_{j-2} + mu~_j h f_{j-1} + gamma~_j h F_n
    __device__ void stage_consume(const float* f) {
        const float muth = cur.z * hf, gth = cur.w * hf;
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            const float dj = cur.x * d1[s] + cur.y * d2[s] + muth * f[s] + gth * Fn[s];
            d2[s] = d1[s];
            d1[s] = dj;
        }
        j += 1;
        if (j <= m)
            cur = cs.stage32(j);
        else
            phase = PH_FINAL;
    }

    // x = w_m (the point F_{n+1} was evaluated at), f = F_{n+1}
    __device__ void final_consume(const BatchArgs& a, const TM& tm, const float* x, const float* f) {
        n_rhs += m;
        const float h04 = 0.4f * hf;
        bool reject, bad_err;
        float err;
        if constexpr (SPEC) {
            const double ms = weighted_ssq(tm, [&](int s) {
                return (-0.8f * d1[s] + h04 * (Fn[s] + f[s])) / (atolf + rtolf * fmaxf(fabsf(x[s]), fabsf(yh[s])));
            }) / (double)n;  // err^2
            bad_err = isnan(ms);
            reject = ms > 1.0;
            err = sqrtf((float)ms);
        } else {
            // FP32 accumulation: the estimate itself carries ~3 digits (its
            // terms cancel), far coarser than the rounding of this sum
            float acc = 0.0f;
#pragma unroll(P <= 64 ? P : 4)
            for (int s = 0; s < P; ++s)
                if (sys.comp(tm, s) >= 0) {
                    const float e = __fdividef(-0.8f * d1[s] + h04 * (Fn[s] + f[s]),
                                               atolf + rtolf * fmaxf(fabsf(x[s]), fabsf(yh[s])));
                    acc = fmaf(e, e, acc);
                }
            const float ms = tm.sum(acc) * inv_nf;  // err^2
            bad_err = isnan(ms);
            reject = ms > 1.0f;
            err = sqrtf(ms);
        }
        if (bad_err) {
            n_rej += 1;
            status |= ODE_ST_NONFINITE;
            phase = PH_DONE;
            return;
        }
        const float c3 = fpow(err, 1.0f / 3.0f);
        if (reject) {
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
            const float temp1 = 0.8f * hf * c3_old;
            const float temp2 = (float)h_old * (c3 * c3);
            if (temp1 < fac * temp2) fac = temp1 / temp2;
        }
        c3_old = c3;
        h_old = h;
        if constexpr (SPEC) {
            t = t + h;
        } else if (h >= remf * 0.999999f) {
            remf = reml = 0.0f;  // the step covered what was left
        } else {
            df_sub(remf, reml, h);
        }
        bool bad = false;
        float chk = 0.0f;  // lean form: one finiteness test of a sum per system
#pragma unroll(P <= 64 ? P : 4)
        for (int s = 0; s < P; ++s) {
            kahan_add(yh[s], yl[s], d1[s]);
            Fn[s] = f[s];
            if constexpr (SPEC) {
                if (sys.comp(tm, s) >= 0 && !isfinite(yh[s])) bad = true;
            } else {
                chk += (sys.comp(tm, s) >= 0) ? yh[s] - yh[s] : 0.0f;
            }
        }
        if constexpr (!SPEC) bad = !(chk == 0.0f);
        if constexpr (SPEC) {
            h = h * (double)fmaxf((float)kP1, fac);
            h = fmax(hmin, fmin(hmax, h));
        } else {
            h = h * fmaxf((float)kP1, fac);
            h = fmaxf(hmin, fminf(hmax, h));
        }
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
            if (c >= 0) a.y_out[a.yidx_out(i, c)] = (double)yh[s] + (double)yl[s];
            if (a.carry != nullptr && c >= 0) a.carry[a.cidx(i, kCarryFixed + c)] = (double)V(s);
        }
        if (a.carry != nullptr && tm.lane == 0) {
            const int st = status & 0xFF;
            const double t_end = SPEC ? (double)t : tend - ((double)remf + (double)reml);
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

}  // namespace bode

#include "integrators_f2.cuh"
