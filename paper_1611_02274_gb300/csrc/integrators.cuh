// integrators.cuh -- per-system RKCK and RKC state machines.
//
// One object integrates one system on one team of lanes (team.cuh);
// attempt() performs exactly one trial step (plus whatever spectral-radius
// or initial-step work precedes it) and returns true once the system is
// finished, so a persistent kernel can refill a team the moment its system
// ends.  Two arithmetic forms:
//   *F64    the plain form: every operation in FP64, following the
//           rkckDriver / rkcDriver listings of Section 3 step by step;
//   *Mixed  FP32 right-hand sides and stage arithmetic, state kept as an
//           FP32 pair (value + Kahan compensation); time, step size and
//           spectral radius in FP64, the RKC weighted error norm accumulated
//           in FP64, Chebyshev coefficients computed in FP64.
#pragma once
#include <cmath>

#include "common.cuh"
#include "team.cuh"
#include "xmath.cuh"

namespace bode {

// Cash-Karp coefficients (Table 1) and c_i - c*_i as exact rationals.
namespace ck {
constexpr double A2 = 1.0 / 5.0, A3 = 3.0 / 10.0, A4 = 3.0 / 5.0, A5 = 1.0, A6 = 7.0 / 8.0;
constexpr double B21 = 1.0 / 5.0;
constexpr double B31 = 3.0 / 40.0, B32 = 9.0 / 40.0;
constexpr double B41 = 3.0 / 10.0, B42 = -9.0 / 10.0, B43 = 6.0 / 5.0;
constexpr double B51 = -11.0 / 54.0, B52 = 5.0 / 2.0, B53 = -70.0 / 27.0, B54 = 35.0 / 27.0;
constexpr double B61 = 1631.0 / 55296.0, B62 = 175.0 / 512.0, B63 = 575.0 / 13824.0,
                 B64 = 44275.0 / 110592.0, B65 = 253.0 / 4096.0;
constexpr double C1 = 37.0 / 378.0, C3 = 250.0 / 621.0, C4 = 125.0 / 594.0, C6 = 512.0 / 1771.0;
constexpr double DC1 = -277.0 / 64512.0, DC3 = 6925.0 / 370944.0, DC4 = -6925.0 / 202752.0,
                 DC5 = -277.0 / 14336.0, DC6 = 277.0 / 7084.0;
}  // namespace ck

// FP32 unit roundoff and its square root: the mixed form's power method
// perturbs the state by sqrt(u) relative, the scale at which an FP32
// difference quotient is meaningful.
constexpr float kSqrtUroundF = 3.4526698e-4f;

// ------------------------------------------------------- RKC coefficients

struct StageCoef {
    double cy, mu, nu, mut, gt, cprev;  // 1 - mu - nu, mu_j, nu_j, mu~_j, gamma~_j, c_{j-1}
};

// Rolling Chebyshev recurrences of an m-stage RKC step (Section 2.2):
// w0 = 1 + kappa / m^2 (kappa = 2/13), T_j, T_j', T_j'' at w0 by the
// three-term recurrence and its derivatives, w1 = T_m'/T_m'',
// b_j = T_j''/(T_j')^2, b_0 = b_1 = b_2, a_j = 1 - b_j T_j,
// mu~_1 = b_1 w1, mu_j = 2 b_j w0 / b_{j-1}, nu_j = -b_j / b_{j-2},
// mu~_j = 2 b_j w1 / b_{j-1}, gamma~_j = -a_{j-1} mu~_j, and stage times
// c_1 = mu~_1, c_j = mu_j c_{j-1} + nu_j c_{j-2} + mu~_j (1 - a_{j-1}).
struct RkcStageGen {
    double w0, w1, b2, mut1;
    double Tm1, Tm2, Pm1, Pm2, Qm1, Qm2, bm1, bm2, cm1, cm2;

    __device__ void start(int m) {
        w0 = 1.0 + (2.0 / 13.0) / ((double)m * (double)m);
        double T0 = 1.0, T1 = w0, P0 = 0.0, P1 = 1.0, Q0 = 0.0, Q1 = 0.0, Tp2 = 0.0, Tpp2 = 0.0;
        for (int j = 2; j <= m; ++j) {
            const double T2 = 2.0 * w0 * T1 - T0;
            const double P2 = 2.0 * T1 + 2.0 * w0 * P1 - P0;
            const double Q2 = 4.0 * P1 + 2.0 * w0 * Q1 - Q0;
            if (j == 2) {
                Tp2 = P2;
                Tpp2 = Q2;
            }
            T0 = T1;
            T1 = T2;
            P0 = P1;
            P1 = P2;
            Q0 = Q1;
            Q1 = Q2;
        }
        w1 = P1 / Q1;
        b2 = Tpp2 / (Tp2 * Tp2);
        mut1 = b2 * w1;
        Tm1 = w0;
        Tm2 = 1.0;
        Pm1 = 1.0;
        Pm2 = 0.0;
        Qm1 = 0.0;
        Qm2 = 0.0;
        bm1 = b2;
        bm2 = b2;
        cm1 = mut1;
        cm2 = 0.0;
    }
    // coefficients of the next stage j = 2, 3, ...
    __device__ StageCoef next() {
        StageCoef s;
        const double Tj = 2.0 * w0 * Tm1 - Tm2;
        const double Pj = 2.0 * Tm1 + 2.0 * w0 * Pm1 - Pm2;
        const double Qj = 4.0 * Pm1 + 2.0 * w0 * Qm1 - Qm2;
        const double bj = Qj / (Pj * Pj);
        s.mu = 2.0 * bj * w0 / bm1;
        s.nu = -bj / bm2;
        s.mut = 2.0 * bj * w1 / bm1;
        const double ajm1 = 1.0 - bm1 * Tm1;
        s.gt = -ajm1 * s.mut;
        s.cy = 1.0 - s.mu - s.nu;
        s.cprev = cm1;
        const double cj = s.mu * cm1 + s.nu * cm2 + s.mut * (1.0 - ajm1);
        cm2 = cm1;
        cm1 = cj;
        Tm2 = Tm1;
        Tm1 = Tj;
        Pm2 = Pm1;
        Pm1 = Pj;
        Qm2 = Qm1;
        Qm1 = Qj;
        bm2 = bm1;
        bm1 = bj;
        return s;
    }
};

// Coefficients from the precomputed table when m is in range, else from the
// rolling recurrence (identical arithmetic: the table is built by it).
struct CoefSource {
    const double* e64;
    const float4* e32;
    bool table;
    RkcStageGen gen;
    __device__ void start(int m, const BatchArgs& a) {
        table = (m <= a.rkc_tab_max) && (a.rkc_tab64 != nullptr);
        if (table) {
            const int base = rkc_tab_index(m, 1);
            e64 = a.rkc_tab64 + 8 * base;
            e32 = a.rkc_tab32 + base;
        } else {
            gen.start(m);
        }
    }
    __device__ double mut1() const { return table ? __ldg(e64 + 3) : gen.mut1; }
    __device__ StageCoef stage64(int j) {
        if (table) {
            const double2* p = reinterpret_cast<const double2*>(e64 + 8 * (j - 1));
            const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
            return StageCoef{a.x, a.y, b.x, b.y, c.x, c.y};
        }
        return gen.next();
    }
    __device__ float4 stage32(int j) {
        if (table) return __ldg(e32 + (j - 1));
        const StageCoef s = gen.next();
        return make_float4((float)s.mu, (float)s.nu, (float)s.mut, (float)s.gt);
    }
};

// Builds the coefficient table for m = 2..mmax (one thread per m).
__global__ void k_build_rkc_table(double* tab64, float4* tab32, int mmax);

// ================================================================= RKCK F64

template <class Model>
struct RkckF64 {
    static constexpr int W = Model::W, P = Model::PER;
    using TM = Team<W>;
    typename Model::template Sys<double> sys;
    double y[P];
    int comp[P];
    double t, tend, h, hmax, delta, rtol;
    int32_t n_acc, n_rej, status, max_att;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq);
#pragma unroll
        for (int s = 0; s < P; ++s) {
            comp[s] = sys.comp(tm, s);
            y[s] = comp[s] >= 0 ? a.y0[i + a.nsys * (int64_t)comp[s]] : 0.0;
        }
        t = a.t0;
        tend = a.tend;
        rtol = a.rtol;
        hmax = fabs(tend - t);
        h = 0.5 * fabs(tend - t);
        delta = (a.atol > 0.0) ? a.atol / a.rtol : kTiny;
        n_acc = n_rej = status = 0;
        max_att = a.max_attempts;
    }

    // One trial step of the rkckDriver loop (Section 3.1) with the error
    // scale of Section 2.1; returns true when the system is finished.
    __device__ bool attempt(const BatchArgs&, const TM& tm) {
        if (!(t < tend)) return true;
        if (n_acc + n_rej >= max_att) {
            status = ODE_ST_MAX_ATTEMPTS;
            return true;
        }
        h = fmin(tend - t, h);
        double F[P], k1[P], k2[P], k3[P], k4[P], k5[P], yt[P], f[P];
        sys.rhs(tm, t, y, F);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k1[i] = h * F[i];
            yt[i] = y[i] + ck::B21 * k1[i];
        }
        sys.rhs(tm, t + ck::A2 * h, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k2[i] = h * f[i];
            yt[i] = y[i] + ck::B31 * k1[i] + ck::B32 * k2[i];
        }
        sys.rhs(tm, t + ck::A3 * h, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k3[i] = h * f[i];
            yt[i] = y[i] + ck::B41 * k1[i] + ck::B42 * k2[i] + ck::B43 * k3[i];
        }
        sys.rhs(tm, t + ck::A4 * h, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k4[i] = h * f[i];
            yt[i] = y[i] + ck::B51 * k1[i] + ck::B52 * k2[i] + ck::B53 * k3[i] + ck::B54 * k4[i];
        }
        sys.rhs(tm, t + ck::A5 * h, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k5[i] = h * f[i];
            yt[i] = y[i] + ck::B61 * k1[i] + ck::B62 * k2[i] + ck::B63 * k3[i] + ck::B64 * k4[i] +
                    ck::B65 * k5[i];
        }
        sys.rhs(tm, t + ck::A6 * h, yt, f);
        double err = 0.0;
        bool nan_flag = false;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const double k6 = h * f[i];
            yt[i] = y[i] + ck::C1 * k1[i] + ck::C3 * k3[i] + ck::C4 * k4[i] + ck::C6 * k6;
            const double ye =
                ck::DC1 * k1[i] + ck::DC3 * k3[i] + ck::DC4 * k4[i] + ck::DC5 * k5[i] + ck::DC6 * k6;
            if (comp[i] >= 0) {
                if (isnan(ye)) nan_flag = true;
                err = fmax(err, fabs(ye) / (fabs(y[i]) + fabs(h * F[i]) + delta));
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
                return true;
            }
            return false;
        }
        n_acc += 1;
        t = t + h;
        if (err > kErrcon)
            h = kSafety * h * xm::pow_series(err, kPgrow);
        else
            h = h * 5.0;
        h = fmax(1.0e-20, fmin(hmax, h));
        bool bad = false;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            y[i] = yt[i];
            if (comp[i] >= 0 && !isfinite(yt[i])) bad = true;
        }
        if (tm.any(bad)) {
            status = ODE_ST_NONFINITE;
            return true;
        }
        return !(t < tend);
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (comp[s] >= 0) a.y_out[i + a.nsys * (int64_t)comp[s]] = y[s];
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
    static constexpr int W = Model::W, P = Model::PER;
    using TM = Team<W>;
    typename Model::template Sys<double> sys;
    double yn[P], Fn[P], v[P];
    int comp[P];
    double t, tend, rtol, atol, hmax, hmin, h, h_old, err_old, sigma;
    int32_t n_acc, n_rej, n_rhs, n_sr, status, max_att, mmax, num_step, sr_step, n;
    bool have_sigma, rejected;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq);
        n = a.neq;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            comp[s] = sys.comp(tm, s);
            yn[s] = comp[s] >= 0 ? a.y0[i + a.nsys * (int64_t)comp[s]] : 0.0;
        }
        t = a.t0;
        tend = a.tend;
        rtol = a.rtol;
        atol = a.atol;
        mmax = (int)round(sqrt(rtol / (10.0 * kUround)));
        if (mmax < 2) mmax = 2;
        hmax = fabs(tend - t);
        hmin = 10.0 * kUround * fmax(fabs(t), hmax);
        sys.rhs(tm, t, yn, Fn);
#pragma unroll
        for (int s = 0; s < P; ++s) v[s] = Fn[s];
        n_acc = n_rej = n_sr = status = 0;
        n_rhs = 1;
        max_att = a.max_attempts;
        h = h_old = err_old = sigma = 0.0;
        num_step = 0;
        sr_step = -1;
        have_sigma = rejected = false;
    }

    // sum of squares in component order (the oracle's sequential loop)
    __device__ double sumsq(const TM& tm, const double* x) const {
        double sq[P];
#pragma unroll
        for (int s = 0; s < P; ++s) sq[s] = x[s] * x[s];
        return sys.ordered_sum(tm, sq);
    }

    // Nonlinear power method (Appendix) around (yn, Fn); v persists.
    __device__ double specrad(const TM& tm) {
        const double small = 1.0 / hmax;
        const double sq = sqrt(kUround);
        const double nrm1 = sqrt(sumsq(tm, yn)), nrm2 = sqrt(sumsq(tm, v));
        double dynrm;
        if (nrm1 != 0.0 && nrm2 != 0.0) {
            dynrm = nrm1 * sq;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = yn[s] + v[s] * (dynrm / nrm2);
        } else if (nrm1 != 0.0) {
            dynrm = nrm1 * sq;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = yn[s] * (1.0 + sq);
        } else if (nrm2 != 0.0) {
            dynrm = kUround;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = v[s] * (dynrm / nrm2);
        } else {
            dynrm = kUround;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = kUround;
        }
        double sig = 0.0;
        for (int iter = 1; iter <= kSpecradItmax; ++iter) {
            double Fv[P];
            sys.rhs(tm, t, v, Fv);
            n_sr += 1;
            double sq[P];
#pragma unroll
            for (int s = 0; s < P; ++s) sq[s] = (Fv[s] - Fn[s]) * (Fv[s] - Fn[s]);
            const double d = sqrt(sys.ordered_sum(tm, sq));
            const double sig_prev = sig;
            sig = d / dynrm;
            if (iter >= 2 && fabs(sig - sig_prev) <= fmax(sig, small) * 0.01) {
#pragma unroll
                for (int s = 0; s < P; ++s) v[s] = v[s] - yn[s];
                return 1.2 * sig;
            }
            if (d != 0.0) {
#pragma unroll
                for (int s = 0; s < P; ++s) v[s] = yn[s] + (Fv[s] - Fn[s]) * (dynrm / d);
            } else {
                const int ind = iter % n;
#pragma unroll
                for (int s = 0; s < P; ++s)
                    if (comp[s] == ind) v[s] = yn[s] - (v[s] - yn[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < P; ++s) v[s] = v[s] - yn[s];
        status |= ODE_ST_SPECRAD_NOCONV;
        return 1.2 * sig;
    }

    // One trial step of the rkcDriver loop (Section 3.2).
    __device__ bool attempt(const BatchArgs& a, const TM& tm) {
        if (!(t < tend)) return true;
        if (n_acc + n_rej >= max_att) {
            status |= ODE_ST_MAX_ATTEMPTS;
            return true;
        }
        if (1.1 * h >= fabs(tend - t)) h = fabs(tend - t);
        if (!have_sigma || rejected || (num_step % kSpecradEvery == 0 && sr_step != num_step)) {
            sigma = specrad(tm);
            have_sigma = true;
            sr_step = num_step;
        }
        double w1v[P], w2[P], f[P];
        if (h < kUround) {
            // initial step: trial Euler step of size 1/sigma
            h = hmax;
            if (sigma * h > 1.0) h = 1.0 / sigma;
            h = fmax(h, hmin);
#pragma unroll
            for (int s = 0; s < P; ++s) w1v[s] = yn[s] + h * Fn[s];
            sys.rhs(tm, t + h, w1v, f);
            n_rhs += 1;
            double sq[P];
#pragma unroll
            for (int s = 0; s < P; ++s) {
                const double e = (f[s] - Fn[s]) / (atol + rtol * fabs(yn[s]));
                sq[s] = e * e;
            }
            const double est = h * sqrt(sys.ordered_sum(tm, sq) / (double)n);
            if (kP1 * h < hmax * sqrt(est))
                h = fmax(kP1 * h / sqrt(est), hmin);
            else
                h = hmax;
        }
        int m = 1 + (int)sqrt(1.54 * h * sigma + 1.0);
        if (m > mmax) {
            m = mmax;
            h = (double)(m * m - 1) / (1.54 * sigma);
        }

        // stages, Eqs. E:rkc0-E:rkcs
        CoefSource cs;
        cs.start(m, a);
        const double mut1 = cs.mut1();
#pragma unroll
        for (int s = 0; s < P; ++s) {
            w2[s] = yn[s];
            w1v[s] = yn[s] + mut1 * h * Fn[s];
        }
        for (int j = 2; j <= m; ++j) {
            const StageCoef c = cs.stage64(j);
            sys.rhs(tm, t + c.cprev * h, w1v, f);
#pragma unroll
            for (int s = 0; s < P; ++s) {
                const double wj = c.cy * yn[s] + c.mu * w1v[s] + c.nu * w2[s] + c.mut * h * f[s] + c.gt * h * Fn[s];
                w2[s] = w1v[s];
                w1v[s] = wj;
            }
        }
        sys.rhs(tm, t + h, w1v, f);  // F_{n+1}
        n_rhs += m;

        double sq[P];
#pragma unroll
        for (int s = 0; s < P; ++s) {
            double e = 0.8 * (yn[s] - w1v[s]) + 0.4 * h * (Fn[s] + f[s]);
            e = e / (atol + rtol * fmax(fabs(w1v[s]), fabs(yn[s])));
            sq[s] = e * e;
        }
        const double err = sqrt(sys.ordered_sum(tm, sq) / (double)n);
        if (isnan(err)) {
            n_rej += 1;
            status |= ODE_ST_NONFINITE;
            return true;
        }
        if (err > 1.0) {
            n_rej += 1;
            h = 0.8 * h / xm::pow_series(err, 1.0 / 3.0);
            rejected = true;
            if (h < hmin) {
                status |= ODE_ST_H_UNDERFLOW;
                return true;
            }
            return false;
        }
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
#pragma unroll
        for (int s = 0; s < P; ++s) {
            yn[s] = w1v[s];
            Fn[s] = f[s];
            if (comp[s] >= 0 && !isfinite(w1v[s])) bad = true;
        }
        h = h * fmax(kP1, fac);
        h = fmax(hmin, fmin(hmax, h));
        if (tm.any(bad)) {
            status |= ODE_ST_NONFINITE;
            return true;
        }
        return !(t < tend);
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (comp[s] >= 0) a.y_out[i + a.nsys * (int64_t)comp[s]] = yn[s];
        if (tm.lane == 0) {
            if (a.n_accept) a.n_accept[i] = n_acc;
            if (a.n_reject) a.n_reject[i] = n_rej;
            if (a.n_rhs) a.n_rhs[i] = n_rhs + n_sr;
            if (a.n_specrad) a.n_specrad[i] = n_sr;
            if (a.status) a.status[i] = status;
        }
    }
};

// ============================================================ mixed helpers

// Kahan-compensated state update (hi, lo) += d.
__device__ __forceinline__ void kahan_add(float& hi, float& lo, float d) {
    const float y = d + lo;
    const float t = hi + y;
    lo = y - (t - hi);
    hi = t;
}

// ============================================================== RKCK mixed

template <class Model>
struct RkckMixed {
    static constexpr int W = Model::W, P = Model::PER;
    using TM = Team<W>;
    typename Model::template Sys<float> sys;
    float yh[P], yl[P];
    int comp[P];
    double t, tend, h, hmax;
    float deltaf, inv_rtolf;
    int32_t n_acc, n_rej, status, max_att;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq);
#pragma unroll
        for (int s = 0; s < P; ++s) {
            comp[s] = sys.comp(tm, s);
            const double y0 = comp[s] >= 0 ? a.y0[i + a.nsys * (int64_t)comp[s]] : 0.0;
            yh[s] = (float)y0;
            yl[s] = (float)(y0 - (double)yh[s]);
        }
        t = a.t0;
        tend = a.tend;
        hmax = fabs(tend - t);
        h = 0.5 * fabs(tend - t);
        deltaf = (float)((a.atol > 0.0) ? a.atol / a.rtol : kTiny);
        inv_rtolf = (float)(1.0 / a.rtol);
        n_acc = n_rej = status = 0;
        max_att = a.max_attempts;
    }

    __device__ bool attempt(const BatchArgs&, const TM& tm) {
        if (!(t < tend)) return true;
        if (n_acc + n_rej >= max_att) {
            status = ODE_ST_MAX_ATTEMPTS;
            return true;
        }
        h = fmin(tend - t, h);
        const float hf = (float)h;
        const float tf = (float)t;
        float F[P], k1[P], k2[P], k3[P], k4[P], k5[P], yt[P], f[P];
        sys.rhs(tm, tf, yh, F);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k1[i] = hf * F[i];
            yt[i] = yh[i] + (float)ck::B21 * k1[i];
        }
        sys.rhs(tm, tf, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k2[i] = hf * f[i];
            yt[i] = yh[i] + ((float)ck::B31 * k1[i] + (float)ck::B32 * k2[i]);
        }
        sys.rhs(tm, tf, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k3[i] = hf * f[i];
            yt[i] = yh[i] + ((float)ck::B41 * k1[i] + (float)ck::B42 * k2[i] + (float)ck::B43 * k3[i]);
        }
        sys.rhs(tm, tf, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k4[i] = hf * f[i];
            yt[i] = yh[i] + ((float)ck::B51 * k1[i] + (float)ck::B52 * k2[i] + (float)ck::B53 * k3[i] +
                             (float)ck::B54 * k4[i]);
        }
        sys.rhs(tm, tf, yt, f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            k5[i] = hf * f[i];
            yt[i] = yh[i] + ((float)ck::B61 * k1[i] + (float)ck::B62 * k2[i] + (float)ck::B63 * k3[i] +
                             (float)ck::B64 * k4[i] + (float)ck::B65 * k5[i]);
        }
        sys.rhs(tm, tf, yt, f);
        float err = 0.0f;
        bool nan_flag = false;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const float k6 = hf * f[i];
            yt[i] = (float)ck::C1 * k1[i] + (float)ck::C3 * k3[i] + (float)ck::C4 * k4[i] + (float)ck::C6 * k6;
            const float ye = (float)ck::DC1 * k1[i] + (float)ck::DC3 * k3[i] + (float)ck::DC4 * k4[i] +
                             (float)ck::DC5 * k5[i] + (float)ck::DC6 * k6;
            if (comp[i] >= 0) {
                if (isnan(ye) || isnan(yt[i])) nan_flag = true;
                err = fmaxf(err, fabsf(ye) / (fabsf(yh[i]) + fabsf(hf * F[i]) + deltaf));
            }
        }
        err = tm.max(err) * inv_rtolf;
        nan_flag = tm.any(nan_flag);
        if (err > 1.0f || isnan(err) || nan_flag) {
            n_rej += 1;
            if (isnan(err) || nan_flag)
                h = h * kP1;
            else
                h = h * (double)fmaxf((float)kSafety * powf(err, (float)kPshrnk), (float)kP1);
            if (h < 1.0e-20 || t + h == t) {
                status = ODE_ST_H_UNDERFLOW;
                return true;
            }
            return false;
        }
        n_acc += 1;
        t = t + h;
        const float fac = (err > (float)kErrcon) ? (float)kSafety * powf(err, (float)kPgrow) : 5.0f;
        h = fmax(1.0e-20, fmin(hmax, h * (double)fac));
        bool bad = false;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            kahan_add(yh[i], yl[i], yt[i]);
            if (comp[i] >= 0 && !isfinite(yh[i])) bad = true;
        }
        if (tm.any(bad)) {
            status = ODE_ST_NONFINITE;
            return true;
        }
        return !(t < tend);
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (comp[s] >= 0) a.y_out[i + a.nsys * (int64_t)comp[s]] = (double)yh[s] + (double)yl[s];
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

template <class Model>
struct RkcMixed {
    static constexpr int W = Model::W, P = Model::PER;
    using TM = Team<W>;
    typename Model::template Sys<float> sys;
    float yh[P], yl[P], Fn[P], v[P];
    int comp[P];
    double t, tend, hmax, hmin, h, h_old, sigma, inv_n;
    float rtolf, atolf, err_old;
    int32_t n_acc, n_rej, n_rhs, n_sr, status, max_att, mmax, num_step, sr_step, n;
    bool have_sigma, rejected;

    __device__ void init(const BatchArgs& a, const typename Model::Ctx& ctx, const TM& tm, int64_t i) {
        sys.load(ctx, tm, a.params[i], a.neq);
        n = a.neq;
        inv_n = 1.0 / (double)n;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            comp[s] = sys.comp(tm, s);
            const double y0 = comp[s] >= 0 ? a.y0[i + a.nsys * (int64_t)comp[s]] : 0.0;
            yh[s] = (float)y0;
            yl[s] = (float)(y0 - (double)yh[s]);
        }
        t = a.t0;
        tend = a.tend;
        rtolf = (float)a.rtol;
        atolf = (float)a.atol;
        mmax = (int)round(sqrt(a.rtol / (10.0 * kUround)));
        if (mmax < 2) mmax = 2;
        hmax = fabs(tend - t);
        hmin = 10.0 * kUround * fmax(fabs(t), hmax);
        sys.rhs(tm, (float)t, yh, Fn);
#pragma unroll
        for (int s = 0; s < P; ++s) v[s] = Fn[s];
        n_acc = n_rej = n_sr = status = 0;
        n_rhs = 1;
        max_att = a.max_attempts;
        h = h_old = sigma = 0.0;
        err_old = 0.0f;
        num_step = 0;
        sr_step = -1;
        have_sigma = rejected = false;
    }

    __device__ float sumsq(const TM& tm, const float* x) const {
        float acc = 0.0f;
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (comp[s] >= 0) acc = acc + x[s] * x[s];
        return tm.sum(acc);
    }

    // Nonlinear power method (Appendix) in FP32 with an FP32-scaled
    // perturbation; v persists as a difference from the state.
    __device__ double specrad(const TM& tm) {
        const float small = (float)(1.0 / hmax);
        const float nrm1 = sqrtf(sumsq(tm, yh)), nrm2 = sqrtf(sumsq(tm, v));
        float dynrm;
        if (nrm1 != 0.0f && nrm2 != 0.0f) {
            dynrm = nrm1 * kSqrtUroundF;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = yh[s] + v[s] * (dynrm / nrm2);
        } else if (nrm1 != 0.0f) {
            dynrm = nrm1 * kSqrtUroundF;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = yh[s] * (1.0f + kSqrtUroundF);
        } else if (nrm2 != 0.0f) {
            dynrm = kSqrtUroundF;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = v[s] * (dynrm / nrm2);
        } else {
            dynrm = kSqrtUroundF;
#pragma unroll
            for (int s = 0; s < P; ++s) v[s] = kSqrtUroundF;
        }
        float sig = 0.0f;
        for (int iter = 1; iter <= kSpecradItmax; ++iter) {
            float Fv[P];
            sys.rhs(tm, (float)t, v, Fv);
            n_sr += 1;
            float acc = 0.0f;
#pragma unroll
            for (int s = 0; s < P; ++s)
                if (comp[s] >= 0) acc = acc + (Fv[s] - Fn[s]) * (Fv[s] - Fn[s]);
            const float d = sqrtf(tm.sum(acc));
            const float sig_prev = sig;
            sig = d / dynrm;
            if (iter >= 2 && fabsf(sig - sig_prev) <= fmaxf(sig, small) * 0.01f) {
#pragma unroll
                for (int s = 0; s < P; ++s) v[s] = v[s] - yh[s];
                return 1.2 * (double)sig;
            }
            if (d != 0.0f) {
                const float sc = dynrm / d;
#pragma unroll
                for (int s = 0; s < P; ++s) v[s] = yh[s] + (Fv[s] - Fn[s]) * sc;
            } else {
                const int ind = iter % n;
#pragma unroll
                for (int s = 0; s < P; ++s)
                    if (comp[s] == ind) v[s] = yh[s] - (v[s] - yh[s]);
            }
        }
#pragma unroll
        for (int s = 0; s < P; ++s) v[s] = v[s] - yh[s];
        status |= ODE_ST_SPECRAD_NOCONV;
        return 1.2 * (double)sig;
    }

    __device__ bool attempt(const BatchArgs& a, const TM& tm) {
        if (!(t < tend)) return true;
        if (n_acc + n_rej >= max_att) {
            status |= ODE_ST_MAX_ATTEMPTS;
            return true;
        }
        if (1.1 * h >= fabs(tend - t)) h = fabs(tend - t);
        if (!have_sigma || rejected || (num_step % kSpecradEvery == 0 && sr_step != num_step)) {
            sigma = specrad(tm);
            have_sigma = true;
            sr_step = num_step;
        }
        const float tf = (float)t;
        float d1[P], d2[P], f[P];
        if (h < kUround) {
            // initial step: trial Euler step of size 1/sigma
            h = hmax;
            if (sigma * h > 1.0) h = 1.0 / sigma;
            h = fmax(h, hmin);
            const float hf = (float)h;
#pragma unroll
            for (int s = 0; s < P; ++s) d1[s] = yh[s] + hf * Fn[s];
            sys.rhs(tm, tf, d1, f);
            n_rhs += 1;
            double acc = 0.0;
#pragma unroll
            for (int s = 0; s < P; ++s)
                if (comp[s] >= 0) {
                    const float e = (f[s] - Fn[s]) / (atolf + rtolf * fabsf(yh[s]));
                    acc = fma((double)e, (double)e, acc);
                }
            const double est = h * sqrt(tm.sum(acc) * inv_n);
            if (kP1 * h < hmax * sqrt(est))
                h = fmax(kP1 * h / sqrt(est), hmin);
            else
                h = hmax;
        }
        int m = 1 + (int)sqrtf((float)(1.54 * h * sigma) + 1.0f);
        if (m > mmax) {
            m = mmax;
            h = (double)(m * m - 1) / (1.54 * sigma);
        }
        const float hf = (float)h;

        // stages as differences d_j = w_j - y_n (d_0 = 0), Eqs. E:rkc0-E:rkcs
        CoefSource cs;
        cs.start(m, a);
        const float mut1h = (float)cs.mut1() * hf;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            d2[s] = 0.0f;
            d1[s] = mut1h * Fn[s];
        }
        for (int j = 2; j <= m; ++j) {
            const float4 c = cs.stage32(j);
            float wv[P];
#pragma unroll
            for (int s = 0; s < P; ++s) wv[s] = yh[s] + (yl[s] + d1[s]);
            sys.rhs(tm, tf, wv, f);
            const float muth = c.z * hf, gth = c.w * hf;
#pragma unroll
            for (int s = 0; s < P; ++s) {
                const float dj = c.x * d1[s] + c.y * d2[s] + muth * f[s] + gth * Fn[s];
                d2[s] = d1[s];
                d1[s] = dj;
            }
        }
        float wm[P];
#pragma unroll
        for (int s = 0; s < P; ++s) wm[s] = yh[s] + (yl[s] + d1[s]);
        sys.rhs(tm, tf, wm, f);  // F_{n+1}
        n_rhs += m;

        // weighted RMS error, accumulated in FP64
        const float h04 = 0.4f * hf;
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (comp[s] >= 0) {
                const float e = (-0.8f * d1[s] + h04 * (Fn[s] + f[s])) / (atolf + rtolf * fmaxf(fabsf(wm[s]), fabsf(yh[s])));
                acc = fma((double)e, (double)e, acc);
            }
        const double ms = tm.sum(acc) * inv_n;  // err^2
        if (isnan(ms)) {
            n_rej += 1;
            status |= ODE_ST_NONFINITE;
            return true;
        }
        const float err = sqrtf((float)ms);
        if (ms > 1.0) {
            n_rej += 1;
            h = h * (double)(0.8f / cbrtf(err));
            rejected = true;
            if (h < hmin) {
                status |= ODE_ST_H_UNDERFLOW;
                return true;
            }
            return false;
        }
        n_acc += 1;
        rejected = false;
        num_step += 1;
        float fac = 10.0f;
        const float c3 = cbrtf(err);
        if (h_old < kUround) {
            if (0.8f < fac * c3) fac = 0.8f / c3;
        } else {
            const float temp1 = 0.8f * hf * cbrtf(err_old);
            const float temp2 = (float)h_old * (c3 * c3);
            if (temp1 < fac * temp2) fac = temp1 / temp2;
        }
        err_old = err;
        h_old = h;
        t = t + h;
        bool bad = false;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            kahan_add(yh[s], yl[s], d1[s]);
            Fn[s] = f[s];
            if (comp[s] >= 0 && !isfinite(yh[s])) bad = true;
        }
        h = h * (double)fmaxf((float)kP1, fac);
        h = fmax(hmin, fmin(hmax, h));
        if (tm.any(bad)) {
            status |= ODE_ST_NONFINITE;
            return true;
        }
        return !(t < tend);
    }

    __device__ void store(const BatchArgs& a, const TM& tm, int64_t i) const {
#pragma unroll
        for (int s = 0; s < P; ++s)
            if (comp[s] >= 0) a.y_out[i + a.nsys * (int64_t)comp[s]] = (double)yh[s] + (double)yl[s];
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
