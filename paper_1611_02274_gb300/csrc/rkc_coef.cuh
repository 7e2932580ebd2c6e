// rkc_coef.cuh -- Cash-Karp tableau and RKC stage coefficients.
#pragma once
#include <cmath>

#include "common.cuh"
#include "f2.cuh"

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

// Coefficients from the precomputed table when m is in range; beyond it,
// each stage's coefficients are recomputed from the start of the recurrence
// (the same arithmetic that built the table, so the values are identical;
// O(m) work per stage, which only stage counts above the table pay).
struct CoefSource {
    const double* e64;
    const float4* e32;
    int m;
    __device__ void start(int m_, const BatchArgs& a) {
        m = m_;
        if (m <= a.rkc_tab_max && a.rkc_tab64 != nullptr) {
            const int base = rkc_tab_index(m, 1);
            e64 = a.rkc_tab64 + 8 * base;
            e32 = a.rkc_tab32 + base;
        } else {
            e64 = nullptr;
            e32 = nullptr;
        }
    }
    __device__ double mut1() const {
        if (e64) return __ldg(e64 + 3);
        RkcStageGen g;
        g.start(m);
        return g.mut1;
    }
    __device__ float mut1f() const {
        if (e32) return __ldg(e32).z;
        RkcStageGen g;
        g.start(m);
        return (float)g.mut1;
    }
    __device__ StageCoef recompute(int j) const {
        RkcStageGen g;
        g.start(m);
        StageCoef s = g.next();
        for (int k = 3; k <= j; ++k) s = g.next();
        return s;
    }
    __device__ StageCoef stage64(int j) const {
        if (e64) {
            const double2* p = reinterpret_cast<const double2*>(e64 + 8 * (j - 1));
            const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
            return StageCoef{a.x, a.y, b.x, b.y, c.x, c.y};
        }
        return recompute(j);
    }
    // two-float mu~_1 and stage coefficients: leading words from the FP32
    // table, trailing words from the FP64 entry's last 16 bytes
    __device__ F2 mut1f2() const {
        if (e32) return F2(__ldg(e32).z, __ldg(reinterpret_cast<const float4*>(e64 + 6)).z);
        RkcStageGen g;
        g.start(m);
        return F2(g.mut1);
    }
    __device__ void stagef2(int j, float4& hi, float4& lo) const {
        if (e32) {
            hi = __ldg(e32 + (j - 1));
            lo = __ldg(reinterpret_cast<const float4*>(e64 + 8 * (j - 1) + 6));
            return;
        }
        const StageCoef s = recompute(j);
        const F2 mu(s.mu), nu(s.nu), mut(s.mut), gt(s.gt);
        hi = make_float4(mu.hi, nu.hi, mut.hi, gt.hi);
        lo = make_float4(mu.lo, nu.lo, mut.lo, gt.lo);
    }
    __device__ float4 stage32(int j) const {
        if (e32) return __ldg(e32 + (j - 1));
        const StageCoef s = recompute(j);
        return make_float4((float)s.mu, (float)s.nu, (float)s.mut, (float)s.gt);
    }
};

// Builds the coefficient table for m = 2..mmax (one thread per m).
__global__ void k_build_rkc_table(double* tab64, float4* tab32, int mmax);

}  // namespace bode
