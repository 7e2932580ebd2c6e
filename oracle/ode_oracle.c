/*
 * ode_oracle.c -- CPU FP64 oracle for batched RKCK / RKC integration.
 *
 * TEST INFRASTRUCTURE.  This is a plain, slow, obviously sequential
 * restatement of the paper's two integrators (Niemeyer & Sung, "GPU-Based
 * Parallel Integration of Large Numbers of Independent ODE Systems"):
 *   - RKCK: Section 2.1 (Table 1, the k1..k6 / y / y* equations, the error
 *     scale and the step-size rule Eq. E:hnew) with the control flow of the
 *     rkckDriver listing in Section 3.1;
 *   - RKC: Section 2.2 (Eqs. E:rkc0-E:rkcs, the coefficient formulas, the
 *     RMS error norm Eq. E:rmsE, Eqs. dtnp1 / rkc-f, the initial step and
 *     the stage count) with the control flow of the rkcDriver listing in
 *     Section 3.2 and the nonlinear power method of the Appendix.
 * Only tests, the package smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code with the CUDA library; the two meet only
 * through the seeded inputs.  Compiled with -O2 -ffp-contract=off: every
 * expression is evaluated as written, left to right, without fused
 * multiply-adds.
 *
 * Readings of the paper where it is silent or garbled (each also listed in
 * the design notes):
 *   R1  P1 (used, never defined) = 0.1: step decreases are limited to a
 *       factor of ten (Section 2.1, last paragraph).
 *   R2  RKCK with separate rtol/atol: delta = atol/rtol (TINY if atol == 0)
 *       and err = max_i |D_i| / (|y_i| + |h F_i| + delta) / rtol, which is
 *       the listing's test exactly when atol = 0.
 *   R3  RKC b_1 = b_2 (= b_0): forced by c_1 = c_2 / T_2'(w0) together with
 *       mu~_1 = b_1 w1 and c_1 = mu~_1.
 *   R4  Spectral radius is computed once per need: when no estimate exists,
 *       after a rejected step, or when the accepted-step count is a
 *       multiple of 25 and no estimate was made at that count yet.
 *   R5  Power-method convergence: |sigma - sigma_prev| <= 0.01 max(sigma,
 *       1/hmax) from the second iteration; on non-convergence after 50
 *       iterations the eigenvector is still re-centred (v -= y) and the
 *       SPECRAD_NOCONV status bit is set.
 *   R6  RKC reject factor follows the listing: h = 0.8 h / err^(1/3) with no
 *       clamp; h < hmin afterwards ends the system with H_UNDERFLOW.
 *   R7  Stage times use the recurrence that makes the scheme exact for
 *       y' = 1: c_1 = mu~_1, c_j = mu_j c_{j-1} + nu_j c_{j-2}
 *       + mu~_j (1 - a_{j-1}).
 *   R8  Guards the listings lack: a per-system attempt cap (MAX_ATTEMPTS),
 *       RKCK h < 1e-20 or t + h == t (H_UNDERFLOW), a NaN RKC error or a
 *       non-finite accepted state (NONFINITE).
 *   R9  UROUND is the literal 2.22e-16 of the listings.
 *   R10 Powers in the step-size rules and the Arrhenius rate use the series
 *       logarithm / exponential below, a fixed sequence of correctly
 *       rounded operations, so their values are reproducible bit for bit.
 *       Compiled with -DORACLE_LIBM the C library's log / exp / pow are
 *       used instead (a build that tests compare with this one).
 *   R21 Warm restart (the outer global-step loop of Section 3, where the
 *       paper notes that carrying step information from one global step to
 *       the next could help but restarts every call): an optional carry
 *       state per system, CARRY_WORDS(neq) doubles -- valid flag, time
 *       reached, h (the controller's next step), sigma, h_old, err_old,
 *       accepted-step count, count at the last spectral-radius estimate,
 *       rejected flag, eigenvector v (RKC; RKCK uses the flag, time and h).
 *       A call given a valid carry resumes the step-size controller and the
 *       25-step spectral-radius schedule where the previous call left
 *       them, instead of the power method and the trial step; F(t0, y0) is
 *       evaluated again.  The carry is written when the system ends, valid
 *       unless the state is unusable (H_UNDERFLOW, NONFINITE).  A run
 *       stopped by the attempt cap and continued this way repeats the
 *       uninterrupted run step for step, wherever the per-call quantities
 *       hmax = |tend - t0| and hmin do not bind.  Carry mode RESTART keeps
 *       the controller (h, h_old, err_old) and the eigenvector but restarts
 *       the spectral-radius schedule: sigma is estimated at the first loop
 *       top (from the carried eigenvector) and the 25-step count starts
 *       again, i.e. the carry is read with num_step = 0, sr_step = -1 and
 *       no rejection pending.
 *   R23 Gershgorin bound (the Appendix names the circle theorem as an
 *       upper-bound alternative to the power method): every eigenvalue of
 *       the Jacobian J lies in a disc centred at J_ii of radius
 *       sum_{j != i} |J_ij|, so sigma <= G = max_i sum_j |J_ij|.  J is the
 *       analytic Jacobian of each right-hand side below; each row sum runs
 *       over the columns in increasing order.  Spectral-radius modes:
 *       POWER (the Appendix method), GERSHGORIN (sigma = G at every point
 *       the power method would run, no right-hand-side evaluations),
 *       POWER_CAPPED (the power method's 1.2 sigma, capped at G).
 *   R26 Jacobian of a clipped rate constant (the kinetics family bounds
 *       k_j to [kmin, kmax]; the paper's mechanism has no such bound): the
 *       clipped value does not vary with T, so dk_j/dT = 0 wherever the
 *       unclipped value lies outside the open interval (kmin, kmax),
 *       including exactly at a bound.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define UROUND 2.22e-16
#define SAFETY 0.9
#define PGROW (-0.2)
#define PSHRNK (-0.25)
#define ERRCON 1.89e-4
#define TINY 1.0e-30
#define P1 0.1

#define ST_OK 0
#define ST_H_UNDERFLOW 1
#define ST_MAX_ATTEMPTS 2
#define ST_NONFINITE 3
#define ST_SPECRAD_NOCONV 256

#define KIND_VDP 1
#define KIND_VDP_CHAIN 2
#define KIND_BRUSS1D 3
#define KIND_MASSACTION 4
#define KIND_NBODY 5
#define KIND_KINETICS 6
#define R_GAS 8.314462618
#define KIND_LINEAR 100    /* f = A y, A row-major in the params (tests only) */
#define KIND_TIME 101      /* f_i = t (tests of the stage times only) */

#define CARRY_FIXED 9
#define CARRY_CONTINUE 0
#define CARRY_RESTART 1
#define SPECRAD_POWER 0
#define SPECRAD_GERSHGORIN 1
#define SPECRAD_POWER_CAPPED 2
#define CARRY_WORDS(neq) (CARRY_FIXED + (neq))

#define OR_MAX_REAC 64
#define OR_MAX_BODIES 16
#define OR_MAX_PARAMS 300

/* A constant-volume gas mechanism (KIND_KINETICS): molecular weights,
 * polynomial thermodynamics (cp/R = a0 + a1 T + a2 T^2, h/(R T) = a0
 * + a1 T / 2 + a2 T^2 / 3 + a3 / T) and irreversible reactions. */
typedef struct {
    int32_t n_species, n_reactions;
    const double* W;        /* [S] kg/mol */
    const double* thermo;   /* [S][4] */
    const int32_t* n_reac;  /* [R] */
    const int32_t* reac;    /* [R][2] */
    const int32_t* n_prod;
    const int32_t* prod;
    const double* log10A;   /* [R] */
    const double* beta;
    const double* Ea;       /* Kelvin */
    double kmin, kmax;
} or_mech;

typedef struct {
    int32_t kind;
    int32_t neq;
    int32_t n_params;
    int32_t n_species;
    int32_t n_reactions;
    int32_t n_reac[OR_MAX_REAC];
    int32_t reac[OR_MAX_REAC][2];
    int32_t n_prod[OR_MAX_REAC];
    int32_t prod[OR_MAX_REAC][2];
    double log10A[OR_MAX_REAC];
    double beta[OR_MAX_REAC];
    double Ea[OR_MAX_REAC];
    double kmin, kmax;
    double bruss_A, bruss_B, bruss_ubc, bruss_vbc;
    double coupling;
    double masses[OR_MAX_BODIES];
    const or_mech* mech;  /* KIND_KINETICS */
} or_model;

/* One system: the model, its dimension, its parameters and (mass-action)
 * its rate constants. */
typedef struct {
    const or_model* m;
    int neq;
    double p[OR_MAX_PARAMS];
    double k[OR_MAX_REAC];
} or_sys;

/* ------------------------------------------------------------------ RHS */

/* van der Pol: y1' = y2, y2' = mu (1 - y1^2) y2 - y1. */
static void rhs_vdp(const or_sys* s, const double* y, double* f) {
    double mu = s->p[0];
    f[0] = y[1];
    f[1] = mu * (1.0 - y[0] * y[0]) * y[1] - y[0];
}

/* Chain of n van der Pol oscillators, state [x_1..x_n, v_1..v_n], coupled
 * diffusively through positions with free ends. */
static void rhs_vdp_chain(const or_sys* s, const double* y, double* f) {
    int n = s->neq / 2;
    double mu = s->p[0];
    double c = s->m->coupling;
    const double* x = y;
    const double* v = y + n;
    for (int i = 0; i < n; ++i) {
        double coup = 0.0;
        if (i > 0) coup = coup + (x[i - 1] - x[i]);
        if (i < n - 1) coup = coup + (x[i + 1] - x[i]);
        f[i] = v[i];
        f[n + i] = mu * (1.0 - x[i] * x[i]) * v[i] - x[i] + c * coup;
    }
}

/* 1D Brusselator on n interior points x_k = k/(n+1), state
 * [u_1..u_n, v_1..v_n], Dirichlet ghost values u = ubc, v = vbc. */
static void rhs_bruss(const or_sys* s, const double* y, double* f) {
    int n = s->neq / 2;
    const or_model* m = s->m;
    double a = s->p[0];
    double dx = 1.0 / (double)(n + 1);
    double D = a / (dx * dx);
    const double* u = y;
    const double* v = y + n;
    for (int k = 0; k < n; ++k) {
        double ul = (k > 0) ? u[k - 1] : m->bruss_ubc;
        double ur = (k < n - 1) ? u[k + 1] : m->bruss_ubc;
        double vl = (k > 0) ? v[k - 1] : m->bruss_vbc;
        double vr = (k < n - 1) ? v[k + 1] : m->bruss_vbc;
        double uuv = u[k] * u[k] * v[k];
        f[k] = m->bruss_A + uuv - (m->bruss_B + 1.0) * u[k] + D * (ul - 2.0 * u[k] + ur);
        f[n + k] = m->bruss_B * u[k] - uuv + D * (vl - 2.0 * v[k] + vr);
    }
}

/* Mass-action kinetics (the omega_i sum of Section 4.2 with constant T):
 * r_j = k_j prod_{reactants} C, C_s' = sum_j (nu''_sj - nu'_sj) r_j,
 * accumulated over reactions in order, reactants then products. */
static void rhs_massaction(const or_sys* s, const double* y, double* f) {
    const or_model* m = s->m;
    for (int i = 0; i < s->neq; ++i) f[i] = 0.0;
    for (int j = 0; j < m->n_reactions; ++j) {
        double r = s->k[j];
        for (int q = 0; q < m->n_reac[j]; ++q) r = r * y[m->reac[j][q]];
        for (int q = 0; q < m->n_reac[j]; ++q) f[m->reac[j][q]] -= r;
        for (int q = 0; q < m->n_prod[j]; ++q) f[m->prod[j][q]] += r;
    }
}

/* Planar n-body gravity (the form of the Pleiades problem, Section 4.1),
 * state [x_1..x_n, y_1..y_n, u_1..u_n, v_1..v_n], masses from the model,
 * gravitational constant G the system's parameter:
 * x_i' = u_i, y_i' = v_i, (u_i', v_i') = G sum_{j != i} m_j d_ij / r_ij^3,
 * d_ij = (x_j - x_i, y_j - y_i), r_ij^3 = r2 sqrt(r2), j ascending. */
static void rhs_nbody(const or_sys* s, const double* y, double* f) {
    int n = s->neq / 4;
    double G = s->p[0];
    const double* x = y;
    const double* yy = y + n;
    for (int i = 0; i < n; ++i) {
        f[i] = y[2 * n + i];
        f[n + i] = y[3 * n + i];
    }
    for (int i = 0; i < n; ++i) {
        double ax = 0.0, ay = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[j] - x[i];
            double dy = yy[j] - yy[i];
            double r2 = dx * dx + dy * dy;
            double r3 = r2 * sqrt(r2);
            ax = ax + s->m->masses[j] * dx / r3;
            ay = ay + s->m->masses[j] * dy / r3;
        }
        f[2 * n + i] = G * ax;
        f[3 * n + i] = G * ay;
    }
}

/* Constant-volume kinetics (Section 4.2), state (T, Y_1..Y_S), density
 * rho the system's parameter:
 *   C_i = rho Y_i / W_i,  k_j = clip(A_j T^beta_j exp(-Ea_j / T)),
 *   q_j = k_j prod_{reactants} C,  omega_i = sum_j (nu''_ij - nu'_ij) q_j
 *   (reaction by reaction, reactants then products),
 *   dY_i/dt = W_i omega_i / rho,
 *   dT/dt = -(sum_i e_i omega_i W_i) / (rho c_v),  c_v = sum_i Y_i c_v,i,
 *   c_v,i = (R / W_i)(cp_i/R - 1),  e_i = (R T / W_i)(h_i/(R T) - 1),
 * species sums in species order. */
static double or_exp(double x);
static double or_log(double x);

static double kin_rate(const or_mech* k, int j, double T, double lnT) {
    const double ln10 = 2.302585092994046;
    double kk = or_exp(ln10 * k->log10A[j] + k->beta[j] * lnT - k->Ea[j] / T);
    return fmin(fmax(kk, k->kmin), k->kmax);
}

static void rhs_kinetics(const or_sys* s, const double* y, double* f) {
    const or_mech* k = s->m->mech;
    int S = k->n_species;
    double rho = s->p[0];
    double T = y[0];
    const double* Y = y + 1;
    double* om = f + 1;
    double lnT = or_log(T);
    for (int i = 0; i < S; ++i) om[i] = 0.0;
    for (int j = 0; j < k->n_reactions; ++j) {
        double q = kin_rate(k, j, T, lnT);
        for (int r = 0; r < k->n_reac[j]; ++r) {
            int i = k->reac[2 * j + r];
            q = q * (rho * Y[i] / k->W[i]);
        }
        for (int r = 0; r < k->n_reac[j]; ++r) om[k->reac[2 * j + r]] -= q;
        for (int r = 0; r < k->n_prod[j]; ++r) om[k->prod[2 * j + r]] += q;
    }
    double cv = 0.0, heat = 0.0;
    for (int i = 0; i < S; ++i) {
        const double* a = k->thermo + 4 * i;
        double cvi = (R_GAS / k->W[i]) * (a[0] + a[1] * T + a[2] * T * T - 1.0);
        double ei = (R_GAS * T / k->W[i]) * (a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] / T - 1.0);
        cv = cv + Y[i] * cvi;
        heat = heat + ei * om[i] * k->W[i];
    }
    f[0] = -heat / (rho * cv);
    for (int i = 0; i < S; ++i) om[i] = k->W[i] * om[i] / rho;
}

static void rhs_linear(const or_sys* s, const double* y, double* f) {
    int n = s->neq;
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = acc + s->p[i * n + j] * y[j];
        f[i] = acc;
    }
}

/* ------------------------------------------------------------ Jacobians
 * Analytic df/dy, row-major n x n (R23).  Each entry is written as the
 * derivative of the expression above it, term by term. */

static void jac_vdp(const or_sys* s, const double* y, double* J) {
    double mu = s->p[0];
    J[0] = 0.0;
    J[1] = 1.0;
    J[2] = mu * (-2.0 * y[0]) * y[1] - 1.0;
    J[3] = mu * (1.0 - y[0] * y[0]);
}

static void jac_vdp_chain(const or_sys* s, const double* y, double* J) {
    int n = s->neq / 2, N = s->neq;
    double mu = s->p[0];
    double c = s->m->coupling;
    const double* x = y;
    const double* v = y + n;
    for (int k = 0; k < N * N; ++k) J[k] = 0.0;
    for (int i = 0; i < n; ++i) {
        double nb = (double)((i > 0) + (i < n - 1));
        J[i * N + (n + i)] = 1.0;                                   /* dx_i'/dv_i */
        double* row = J + (n + i) * N;
        row[i] = mu * (-2.0 * x[i]) * v[i] - 1.0 - c * nb;          /* dv_i'/dx_i */
        if (i > 0) row[i - 1] = c;
        if (i < n - 1) row[i + 1] = c;
        row[n + i] = mu * (1.0 - x[i] * x[i]);                      /* dv_i'/dv_i */
    }
}

static void jac_bruss(const or_sys* s, const double* y, double* J) {
    int n = s->neq / 2, N = s->neq;
    const or_model* m = s->m;
    double a = s->p[0];
    double dx = 1.0 / (double)(n + 1);
    double D = a / (dx * dx);
    const double* u = y;
    const double* v = y + n;
    for (int k = 0; k < N * N; ++k) J[k] = 0.0;
    for (int k = 0; k < n; ++k) {
        double* ru = J + k * N;
        double* rv = J + (n + k) * N;
        ru[k] = 2.0 * u[k] * v[k] - (m->bruss_B + 1.0) - 2.0 * D;  /* du'/du */
        ru[n + k] = u[k] * u[k];                                    /* du'/dv */
        rv[k] = m->bruss_B - 2.0 * u[k] * v[k];                     /* dv'/du */
        rv[n + k] = -(u[k] * u[k]) - 2.0 * D;                       /* dv'/dv */
        if (k > 0) {
            ru[k - 1] = D;
            rv[n + k - 1] = D;
        }
        if (k < n - 1) {
            ru[k + 1] = D;
            rv[n + k + 1] = D;
        }
    }
}

/* dr_j/dC_l summed over the reactant occurrences of species l; the rows of
 * the reaction's reactants lose it and its products' rows gain it, reaction
 * by reaction, reactants before products. */
static void jac_massaction(const or_sys* s, const double* y, double* J) {
    const or_model* m = s->m;
    int N = s->neq;
    for (int k = 0; k < N * N; ++k) J[k] = 0.0;
    for (int j = 0; j < m->n_reactions; ++j) {
        int nr = m->n_reac[j];
        double d[2];
        for (int q = 0; q < nr; ++q) {  /* d[q]: derivative by the q-th reactant occurrence */
            double t = s->k[j];
            for (int o = 0; o < nr; ++o)
                if (o != q) t = t * y[m->reac[j][o]];
            d[q] = t;
        }
        for (int l = 0; l < N; ++l) {
            double dl = 0.0;
            int any = 0;
            for (int q = 0; q < nr; ++q)
                if (m->reac[j][q] == l) {
                    dl = dl + d[q];
                    any = 1;
                }
            if (!any) continue;
            for (int q = 0; q < nr; ++q) J[m->reac[j][q] * N + l] -= dl;
            for (int q = 0; q < m->n_prod[j]; ++q) J[m->prod[j][q] * N + l] += dl;
        }
    }
}

/* d(G m_j d / r^3)/dp_j = G m_j (I / r^3 - 3 d d^T / r^5); the body's own
 * block is minus the sum of the others, subtracted j by j in order. */
static void jac_nbody(const or_sys* s, const double* y, double* J) {
    int n = s->neq / 4, N = s->neq;
    double G = s->p[0];
    const double* x = y;
    const double* yy = y + n;
    for (int k = 0; k < N * N; ++k) J[k] = 0.0;
    for (int i = 0; i < n; ++i) {
        J[i * N + 2 * n + i] = 1.0;
        J[(n + i) * N + 3 * n + i] = 1.0;
        double* ru = J + (2 * n + i) * N;
        double* rv = J + (3 * n + i) * N;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[j] - x[i];
            double dy = yy[j] - yy[i];
            double r2 = dx * dx + dy * dy;
            double r3 = r2 * sqrt(r2);
            double r5 = r3 * r2;
            double gm = G * s->m->masses[j];
            double axx = gm * (1.0 / r3 - 3.0 * dx * dx / r5);
            double axy = gm * (-3.0 * dx * dy / r5);
            double ayy = gm * (1.0 / r3 - 3.0 * dy * dy / r5);
            ru[j] = axx;
            ru[n + j] = axy;
            rv[j] = axy;
            rv[n + j] = ayy;
            ru[i] -= axx;
            ru[n + i] -= axy;
            rv[i] -= axy;
            rv[n + i] -= ayy;
        }
    }
}

/* Kinetics (state T, Y_1..Y_S): with C_i = rho Y_i / W_i, q_j = k_j(T)
 * prod over reactant occurrences of C, omega_i = sum_j nu_ij q_j,
 * H = sum_i e_i W_i omega_i and f_T = -H / (rho c_v):
 *   dq_j/dY_l: product rule over the reactant occurrences of species l,
 *              each giving k_j (prod of the other occurrences) rho / W_l;
 *   dq_j/dT  = q_j (beta_j / T + Ea_j / T^2) where k_j is not clipped, else 0;
 *   row Y_i  = (W_i / rho) d omega_i;
 *   row T    = -(dH c_v - H dc_v) / (rho c_v^2), dH/dT taking de_i/dT =
 *              c_v,i and dc_v/dT = sum_i Y_i (R / W_i)(a1 + 2 a2 T).
 * The omega_i derivatives are summed reaction by reaction, reactants before
 * products, as omega_i is. */
static void jac_kinetics(const or_sys* s, const double* y, double* J) {
    const or_mech* k = s->m->mech;
    const double ln10 = 2.302585092994046;
    int S = k->n_species, N = s->neq;
    double rho = s->p[0];
    double T = y[0];
    const double* Y = y + 1;
    double lnT = or_log(T);
    double om[S > 0 ? S : 1];
    for (int z = 0; z < N * N; ++z) J[z] = 0.0;
    for (int i = 0; i < S; ++i) om[i] = 0.0;
    for (int j = 0; j < k->n_reactions; ++j) {
        double raw = or_exp(ln10 * k->log10A[j] + k->beta[j] * lnT - k->Ea[j] / T);
        double kj = fmin(fmax(raw, k->kmin), k->kmax);
        int nr = k->n_reac[j], np = k->n_prod[j];
        double c[2];
        for (int r = 0; r < nr; ++r) c[r] = rho * Y[k->reac[2 * j + r]] / k->W[k->reac[2 * j + r]];
        double q = kj;
        for (int r = 0; r < nr; ++r) q = q * c[r];
        double dT = (raw > k->kmin && raw < k->kmax) ? q * (k->beta[j] / T + k->Ea[j] / (T * T)) : 0.0;
        for (int r = 0; r < nr; ++r) J[(1 + k->reac[2 * j + r]) * N] -= dT;
        for (int r = 0; r < np; ++r) J[(1 + k->prod[2 * j + r]) * N] += dT;
        for (int o = 0; o < nr; ++o) {  /* the o-th reactant occurrence */
            int l = k->reac[2 * j + o];
            double d = kj;
            for (int r = 0; r < nr; ++r)
                if (r != o) d = d * c[r];
            d = d * rho / k->W[l];
            for (int r = 0; r < nr; ++r) J[(1 + k->reac[2 * j + r]) * N + 1 + l] -= d;
            for (int r = 0; r < np; ++r) J[(1 + k->prod[2 * j + r]) * N + 1 + l] += d;
        }
        for (int r = 0; r < nr; ++r) om[k->reac[2 * j + r]] -= q;
        for (int r = 0; r < np; ++r) om[k->prod[2 * j + r]] += q;
    }
    double cv = 0.0, H = 0.0, dcv_dT = 0.0, dH_dT_e = 0.0;
    for (int i = 0; i < S; ++i) {
        const double* a = k->thermo + 4 * i;
        double cvi = (R_GAS / k->W[i]) * (a[0] + a[1] * T + a[2] * T * T - 1.0);
        double ei = (R_GAS * T / k->W[i]) * (a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] / T - 1.0);
        cv = cv + Y[i] * cvi;
        H = H + ei * om[i] * k->W[i];
        dcv_dT = dcv_dT + Y[i] * (R_GAS / k->W[i]) * (a[1] + 2.0 * a[2] * T);
        dH_dT_e = dH_dT_e + cvi * om[i] * k->W[i];
    }
    for (int l = 0; l < N; ++l) {
        double dH = (l == 0) ? dH_dT_e : 0.0;
        for (int i = 0; i < S; ++i) {
            const double* a = k->thermo + 4 * i;
            double ei = (R_GAS * T / k->W[i]) * (a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] / T - 1.0);
            dH = dH + ei * k->W[i] * J[(1 + i) * N + l];
        }
        double dcv;
        if (l == 0) {
            dcv = dcv_dT;
        } else {
            const double* a = k->thermo + 4 * (l - 1);
            dcv = (R_GAS / k->W[l - 1]) * (a[0] + a[1] * T + a[2] * T * T - 1.0);
        }
        J[l] = -(dH * cv - H * dcv) / (rho * cv * cv);
    }
    for (int i = 0; i < S; ++i)
        for (int l = 0; l < N; ++l) J[(1 + i) * N + l] = J[(1 + i) * N + l] * k->W[i] / rho;
}

static void jacobian(const or_sys* s, const double* y, double* J) {
    int N = s->neq;
    switch (s->m->kind) {
    case KIND_VDP: jac_vdp(s, y, J); break;
    case KIND_VDP_CHAIN: jac_vdp_chain(s, y, J); break;
    case KIND_BRUSS1D: jac_bruss(s, y, J); break;
    case KIND_MASSACTION: jac_massaction(s, y, J); break;
    case KIND_NBODY: jac_nbody(s, y, J); break;
    case KIND_KINETICS: jac_kinetics(s, y, J); break;
    case KIND_LINEAR:
        for (int k = 0; k < N * N; ++k) J[k] = s->p[k];
        break;
    default:
        for (int k = 0; k < N * N; ++k) J[k] = (s->m->kind == KIND_TIME) ? 0.0 : NAN;
    }
}

/* G = max_i sum_j |J_ij| (R23). */
static double gershgorin(const or_sys* s, const double* y, double* J) {
    int N = s->neq;
    jacobian(s, y, J);
    double g = 0.0;
    for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc = acc + fabs(J[i * N + j]);
        g = fmax(g, acc);
    }
    return g;
}

static void dydt(const or_sys* s, double t, const double* y, double* f) {
    switch (s->m->kind) {
    case KIND_VDP: rhs_vdp(s, y, f); break;
    case KIND_VDP_CHAIN: rhs_vdp_chain(s, y, f); break;
    case KIND_BRUSS1D: rhs_bruss(s, y, f); break;
    case KIND_MASSACTION: rhs_massaction(s, y, f); break;
    case KIND_NBODY: rhs_nbody(s, y, f); break;
    case KIND_KINETICS: rhs_kinetics(s, y, f); break;
    case KIND_LINEAR: rhs_linear(s, y, f); break;
    case KIND_TIME:
        for (int i = 0; i < s->neq; ++i) f[i] = t;
        break;
    default:
        for (int i = 0; i < s->neq; ++i) f[i] = NAN;
    }
}

/* ------------------------------------------------ logarithm / exponential
 *
 * The step-size rules (err^(-1/4), err^(-1/5), err^(1/3), err^(2/3)) and
 * the Arrhenius rate need powers.  They are computed here from the textbook
 * series with only correctly rounded operations (+, -, *, /, frexp, ldexp,
 * rint), so any implementation that performs the same operations gets the
 * same bits (R10):
 *   ln x  : x = 2^k m with m in [sqrt(1/2), sqrt(2)), s = (m - 1)/(m + 1),
 *           ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + ... + s^22/23),
 *           ln x = k ln2_hi + (k ln2_lo + ln m);
 *   exp x : k = rint(x log2 e), r = (x - k ln2_hi) - k ln2_lo (Cody & Waite
 *           reduction, ln2_hi holding 32 significant bits), e^r by its Taylor
 *           series to r^14/14!, then scaled by 2^k;
 *   x^y   : exp(y ln x) for x > 0.
 * Accuracy is a few units in the last place (checked against libm). */
#define LN2_HI 0.6931471806019545
#define LN2_LO (-4.2009150726810846e-11)
#define LOG2E 1.4426950408889634
#define LN10 2.302585092994046
#define SQRT_HALF 0.7071067811865476

static double or_log(double x) {
#ifdef ORACLE_LIBM
    return log(x);  /* R10 off: the C library's function (a comparison build) */
#endif
    if (!(x > 0.0)) return (x == 0.0) ? -INFINITY : NAN;
    if (isinf(x)) return x;
    int k;
    double m = frexp(x, &k);
    if (m < SQRT_HALF) {
        m = m * 2.0;
        k = k - 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = 0.043478260869565216;     /* 1/23 */
    p = p * z + 0.047619047619047616;    /* 1/21 */
    p = p * z + 0.05263157894736842;     /* 1/19 */
    p = p * z + 0.058823529411764705;    /* 1/17 */
    p = p * z + 0.06666666666666667;     /* 1/15 */
    p = p * z + 0.07692307692307693;     /* 1/13 */
    p = p * z + 0.09090909090909091;     /* 1/11 */
    p = p * z + 0.1111111111111111;      /* 1/9 */
    p = p * z + 0.14285714285714285;     /* 1/7 */
    p = p * z + 0.2;                     /* 1/5 */
    p = p * z + 0.3333333333333333;      /* 1/3 */
    p = p * z + 1.0;
    double lnm = 2.0 * s * p;
    double kd = (double)k;
    return kd * LN2_HI + (kd * LN2_LO + lnm);
}

static double or_exp(double x) {
#ifdef ORACLE_LIBM
    return exp(x);
#endif
    if (isnan(x)) return x;
    if (x > 709.0) return INFINITY;
    if (x < -745.0) return 0.0;
    double kf = rint(x * LOG2E);
    double r = (x - kf * LN2_HI) - kf * LN2_LO;
    double p = 1.1470745597729725e-11;   /* 1/14! */
    p = p * r + 1.6059043836821613e-10;  /* 1/13! */
    p = p * r + 2.08767569878681e-09;    /* 1/12! */
    p = p * r + 2.505210838544172e-08;   /* 1/11! */
    p = p * r + 2.755731922398589e-07;   /* 1/10! */
    p = p * r + 2.7557319223985893e-06;  /* 1/9! */
    p = p * r + 2.48015873015873e-05;    /* 1/8! */
    p = p * r + 0.0001984126984126984;   /* 1/7! */
    p = p * r + 0.001388888888888889;    /* 1/6! */
    p = p * r + 0.008333333333333333;    /* 1/5! */
    p = p * r + 0.041666666666666664;    /* 1/4! */
    p = p * r + 0.16666666666666666;     /* 1/3! */
    p = p * r + 0.5;
    p = p * r + 1.0;
    p = p * r + 1.0;
    return ldexp(p, (int)kf);
}

static double or_pow(double x, double y) {
#ifdef ORACLE_LIBM
    return pow(x, y);
#endif
    if (x == 0.0) return (y > 0.0) ? 0.0 : INFINITY;
    return or_exp(y * or_log(x));
}

/* Arrhenius rate constant k = A T^b exp(-Ea / T) of Section 4.2 (Ea in
 * Kelvin, i.e. E/R) with A = 10^log10A, evaluated as one exponential
 * exp(ln(10) log10A + b ln T - Ea / T), then clipped to [kmin, kmax]. */
static double arrhenius(double log10A, double b, double Ea, double T, double kmin, double kmax) {
    double k = or_exp(LN10 * log10A + b * or_log(T) - Ea / T);
    if (k < kmin) k = kmin;
    if (k > kmax) k = kmax;
    return k;
}

static void sys_init(or_sys* s, const or_model* m, int neq, const double* p, int np) {
    s->m = m;
    s->neq = neq;
    for (int q = 0; q < np && q < OR_MAX_PARAMS; ++q) s->p[q] = p[q];
    if (m->kind == KIND_MASSACTION) {
        for (int j = 0; j < m->n_reactions; ++j)
            s->k[j] = arrhenius(m->log10A[j], m->beta[j], m->Ea[j], s->p[0], m->kmin, m->kmax);
    }
}

/* A model the fixed-size parameter store can hold (a linear test model
 * needs neq^2 parameters). */
static int model_fits(const or_model* m) {
    if (m->neq <= 0 || m->n_params > OR_MAX_PARAMS) return 0;
    if (m->kind == KIND_LINEAR && m->neq * m->neq > m->n_params) return 0;
    return 1;
}

static int all_finite(const double* y, int n) {
    for (int i = 0; i < n; ++i)
        if (!isfinite(y[i])) return 0;
    return 1;
}

/* ----------------------------------------------------------------- RKCK */

/* Table 1 (Cash-Karp coefficients). */
static const double A2 = 1.0 / 5.0, A3 = 3.0 / 10.0, A4 = 3.0 / 5.0, A5 = 1.0, A6 = 7.0 / 8.0;
static const double B21 = 1.0 / 5.0;
static const double B31 = 3.0 / 40.0, B32 = 9.0 / 40.0;
static const double B41 = 3.0 / 10.0, B42 = -9.0 / 10.0, B43 = 6.0 / 5.0;
static const double B51 = -11.0 / 54.0, B52 = 5.0 / 2.0, B53 = -70.0 / 27.0, B54 = 35.0 / 27.0;
static const double B61 = 1631.0 / 55296.0, B62 = 175.0 / 512.0, B63 = 575.0 / 13824.0,
                    B64 = 44275.0 / 110592.0, B65 = 253.0 / 4096.0;
static const double C1 = 37.0 / 378.0, C3 = 250.0 / 621.0, C4 = 125.0 / 594.0, C6 = 512.0 / 1771.0;
/* c_i - c*_i as exact rationals (c_2 = c*_2 = 0). */
static const double DC1 = -277.0 / 64512.0, DC3 = 6925.0 / 370944.0, DC4 = -6925.0 / 202752.0,
                    DC5 = -277.0 / 14336.0, DC6 = 277.0 / 7084.0;

/* One RKCK trial step (the k1..k6, y_{n+1} and Delta equations of Section
 * 2.1): k_i = h f(t + a_i h, y + sum_j b_ij k_j) with k_1 = h F.
 * Writes the fifth-order solution and the error vector. */
static void rkck_step(const or_sys* s, double t, const double* y, const double* F, double h,
                      double* yout, double* yerr, double* work) {
    int n = s->neq;
    double* k1 = work;
    double* k2 = k1 + n;
    double* k3 = k2 + n;
    double* k4 = k3 + n;
    double* k5 = k4 + n;
    double* k6 = k5 + n;
    double* yt = k6 + n;
    double* ft = yt + n;
    for (int i = 0; i < n; ++i) k1[i] = h * F[i];
    for (int i = 0; i < n; ++i) yt[i] = y[i] + B21 * k1[i];
    dydt(s, t + A2 * h, yt, ft);
    for (int i = 0; i < n; ++i) k2[i] = h * ft[i];
    for (int i = 0; i < n; ++i) yt[i] = y[i] + B31 * k1[i] + B32 * k2[i];
    dydt(s, t + A3 * h, yt, ft);
    for (int i = 0; i < n; ++i) k3[i] = h * ft[i];
    for (int i = 0; i < n; ++i) yt[i] = y[i] + B41 * k1[i] + B42 * k2[i] + B43 * k3[i];
    dydt(s, t + A4 * h, yt, ft);
    for (int i = 0; i < n; ++i) k4[i] = h * ft[i];
    for (int i = 0; i < n; ++i) yt[i] = y[i] + B51 * k1[i] + B52 * k2[i] + B53 * k3[i] + B54 * k4[i];
    dydt(s, t + A5 * h, yt, ft);
    for (int i = 0; i < n; ++i) k5[i] = h * ft[i];
    for (int i = 0; i < n; ++i)
        yt[i] = y[i] + B61 * k1[i] + B62 * k2[i] + B63 * k3[i] + B64 * k4[i] + B65 * k5[i];
    dydt(s, t + A6 * h, yt, ft);
    for (int i = 0; i < n; ++i) k6[i] = h * ft[i];
    for (int i = 0; i < n; ++i) {
        yout[i] = y[i] + C1 * k1[i] + C3 * k3[i] + C4 * k4[i] + C6 * k6[i];
        yerr[i] = DC1 * k1[i] + DC3 * k3[i] + DC4 * k4[i] + DC5 * k5[i] + DC6 * k6[i];
    }
}

typedef struct {
    int32_t n_accept, n_reject, n_rhs, n_specrad_iter, status;
} or_counts;

/* Adaptive RKCK for one system (rkckDriver of Section 3.1 with R1, R2, R8).
 * y holds y(t0) on entry and the final state on exit. */
static void rkck_system(const or_sys* s, double t, double tend, double rtol, double atol,
                        int max_attempts, double* y, or_counts* cnt, const double* carry_in,
                        double* carry_out) {
    int n = s->neq;
    double* mem = (double*)malloc(sizeof(double) * (size_t)n * 11);
    double* F = mem;
    double* ytemp = F + n;
    double* yerr = ytemp + n;
    double* work = yerr + n;
    const double hmax = fabs(tend - t);
    const double hmin = 1.0e-20;
    const double delta = (atol > 0.0) ? atol / rtol : TINY;
    double h = 0.5 * fabs(tend - t);
    if (carry_in && carry_in[0] == 1.0 && carry_in[2] > 0.0) h = carry_in[2];  /* R21 */
    memset(cnt, 0, sizeof(*cnt));
    while (t < tend) {
        if (cnt->n_accept + cnt->n_reject >= max_attempts) {
            cnt->status = ST_MAX_ATTEMPTS;
            break;
        }
        h = fmin(tend - t, h);
        dydt(s, t, y, F);
        rkck_step(s, t, y, F, h, ytemp, yerr, work);
        cnt->n_rhs += 6;
        double err = 0.0;
        int nan_flag = 0;
        for (int i = 0; i < n; ++i) {
            if (isnan(yerr[i])) nan_flag = 1;
            err = fmax(err, fabs(yerr[i]) / (fabs(y[i]) + fabs(h * F[i]) + delta));
        }
        err = err / rtol;
        if (err > 1.0 || isnan(err) || nan_flag) {
            cnt->n_reject += 1;
            if (isnan(err) || nan_flag)
                h = h * P1;
            else
                h = fmax(SAFETY * h * or_pow(err, PSHRNK), P1 * h);
            if (h < hmin || t + h == t) {
                cnt->status = ST_H_UNDERFLOW;
                break;
            }
        } else {
            cnt->n_accept += 1;
            t = t + h;
            if (err > ERRCON)
                h = SAFETY * h * or_pow(err, PGROW);
            else
                h = h * 5.0;
            h = fmax(hmin, fmin(hmax, h));
            for (int i = 0; i < n; ++i) y[i] = ytemp[i];
            if (!all_finite(y, n)) {
                cnt->status = ST_NONFINITE;
                break;
            }
        }
    }
    if (carry_out) {
        for (int w = 0; w < CARRY_WORDS(n); ++w) carry_out[w] = 0.0;
        carry_out[0] = (cnt->status == ST_OK || cnt->status == ST_MAX_ATTEMPTS) ? 1.0 : 0.0;
        carry_out[1] = t;
        carry_out[2] = h;
    }
    free(mem);
}

/* ------------------------------------------------------------------ RKC */

/* Coefficients of an m-stage RKC step (Section 2.2), for j = 1..m:
 *   w0 = 1 + kappa/m^2 with kappa = 2/13, Chebyshev T_j, T_j', T_j'' at w0
 *   by the three-term recurrence and its derivatives, w1 = T_m'/T_m'',
 *   b_j = T_j''/(T_j')^2 (j >= 2), b_0 = b_1 = b_2 (R3), a_j = 1 - b_j T_j,
 *   mu~_1 = b_1 w1, mu_j = 2 b_j w0 / b_{j-1}, nu_j = -b_j / b_{j-2},
 *   mu~_j = 2 b_j w1 / b_{j-1}, gamma~_j = -a_{j-1} mu~_j,
 * and the stage times c_j of R7.  Arrays have m + 1 entries. */
static void rkc_coeffs(int m, double* mu, double* nu, double* mut, double* gt, double* c) {
    double* T = (double*)malloc(sizeof(double) * (size_t)(m + 1) * 5);
    double* Tp = T + (m + 1);
    double* Tpp = Tp + (m + 1);
    double* b = Tpp + (m + 1);
    double* a = b + (m + 1);
    const double w0 = 1.0 + (2.0 / 13.0) / ((double)m * (double)m);
    T[0] = 1.0;
    T[1] = w0;
    Tp[0] = 0.0;
    Tp[1] = 1.0;
    Tpp[0] = 0.0;
    Tpp[1] = 0.0;
    for (int j = 2; j <= m; ++j) {
        T[j] = 2.0 * w0 * T[j - 1] - T[j - 2];
        Tp[j] = 2.0 * T[j - 1] + 2.0 * w0 * Tp[j - 1] - Tp[j - 2];
        Tpp[j] = 4.0 * Tp[j - 1] + 2.0 * w0 * Tpp[j - 1] - Tpp[j - 2];
    }
    const double w1 = Tp[m] / Tpp[m];
    for (int j = 2; j <= m; ++j) b[j] = Tpp[j] / (Tp[j] * Tp[j]);
    b[0] = b[2];
    b[1] = b[2];
    for (int j = 0; j <= m; ++j) a[j] = 1.0 - b[j] * T[j];
    mu[0] = nu[0] = mut[0] = gt[0] = 0.0;
    mu[1] = nu[1] = gt[1] = 0.0;
    mut[1] = b[1] * w1;
    c[0] = 0.0;
    c[1] = mut[1];
    for (int j = 2; j <= m; ++j) {
        mu[j] = 2.0 * b[j] * w0 / b[j - 1];
        nu[j] = -b[j] / b[j - 2];
        mut[j] = 2.0 * b[j] * w1 / b[j - 1];
        gt[j] = -a[j - 1] * mut[j];
        c[j] = mu[j] * c[j - 1] + nu[j] * c[j - 2] + mut[j] * (1.0 - a[j - 1]);
    }
    free(T);
}

/* One m-stage RKC step, Eqs. E:rkc0-E:rkcs: w_0 = y_n,
 * w_1 = w_0 + mu~_1 h f_0,
 * w_j = (1 - mu_j - nu_j) w_0 + mu_j w_{j-1} + nu_j w_{j-2}
 *       + mu~_j h f(t + c_{j-1} h, w_{j-1}) + gamma~_j h f_0,
 * y_{n+1} = w_m.  Uses m - 1 RHS evaluations. */
static void rkc_step(const or_sys* s, double t, const double* yn, const double* Fn, double h, int m,
                     double* y, double* work) {
    int n = s->neq;
    double* co = (double*)malloc(sizeof(double) * (size_t)(m + 1) * 5);
    double* mu = co;
    double* nu = mu + (m + 1);
    double* mut = nu + (m + 1);
    double* gt = mut + (m + 1);
    double* c = gt + (m + 1);
    rkc_coeffs(m, mu, nu, mut, gt, c);
    double* wm2 = work;       /* w_{j-2} */
    double* wm1 = wm2 + n;    /* w_{j-1} */
    double* wj = wm1 + n;     /* w_j */
    double* fj = wj + n;      /* f_{j-1} */
    for (int i = 0; i < n; ++i) wm2[i] = yn[i];
    for (int i = 0; i < n; ++i) wm1[i] = yn[i] + mut[1] * h * Fn[i];
    for (int j = 2; j <= m; ++j) {
        dydt(s, t + c[j - 1] * h, wm1, fj);
        double cy = 1.0 - mu[j] - nu[j];
        for (int i = 0; i < n; ++i)
            wj[i] = cy * yn[i] + mu[j] * wm1[i] + nu[j] * wm2[i] + mut[j] * h * fj[i] + gt[j] * h * Fn[i];
        double* tmp = wm2;
        wm2 = wm1;
        wm1 = wj;
        wj = tmp;
    }
    for (int i = 0; i < n; ++i) y[i] = wm1[i];
    free(co);
}

static double norm2(const double* x, int n) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc = acc + x[i] * x[i];
    return sqrt(acc);
}

/* Nonlinear power method of the Appendix with R5.  v is the persistent
 * eigenvector estimate (a difference from y); Fv is scratch.  Returns
 * 1.2 sigma and adds the iteration count to *iters. */
static double rkc_specrad(const or_sys* s, double t, const double* y, const double* F, double hmax,
                          double* v, double* Fv, int32_t* iters, int32_t* status) {
    const int itmax = 50;
    int n = s->neq;
    double small = 1.0 / hmax;
    double sq = sqrt(UROUND);
    double nrm1 = norm2(y, n);
    double nrm2 = norm2(v, n);
    double dynrm;
    if (nrm1 != 0.0 && nrm2 != 0.0) {
        dynrm = nrm1 * sq;
        for (int i = 0; i < n; ++i) v[i] = y[i] + v[i] * (dynrm / nrm2);
    } else if (nrm1 != 0.0) {
        dynrm = nrm1 * sq;
        for (int i = 0; i < n; ++i) v[i] = y[i] * (1.0 + sq);
    } else if (nrm2 != 0.0) {
        dynrm = UROUND;
        for (int i = 0; i < n; ++i) v[i] = v[i] * (dynrm / nrm2);
    } else {
        dynrm = UROUND;
        for (int i = 0; i < n; ++i) v[i] = UROUND;
    }
    double sigma = 0.0;
    for (int iter = 1; iter <= itmax; ++iter) {
        dydt(s, t, v, Fv);
        *iters += 1;
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc = acc + (Fv[i] - F[i]) * (Fv[i] - F[i]);
        nrm1 = sqrt(acc);
        double sigma_prev = sigma;
        sigma = nrm1 / dynrm;
        if (iter >= 2 && fabs(sigma - sigma_prev) <= fmax(sigma, small) * 0.01) {
            for (int i = 0; i < n; ++i) v[i] = v[i] - y[i];
            return 1.2 * sigma;
        }
        if (nrm1 != 0.0) {
            for (int i = 0; i < n; ++i) v[i] = y[i] + (Fv[i] - F[i]) * (dynrm / nrm1);
        } else {
            int ind = iter % n;
            v[ind] = y[ind] - (v[ind] - y[ind]);
        }
    }
    for (int i = 0; i < n; ++i) v[i] = v[i] - y[i];
    *status |= ST_SPECRAD_NOCONV;
    return 1.2 * sigma;
}

/* Adaptive RKC for one system (rkcDriver of Section 3.2 with R1, R4-R9).
 * y holds y(t0) on entry and the final state on exit. */
static void rkc_system(const or_sys* s, double t, double tend, double rtol, double atol,
                       int max_attempts, double* y, or_counts* cnt, const double* carry_in,
                       double* carry_out, int carry_mode, int specrad_mode) {
    int n = s->neq;
    double* mem = (double*)malloc(sizeof(double) * ((size_t)n * 10 + (size_t)n * n));
    double* jac = mem + (size_t)n * 10;
    double* yn = mem;
    double* Fn = yn + n;
    double* Fnp1 = Fn + n;
    double* v = Fnp1 + n;
    double* tmp = v + n;
    double* tmp2 = tmp + n;
    double* work = tmp2 + n;  /* 4 n for the stages */
    memset(cnt, 0, sizeof(*cnt));

    int mmax = (int)round(sqrt(rtol / (10.0 * UROUND)));
    if (mmax < 2) mmax = 2;
    const double hmax = fabs(tend - t);
    const double hmin = 10.0 * UROUND * fmax(fabs(t), hmax);

    for (int i = 0; i < n; ++i) yn[i] = y[i];
    dydt(s, t, yn, Fn);
    cnt->n_rhs += 1;
    double err_old = 0.0, h_old = 0.0, h = 0.0, sigma = 0.0;
    for (int i = 0; i < n; ++i) v[i] = Fn[i];

    int num_step = 0;
    int have_sigma = 0, rejected = 0, sr_step = -1;
    if (carry_in && carry_in[0] == 1.0) {  /* R21: resume the controller */
        h = carry_in[2];
        sigma = carry_in[3];
        h_old = carry_in[4];
        err_old = carry_in[5];
        num_step = (int)carry_in[6];
        sr_step = (int)carry_in[7];
        rejected = (int)carry_in[8];
        for (int i = 0; i < n; ++i) v[i] = carry_in[CARRY_FIXED + i];
        have_sigma = 1;
        if (carry_mode == CARRY_RESTART) {
            num_step = 0;
            sr_step = -1;
            rejected = 0;
        }
    }
    while (t < tend) {
        if (cnt->n_accept + cnt->n_reject >= max_attempts) {
            cnt->status |= ST_MAX_ATTEMPTS;
            break;
        }
        if (1.1 * h >= fabs(tend - t)) h = fabs(tend - t);

        if (!have_sigma || rejected || (num_step % 25 == 0 && sr_step != num_step)) {
            if (specrad_mode == SPECRAD_GERSHGORIN) {
                sigma = gershgorin(s, yn, jac);
            } else {
                sigma = rkc_specrad(s, t, yn, Fn, hmax, v, tmp2, &cnt->n_specrad_iter, &cnt->status);
                if (specrad_mode == SPECRAD_POWER_CAPPED) sigma = fmin(sigma, gershgorin(s, yn, jac));
            }
            have_sigma = 1;
            sr_step = num_step;
        }

        if (h < UROUND) {
            /* initial step: trial Euler step of size 1/sigma */
            h = hmax;
            if (sigma * h > 1.0) h = 1.0 / sigma;
            h = fmax(h, hmin);
            for (int i = 0; i < n; ++i) tmp[i] = yn[i] + h * Fn[i];
            dydt(s, t + h, tmp, tmp2);
            cnt->n_rhs += 1;
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                double est = (tmp2[i] - Fn[i]) / (atol + rtol * fabs(yn[i]));
                acc = acc + est * est;
            }
            double est = h * sqrt(acc / (double)n);
            if (P1 * h < hmax * sqrt(est))
                h = fmax(P1 * h / sqrt(est), hmin);
            else
                h = hmax;
        }

        int m = 1 + (int)sqrt(1.54 * h * sigma + 1.0);
        if (m > mmax) {
            m = mmax;
            h = (double)(m * m - 1) / (1.54 * sigma);
        }

        rkc_step(s, t, yn, Fn, h, m, y, work);
        dydt(s, t + h, y, Fnp1);
        cnt->n_rhs += m;   /* m - 1 stage evaluations and F_{n+1} */

        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            double est = 0.8 * (yn[i] - y[i]) + 0.4 * h * (Fn[i] + Fnp1[i]);
            est = est / (atol + rtol * fmax(fabs(y[i]), fabs(yn[i])));
            acc = acc + est * est;
        }
        double err = sqrt(acc / (double)n);

        if (isnan(err)) {
            cnt->n_reject += 1;
            cnt->status |= ST_NONFINITE;
            break;
        }
        if (err > 1.0) {
            cnt->n_reject += 1;
            h = 0.8 * h / or_pow(err, 1.0 / 3.0);
            rejected = 1;
            if (h < hmin) {
                cnt->status |= ST_H_UNDERFLOW;
                break;
            }
        } else {
            cnt->n_accept += 1;
            rejected = 0;
            t = t + h;
            num_step += 1;
            double fac = 10.0;
            if (h_old < UROUND) {
                double temp2 = or_pow(err, 1.0 / 3.0);
                if (0.8 < fac * temp2) fac = 0.8 / temp2;
            } else {
                double temp1 = 0.8 * h * or_pow(err_old, 1.0 / 3.0);
                double temp2 = h_old * or_pow(err, 2.0 / 3.0);
                if (temp1 < fac * temp2) fac = temp1 / temp2;
            }
            err_old = err;
            h_old = h;
            for (int i = 0; i < n; ++i) {
                yn[i] = y[i];
                Fn[i] = Fnp1[i];
            }
            h = h * fmax(P1, fac);
            h = fmax(hmin, fmin(hmax, h));
            if (!all_finite(yn, n)) {
                cnt->status |= ST_NONFINITE;
                break;
            }
        }
    }
    cnt->n_rhs += cnt->n_specrad_iter;
    for (int i = 0; i < n; ++i) y[i] = yn[i];
    if (carry_out) {
        const int st = cnt->status & 0xFF;
        carry_out[0] = (st == ST_OK || st == ST_MAX_ATTEMPTS) && have_sigma ? 1.0 : 0.0;
        carry_out[1] = t;
        carry_out[2] = h;
        carry_out[3] = sigma;
        carry_out[4] = h_old;
        carry_out[5] = err_old;
        carry_out[6] = (double)num_step;
        carry_out[7] = (double)sr_step;
        carry_out[8] = (double)rejected;
        for (int i = 0; i < n; ++i) carry_out[CARRY_FIXED + i] = v[i];
    }
    free(mem);
}

/* ------------------------------------------------------------ exports */

static int resolve_threads(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Gather the SoA column of system i into the per-system arrays. */
static void gather(const double* src, int64_t nsys, int64_t i, int n, double* dst) {
    for (int j = 0; j < n; ++j) dst[j] = src[i + nsys * (int64_t)j];
}

/* Batched integration of a uniform batch (SoA [neq][nsys] in and out).
 * method 0 = RKCK, 1 = RKC.  Counters are per system and may be NULL. */
/* carry_in / carry_out (R21, may be NULL): SoA [CARRY_WORDS(neq)][nsys]. */
int oracle_integrate(const or_model* m, int method, int64_t nsys, const double* y0,
                     const double* params, double t0, double tend, double rtol, double atol,
                     int max_attempts, double* y_out, int32_t* n_accept, int32_t* n_reject,
                     int32_t* n_rhs, int32_t* n_specrad_iter, int32_t* status, int nthreads,
                     const double* carry_in, double* carry_out, int carry_mode, int specrad_mode) {
    if (!model_fits(m)) return -1;
    int nt = resolve_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < nsys; ++i) {
        or_sys s;
        double p[OR_MAX_PARAMS];
        gather(params, nsys, i, m->n_params, p);
        sys_init(&s, m, m->neq, p, m->n_params);
        double* y = (double*)malloc(sizeof(double) * (size_t)m->neq);
        gather(y0, nsys, i, m->neq, y);
        const int K = CARRY_WORDS(m->neq);
        double* cin = NULL;
        double* cout = NULL;
        if (carry_in) {
            cin = (double*)malloc(sizeof(double) * (size_t)K);
            gather(carry_in, nsys, i, K, cin);
        }
        if (carry_out) cout = (double*)malloc(sizeof(double) * (size_t)K);
        or_counts cnt;
        if (method == 0)
            rkck_system(&s, t0, tend, rtol, atol, max_attempts, y, &cnt, cin, cout);
        else
            rkc_system(&s, t0, tend, rtol, atol, max_attempts, y, &cnt, cin, cout, carry_mode, specrad_mode);
        for (int j = 0; j < m->neq; ++j) y_out[i + nsys * (int64_t)j] = y[j];
        if (cout)
            for (int w = 0; w < K; ++w) carry_out[i + nsys * (int64_t)w] = cout[w];
        free(cin);
        free(cout);
        if (n_accept) n_accept[i] = cnt.n_accept;
        if (n_reject) n_reject[i] = cnt.n_reject;
        if (n_rhs) n_rhs[i] = cnt.n_rhs;
        if (n_specrad_iter) n_specrad_iter[i] = cnt.n_specrad_iter;
        if (status) status[i] = cnt.status;
        free(y);
    }
    return 0;
}

/* Ragged batch: system i has model models[model_idx[i]] with neq[i]
 * unknowns stored contiguously at y0[offset[i]..], one scalar parameter
 * param[i], its own method, time interval and tolerances. */
int oracle_integrate_ragged(const or_model* models, const int32_t* model_idx, int64_t nsys,
                            const int32_t* neq, const int64_t* offset, const double* y0,
                            const double* param, const int32_t* method, const double* t0,
                            const double* tend, const double* rtol, const double* atol,
                            int max_attempts, double* y_out, int32_t* n_accept, int32_t* n_reject,
                            int32_t* n_rhs, int32_t* n_specrad_iter, int32_t* status, int nthreads) {
    int nt = resolve_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t i = 0; i < nsys; ++i) {
        or_sys s;
        double p = param[i];
        sys_init(&s, &models[model_idx[i]], neq[i], &p, 1);
        double* y = y_out + offset[i];
        for (int j = 0; j < neq[i]; ++j) y[j] = y0[offset[i] + j];
        or_counts cnt;
        if (method[i] == 0)
            rkck_system(&s, t0[i], tend[i], rtol[i], atol[i], max_attempts, y, &cnt, NULL, NULL);
        else
            rkc_system(&s, t0[i], tend[i], rtol[i], atol[i], max_attempts, y, &cnt, NULL, NULL, 0, SPECRAD_POWER);
        if (n_accept) n_accept[i] = cnt.n_accept;
        if (n_reject) n_reject[i] = cnt.n_reject;
        if (n_rhs) n_rhs[i] = cnt.n_rhs;
        if (n_specrad_iter) n_specrad_iter[i] = cnt.n_specrad_iter;
        if (status) status[i] = cnt.status;
    }
    return 0;
}

/* Single-system entry points used by the oracle's own tests. */

void oracle_rhs(const or_model* m, const double* p, double t, const double* y, double* f) {
    if (!model_fits(m)) {
        for (int k = 0; k < m->neq; ++k) f[k] = NAN;
        return;
    }
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    dydt(&s, t, y, f);
}

void oracle_rate_constants(const or_model* m, double T, double* k) {
    for (int j = 0; j < m->n_reactions; ++j)
        k[j] = arrhenius(m->log10A[j], m->beta[j], m->Ea[j], T, m->kmin, m->kmax);
}

void oracle_rkck_step(const or_model* m, const double* p, double t, const double* y, double h,
                      double* yout, double* yerr) {
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    int n = m->neq;
    double* F = (double*)malloc(sizeof(double) * (size_t)n * 9);
    dydt(&s, t, y, F);
    rkck_step(&s, t, y, F, h, yout, yerr, F + n);
    free(F);
}

void oracle_rkc_step(const or_model* m, const double* p, double t, const double* y, double h,
                     int stages, double* yout) {
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    int n = m->neq;
    double* F = (double*)malloc(sizeof(double) * (size_t)n * 5);
    dydt(&s, t, y, F);
    rkc_step(&s, t, y, F, h, stages, yout, F + n);
    free(F);
}

void oracle_rkc_coeffs(int m, double* mu, double* nu, double* mut, double* gt, double* c) {
    rkc_coeffs(m, mu, nu, mut, gt, c);
}

/* Fixed-step integration (controller off): nsteps steps of size h from t0.
 * method 0 = RKCK, 1 = RKC with the given stage count. */
void oracle_fixed_steps(const or_model* m, const double* p, int method, int stages, double t0,
                        double h, int nsteps, const double* y0, double* yout) {
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    int n = m->neq;
    double* mem = (double*)malloc(sizeof(double) * (size_t)n * 14);
    double* y = mem;
    double* F = y + n;
    double* yerr = F + n;
    double* work = yerr + n;
    for (int i = 0; i < n; ++i) y[i] = y0[i];
    double t = t0;
    for (int k = 0; k < nsteps; ++k) {
        dydt(&s, t, y, F);
        if (method == 0)
            rkck_step(&s, t, y, F, h, yout, yerr, work);
        else
            rkc_step(&s, t, y, F, h, stages, yout, work);
        for (int i = 0; i < n; ++i) y[i] = yout[i];
        t = t0 + (double)(k + 1) * h;
    }
    for (int i = 0; i < n; ++i) yout[i] = y[i];
    free(mem);
}

void oracle_jacobian(const or_model* m, const double* p, const double* y, double* J) {
    if (!model_fits(m)) {
        for (int k = 0; k < m->neq * m->neq; ++k) J[k] = NAN;
        return;
    }
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    jacobian(&s, y, J);
}

double oracle_gershgorin(const or_model* m, const double* p, const double* y) {
    if (!model_fits(m)) return NAN;
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    double* J = (double*)malloc(sizeof(double) * (size_t)m->neq * m->neq);
    double g = gershgorin(&s, y, J);
    free(J);
    return g;
}

double oracle_specrad(const or_model* m, const double* p, double t, const double* y, double hmax,
                      double* v, int32_t* iters, int32_t* status) {
    or_sys s;
    sys_init(&s, m, m->neq, p, m->n_params);
    int n = m->neq;
    double* F = (double*)malloc(sizeof(double) * (size_t)n * 2);
    dydt(&s, t, y, F);
    double r = rkc_specrad(&s, t, y, F, hmax, v, F + n, iters, status);
    free(F);
    return r;
}

int oracle_model_size(void) { return (int)sizeof(or_model); }

double oracle_pow(double x, double y) { return or_pow(x, y); }
double oracle_exp(double x) { return or_exp(x); }
double oracle_log(double x) { return or_log(x); }
