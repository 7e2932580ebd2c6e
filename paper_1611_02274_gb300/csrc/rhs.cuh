// rhs.cuh -- device right-hand sides f(t, y; g) of the registered families.
//
// A Model fixes the team width W (lanes per system) and PER (state slots
// per lane).  Its Sys<R> holds one system's parameters in registers
// (R = double for the plain form, float for the mixed form) and provides
//   comp(team, s)  component index held in slot s by this lane (-1 = unused)
//   rhs(team, t, y, f)  f = f(t, y) on this lane's slots.
//   gershgorin(team, y)  max_i sum_j |J_ij| of the analytic Jacobian J at y
//                  (the Gershgorin bound on the spectral radius), each row
//                  sum over its nonzero columns in increasing order
// Grid families (Brusselator, oscillator chain) place grid point
// g = q W + lane in slots 2q (u or x) and 2q + 1 (v), so stencil neighbours
// are one lane away and come from shuffles.  Evaluation orders follow the
// defining formulas left to right (the compiler may fuse a multiply-add).
#pragma once
#include <cmath>

#include "common.cuh"
#include "team.cuh"
#include "xmath.cuh"

namespace bode {

template <class R>
__device__ __forceinline__ R rabs(R x) {
    if constexpr (sizeof(R) == 8)
        return fabs(x);
    else
        return fabsf(x);
}
template <class R>
__device__ __forceinline__ R rmax(R a, R b) {
    if constexpr (sizeof(R) == 8)
        return fmax(a, b);
    else
        return fmaxf(a, b);
}

// van der Pol: y1' = y2, y2' = mu (1 - y1^2) y2 - y1.  params [mu].
struct VdpModel {
    static constexpr int W = 1, PER = 2;
    using Ctx = NoCtx;
    template <class R>
    struct Sys {
        R mu;
        int n;
        __device__ void load(const Ctx&, const Team<W>&, double param, int neq) {
            mu = (R)param;
            n = neq;
        }
        __device__ int comp(const Team<W>&, int s) const { return s; }
        // sum over components in component order (the plain form's norms)
        template <class T>
        __device__ T ordered_sum(const Team<W>&, const T* x) const {
            T acc = T(0);
            acc = acc + x[0];
            acc = acc + x[1];
            return acc;
        }
        __device__ void rhs(const Team<W>&, R, const R* y, R* f) const {
            f[0] = y[1];
            f[1] = mu * (R(1) - y[0] * y[0]) * y[1] - y[0];
        }
        // rows: (0, 1) and (mu (-2 y1) y2 - 1, mu (1 - y1^2))
        __device__ R gershgorin(const Team<W>&, const R* y) const {
            const R j10 = mu * (R(-2) * y[0]) * y[1] - R(1);
            const R j11 = mu * (R(1) - y[0] * y[0]);
            return rmax(R(1), rabs(j10) + rabs(j11));
        }
    };
};

struct GridCtx {
    double A, B, ubc, vbc;  // Brusselator constants
    double coupling;        // chain coupling
};

// Chain of n van der Pol oscillators, state [x_1..x_n, v_1..v_n]:
// x_i' = v_i, v_i' = mu (1 - x_i^2) v_i - x_i + c ((x_{i-1} - x_i) + (x_{i+1} - x_i)),
// neighbour terms dropped at the free ends.  params [mu].
template <int W_, int G>
struct ChainModel {
    static constexpr int W = W_, PER = 2 * G;
    using Ctx = GridCtx;
    template <class R>
    struct Sys {
        R mu, c;
        int n, npts;
        __device__ void load(const Ctx& ctx, const Team<W>&, double param, int neq) {
            mu = (R)param;
            c = (R)ctx.coupling;
            n = neq;
            npts = neq / 2;
        }
        __device__ int comp(const Team<W>& tm, int s) const {
            const int g = (s >> 1) * W + tm.lane;
            return g < npts ? ((s & 1) ? npts + g : g) : -1;
        }
        // sum over components in component order, first field then second
        // (the plain form's norms, reproducing a sequential loop)
        template <class T>
        __device__ T ordered_sum(const Team<W>& tm, const T* x) const {
            T acc = T(0);
#pragma unroll
            for (int fld = 0; fld < 2; ++fld)
#pragma unroll(G <= 32 ? G : 2)
                for (int q = 0; q < G; ++q)
#pragma unroll
                    for (int l = 0; l < W; ++l) {
                        const T v = tm.bcast(x[2 * q + fld], l);
                        if (q * W + l < npts) acc = acc + v;
                    }
            return acc;
        }
        __device__ void rhs(const Team<W>& tm, R, const R* y, R* f) const {
#pragma unroll(G <= 32 ? G : 2)
            for (int q = 0; q < G; ++q) {
                const int g = q * W + tm.lane;
                const R x = y[2 * q];
                R xl = tm.from_left(x);
                if (q > 0) {
                    const R w = tm.bcast(y[2 * q - 2], W - 1);
                    if (tm.lane == 0) xl = w;
                }
                R xr = tm.from_right(x);
                if (q < G - 1) {
                    const R w = tm.bcast(y[2 * q + 2], 0);
                    if (tm.lane == W - 1) xr = w;
                }
                R coup = R(0);
                if (g > 0) coup = coup + (xl - x);
                if (g + 1 < npts) coup = coup + (xr - x);
                const R v = y[2 * q + 1];
                f[2 * q] = v;
                f[2 * q + 1] = mu * (R(1) - x * x) * v - x + c * coup;
            }
        }
        // row x_i: one entry 1; row v_i: c (x_{i-1}), mu (-2 x) v - 1 - c nb
        // (x_i), c (x_{i+1}), mu (1 - x^2) (v_i), neighbours that exist only
        __device__ R gershgorin(const Team<W>& tm, const R* y) const {
            R g = R(0);
#pragma unroll(G <= 32 ? G : 2)
            for (int q = 0; q < G; ++q) {
                const int gp = q * W + tm.lane;
                if (gp >= npts) continue;
                const R x = y[2 * q], v = y[2 * q + 1];
                const bool left = gp > 0, right = gp + 1 < npts;
                const R nb = R((int)left + (int)right);
                const R jxx = mu * (R(-2) * x) * v - R(1) - c * nb;
                const R jvv = mu * (R(1) - x * x);
                R acc = R(0);
                if (left) acc = acc + rabs(c);
                acc = acc + rabs(jxx);
                if (right) acc = acc + rabs(c);
                acc = acc + rabs(jvv);
                g = rmax(g, rmax(R(1), acc));
            }
            return tm.max(g);
        }
    };
};

// 1D Brusselator on n interior points, state [u_1..u_n, v_1..v_n]:
// u' = A + u^2 v - (B + 1) u + D (u_{k-1} - 2 u_k + u_{k+1}),
// v' = B u - u^2 v + D (v_{k-1} - 2 v_k + v_{k+1}),
// D = a / dx^2, dx = 1/(n+1), ghosts u = ubc, v = vbc.  params [a].
template <int W_, int G>
struct BrussModel {
    static constexpr int W = W_, PER = 2 * G;
    using Ctx = GridCtx;
    template <class R>
    struct Sys {
        R D, A, B1, B, ubc, vbc;
        int n, npts;
        __device__ void load(const Ctx& ctx, const Team<W>&, double a, int neq) {
            n = neq;
            npts = neq / 2;
            const double dx = 1.0 / (double)(npts + 1);
            D = (R)(a / (dx * dx));
            A = (R)ctx.A;
            B = (R)ctx.B;
            B1 = (R)(ctx.B + 1.0);
            ubc = (R)ctx.ubc;
            vbc = (R)ctx.vbc;
        }
        __device__ int comp(const Team<W>& tm, int s) const {
            const int g = (s >> 1) * W + tm.lane;
            return g < npts ? ((s & 1) ? npts + g : g) : -1;
        }
        // sum over components in component order, first field then second
        // (the plain form's norms, reproducing a sequential loop)
        template <class T>
        __device__ T ordered_sum(const Team<W>& tm, const T* x) const {
            T acc = T(0);
#pragma unroll
            for (int fld = 0; fld < 2; ++fld)
#pragma unroll(G <= 32 ? G : 2)
                for (int q = 0; q < G; ++q)
#pragma unroll
                    for (int l = 0; l < W; ++l) {
                        const T v = tm.bcast(x[2 * q + fld], l);
                        if (q * W + l < npts) acc = acc + v;
                    }
            return acc;
        }
        __device__ void rhs(const Team<W>& tm, R, const R* y, R* f) const {
#pragma unroll(G <= 32 ? G : 2)
            for (int q = 0; q < G; ++q) {
                const int g = q * W + tm.lane;
                const R u = y[2 * q], v = y[2 * q + 1];
                R ul = tm.from_left(u), vl = tm.from_left(v);
                if (q > 0) {
                    const R uw = tm.bcast(y[2 * q - 2], W - 1), vw = tm.bcast(y[2 * q - 1], W - 1);
                    if (tm.lane == 0) {
                        ul = uw;
                        vl = vw;
                    }
                }
                R ur = tm.from_right(u), vr = tm.from_right(v);
                if (q < G - 1) {
                    const R uw = tm.bcast(y[2 * q + 2], 0), vw = tm.bcast(y[2 * q + 3], 0);
                    if (tm.lane == W - 1) {
                        ur = uw;
                        vr = vw;
                    }
                }
                if (g == 0) {
                    ul = ubc;
                    vl = vbc;
                }
                if (g + 1 >= npts) {
                    ur = ubc;
                    vr = vbc;
                }
                const R uuv = u * u * v;
                f[2 * q] = A + uuv - B1 * u + D * (ul - R(2) * u + ur);
                f[2 * q + 1] = B * u - uuv + D * (vl - R(2) * v + vr);
            }
        }
        // row u_k: D (u_{k-1}), 2 u v - (B + 1) - 2 D (u_k), D (u_{k+1}), u^2 (v_k);
        // row v_k: B - 2 u v (u_k), D (v_{k-1}), -u^2 - 2 D (v_k), D (v_{k+1});
        // the Dirichlet ghosts are constants: no boundary neighbour entries
        __device__ R gershgorin(const Team<W>& tm, const R* y) const {
            R g = R(0);
#pragma unroll(G <= 32 ? G : 2)
            for (int q = 0; q < G; ++q) {
                const int gp = q * W + tm.lane;
                if (gp >= npts) continue;
                const R u = y[2 * q], v = y[2 * q + 1];
                const bool left = gp > 0, right = gp + 1 < npts;
                const R juu = R(2) * u * v - B1 - R(2) * D;
                const R juv = u * u;
                const R jvu = B - R(2) * u * v;
                const R jvv = -(u * u) - R(2) * D;
                R ru = R(0), rv = R(0);
                if (left) ru = ru + rabs(D);
                ru = ru + rabs(juu);
                if (right) ru = ru + rabs(D);
                ru = ru + rabs(juv);
                rv = rv + rabs(jvu);
                if (left) rv = rv + rabs(D);
                rv = rv + rabs(jvv);
                if (right) rv = rv + rabs(D);
                g = rmax(g, rmax(ru, rv));
            }
            return tm.max(g);
        }
    };
};

struct KinCtx {
    KinDevice k;
};

// Constant-volume kinetics with a temperature equation (Section 4.2), one
// warp per system: component c (0 = T, 1 + i = Y_i) in slot c / 32 of lane
// c % 32.  Per evaluation the team stages the S concentrations
// C_i = rho Y_i / W_i and the R rate constants in its shared memory; each
// lane then sums omega_i over the incidence lists of the species the
// mechanism's schedule gives it (balanced by list length; each list in
// reaction order, reactants first, as the oracle accumulates), the owners
// read omega_i back, and the temperature equation's species sums run in
// species order by shuffles.
// The plain form takes the rate constants through the series exponential
// and logarithm (bitwise equal to the oracle's); the mixed form in FP32.
// params [rho].
template <int W_>
struct KinModel {
    static_assert(W_ == 32, "one warp per kinetics system");
    static constexpr int W = W_, PER = 2;
    using Ctx = KinCtx;
    // shared memory per thread (floats): a team stages up to 64
    // concentrations, 64 omega_i and kKinMaxReactions rate constants in FP64
    static constexpr int SMEM_FLOATS = (2 * (64 + 64 + kKinMaxReactions) + W_ - 1) / W_;
    static_assert((W_ * SMEM_FLOATS) % 2 == 0, "team regions keep FP64 alignment");
    template <class R>
    struct Sys {
        const KinDevice* k;
        R rho;
        int n;
        R* sC;   // [64] concentrations of this team's system
        R* sOm;  // [64] omega_i, summed on the schedule's lanes
        R* sK;   // [kKinMaxReactions] rate constants
        __device__ void load(const Ctx& ctx, const Team<W>&, double p, int neq) {
            k = &ctx.k;
            rho = (R)p;
            n = neq;
        }
        // block_base: this model's part of the block's dynamic shared memory
        // (16-byte aligned; each team's region is W * SMEM_FLOATS floats, a
        // multiple of 8 bytes)
        __device__ void bind(float* block_base, int) {
            R* team = reinterpret_cast<R*>(block_base + (threadIdx.x / W) * W * SMEM_FLOATS);
            sC = team;
            sOm = team + 64;
            sK = team + 128;
        }
        __device__ int comp(const Team<W>& tm, int s) const {
            const int c = s * W + tm.lane;
            return c < n ? c : -1;
        }
        template <class T>
        __device__ T ordered_sum(const Team<W>& tm, const T* x) const {
            T acc = T(0);
#pragma unroll
            for (int s = 0; s < PER; ++s)
#pragma unroll
                for (int l = 0; l < W; ++l) {
                    const T v = tm.bcast(x[s], l);
                    if (s * W + l < n) acc = acc + v;
                }
            return acc;
        }
        __device__ R rate(int j, R T, R lnT) const {
            if constexpr (sizeof(R) == 8) {
                const double kk = xm::exp_series(xm::kLn10 * __ldg(k->log10A + j) + __ldg(k->beta + j) * lnT -
                                                 __ldg(k->Ea + j) / T);
                return fmin(fmax(kk, k->kmin), k->kmax);
            } else {  // lnT holds log2 T here, and T the reciprocal 1 / T
                const float4 q = __ldg(k->rate32 + j);
                return fminf(fmaxf(exp2f(q.x + q.y * lnT - q.z * T), (float)k->kmin), (float)k->kmax);
            }
        }
        // omega_i of species i: the signed rates of progress over its
        // incidence list, in list order
        __device__ R omega(int i) const {
            R om = R(0);
            const int e1 = __ldg(k->inc_off + i + 1);
            for (int e = __ldg(k->inc_off + i); e < e1; ++e) {
                const unsigned word = (unsigned)__ldg(k->inc + e);
                R q = sK[word & 1023u] * sC[__byte_perm(word, 0u, 0x4442)];
                if constexpr (sizeof(R) == 8) {  // FP64 pipe bound: skip the factor 1
                    if ((word >> 24) != (unsigned)kKinOne) q = q * sC[word >> 24];
                } else {
                    q = q * sC[word >> 24];
                }
                om = (word & (1u << 10)) ? om + q : om - q;
            }
            return om;
        }
        // every omega_i into sOm, each on its scheduled lane (reads the
        // staged sC / sK; the warp synchronises before and after)
        __device__ void omegas(const Team<W>& tm) const {
            __syncwarp();
            for (int kk = 0; kk < k->sched_k; ++kk) {
                const int i = __ldg(k->sched + kk * 32 + tm.lane);
                if (i >= 0) sOm[i] = omega(i);
            }
            __syncwarp();
        }
        __device__ void rhs(const Team<W>& tm, R, const R* y, R* f) const {
            const R T = tm.bcast(y[0], 0);
            R om[PER], cvy[PER], hw[PER];
            if constexpr (sizeof(R) == 8) {
                const R lnT = xm::log_series(T);
#pragma unroll
                for (int s = 0; s < PER; ++s) {
                    const int c = s * W + tm.lane;
                    if (c >= 1 && c < n) sC[c - 1] = rho * y[s] / (R)__ldg(k->W + c - 1);
                }
                if (tm.lane == 0) sC[kKinOne] = R(1);
                for (int j = tm.lane; j < k->R; j += W) sK[j] = rate(j, T, lnT);
                omegas(tm);
#pragma unroll
                for (int s = 0; s < PER; ++s) {
                    om[s] = cvy[s] = hw[s] = f[s] = R(0);
                    const int c = s * W + tm.lane;
                    if (c < 1 || c >= n) continue;
                    const int i = c - 1;
                    om[s] = sOm[i];
                    const double* a = k->thermo + 4 * i;
                    const R a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3);
                    const R Wi = __ldg(k->W + i);
                    const R Rg = 8.314462618;
                    const R cvi = (Rg / Wi) * (a0 + a1 * T + a2 * T * T - R(1));
                    const R ei = (Rg * T / Wi) * (a0 + a1 * T / R(2) + a2 * T * T / R(3) + a3 / T - R(1));
                    cvy[s] = y[s] * cvi;
                    hw[s] = ei * om[s] * Wi;
                    f[s] = Wi * om[s] / rho;
                }
            } else {  // FP32: reciprocals instead of divisions, coefficients pre-scaled at registration
                const R invT = R(1) / T, log2T = __log2f(T), inv_rho = R(1) / rho;
#pragma unroll
                for (int s = 0; s < PER; ++s) {
                    const int c = s * W + tm.lane;
                    if (c >= 1 && c < n) sC[c - 1] = rho * y[s] * __ldg(k->thermo32 + 2 * (c - 1) + 1).z;
                }
                if (tm.lane == 0) sC[kKinOne] = R(1);
                for (int j = tm.lane; j < k->R; j += W) sK[j] = rate(j, invT, log2T);
                omegas(tm);
#pragma unroll
                for (int s = 0; s < PER; ++s) {
                    om[s] = cvy[s] = hw[s] = f[s] = R(0);
                    const int c = s * W + tm.lane;
                    if (c < 1 || c >= n) continue;
                    const int i = c - 1;
                    om[s] = sOm[i];
                    const float4 a = __ldg(k->thermo32 + 2 * i), wv = __ldg(k->thermo32 + 2 * i + 1);
                    const R cvi = wv.x * (a.x + a.y * T + a.z * T * T - R(1));
                    const R ei = (wv.x * T) * (a.x + a.y * T * R(0.5) + a.z * T * T * R(1.0 / 3.0) + a.w * invT - R(1));
                    cvy[s] = y[s] * cvi;
                    hw[s] = ei * om[s] * wv.y;
                    f[s] = wv.y * om[s] * inv_rho;
                }
            }
            __syncwarp();  // the staged values are read before the next evaluation writes them
            const R cv = ordered_sum(tm, cvy);
            const R heat = ordered_sum(tm, hw);
            if (tm.lane == 0) f[0] = -heat / (rho * cv);
        }
        __device__ R gershgorin(const Team<W>&, const R*) const { return R(0) / R(0); }  // not provided
    };
};

struct NbodyCtx {
    double m[kMaxBodies];  // body masses
};

// Planar n-body gravity (the Pleiades problem's form), one body per lane
// (n <= W): slots 0..3 of lane b hold x_b, y_b, u_b, v_b; the other bodies'
// positions come from shuffles, taken in ascending order j as in the
// defining sum.  The plain form evaluates m_j d / (r2 sqrt(r2)) as written;
// the mixed form uses the reciprocal square root.  params [G].
template <int W_>
struct NbodyModel {
    static constexpr int W = W_, PER = 4;
    using Ctx = NbodyCtx;
    template <class R>
    struct Sys {
        R G;
        R m[W_];
        int n, nb;
        __device__ void load(const Ctx& ctx, const Team<W>&, double g, int neq) {
            G = (R)g;
            n = neq;
            nb = neq / 4;
#pragma unroll
            for (int j = 0; j < W_; ++j) m[j] = (R)(j < nb ? ctx.m[j] : 0.0);
        }
        __device__ int comp(const Team<W>& tm, int s) const { return tm.lane < nb ? s * nb + tm.lane : -1; }
        // sum over components in component order (x, then y, u, v)
        template <class T>
        __device__ T ordered_sum(const Team<W>& tm, const T* x) const {
            T acc = T(0);
#pragma unroll
            for (int fld = 0; fld < 4; ++fld)
#pragma unroll
                for (int l = 0; l < W_; ++l) {
                    const T v = tm.bcast(x[fld], l);
                    if (l < nb) acc = acc + v;
                }
            return acc;
        }
        __device__ void rhs(const Team<W>& tm, R, const R* y, R* f) const {
            const R x = y[0], yy = y[1];
            R ax = R(0), ay = R(0);
#pragma unroll
            for (int j = 0; j < W_; ++j) {
                const R xj = tm.bcast(x, j), yj = tm.bcast(yy, j);
                if (j < nb && j != tm.lane) {
                    const R dx = xj - x, dy = yj - yy;
                    const R r2 = dx * dx + dy * dy;
                    if constexpr (sizeof(R) == 8) {
                        const R r3 = r2 * sqrt(r2);
                        ax = ax + m[j] * dx / r3;
                        ay = ay + m[j] * dy / r3;
                    } else {
                        const R ir = rsqrtf(r2);
                        const R w = m[j] * (ir * ir * ir);
                        ax = fmaf(w, dx, ax);
                        ay = fmaf(w, dy, ay);
                    }
                }
            }
            f[0] = y[2];
            f[1] = y[3];
            f[2] = G * ax;
            f[3] = G * ay;
        }
        // (xx, xy, yy) block of d(acceleration of this body)/d(position of
        // body j): G m_j (I / r^3 - 3 d d^T / r^5), as the Jacobian writes it
        __device__ void block(R x, R yy, R xj, R yj, int j, R& bxx, R& bxy, R& byy) const {
            const R dx = xj - x, dy = yj - yy;
            const R r2 = dx * dx + dy * dy;
            R r3;
            if constexpr (sizeof(R) == 8)
                r3 = r2 * sqrt(r2);
            else
                r3 = r2 * sqrtf(r2);
            const R r5 = r3 * r2;
            const R gm = G * m[j];
            bxx = gm * (R(1) / r3 - R(3) * dx * dx / r5);
            bxy = gm * (R(-3) * dx * dy / r5);
            byy = gm * (R(1) / r3 - R(3) * dy * dy / r5);
        }
        // rows x_i, y_i: one entry 1; rows u_i, v_i over the x columns then
        // the y columns, the own block being minus the sum of the others
        // (three passes, the blocks recomputed instead of kept)
        __device__ R gershgorin(const Team<W>& tm, const R* y) const {
            const R x = y[0], yy = y[1];
            const int i = tm.lane;
            R dxx = R(0), dxy = R(0), dyy = R(0);
#pragma unroll
            for (int j = 0; j < W_; ++j) {
                const R xj = tm.bcast(x, j), yj = tm.bcast(yy, j);
                if (j < nb && j != i) {
                    R bxx, bxy, byy;
                    block(x, yy, xj, yj, j, bxx, bxy, byy);
                    dxx = dxx - bxx;
                    dxy = dxy - bxy;
                    dyy = dyy - byy;
                }
            }
            R ru = R(0), rv = R(0);
#pragma unroll
            for (int pass = 0; pass < 2; ++pass)  // x columns, then y columns
#pragma unroll
                for (int j = 0; j < W_; ++j) {
                    const R xj = tm.bcast(x, j), yj = tm.bcast(yy, j);
                    if (j < nb) {
                        R bxx = dxx, bxy = dxy, byy = dyy;
                        if (j != i) block(x, yy, xj, yj, j, bxx, bxy, byy);
                        ru = ru + rabs(pass == 0 ? bxx : bxy);
                        rv = rv + rabs(pass == 0 ? bxy : byy);
                    }
                }
            return tm.max(i < nb ? rmax(R(1), rmax(ru, rv)) : R(0));
        }
    };
};

// Mass-action kinetics with a registered network (Section 4.2 omega_i at
// constant T): r_j = k_j prod_{reactants} C, C_s' = sum_j (nu''_sj - nu'_sj) r_j,
// accumulated over reactions in order, reactants then products.  params [T].
// The rate constants (step a2: Arrhenius, clipped) are computed once per
// system and kept in registers.  One thread per system.
template <int NS, int NR>
struct MassActionModel {
    static constexpr int W = 1, PER = NS;
    using Ctx = MassActionNet;
    template <class R>
    struct Sys {
        const MassActionNet* net;
        R k[NR];
        int n;
        __device__ void load(const Ctx& ctx, const Team<W>&, double T, int neq) {
            net = &ctx;
            n = neq;
            // mixed form: log2 k in FP64 (a few operations per reaction), then
            // the fractional power of two in FP32 (accurate to an FP32 ulp)
            const double lnT = (sizeof(R) == 8) ? 0.0 : log(T);
            const double lnT64 = (sizeof(R) == 8) ? xm::log_series(T) : 0.0;
            const double invT = (sizeof(R) == 8) ? 0.0 : 1.0 / T;
#pragma unroll(NR <= 32 ? NR : 1)
            for (int j = 0; j < NR; ++j) {
                if (j < ctx.n_reactions) {
                    double kk;
                    if constexpr (sizeof(R) == 8) {
                        // A T^b exp(-Ea/T) with A = 10^log10A, as one series exponential
                        kk = xm::exp_series(xm::kLn10 * ctx.log10A[j] + ctx.beta[j] * lnT64 - ctx.Ea[j] / T);
                    } else {
                        const double l2 = (2.302585092994046 * ctx.log10A[j] + ctx.beta[j] * lnT - ctx.Ea[j] * invT) *
                                          1.4426950408889634;
                        const double li = floor(l2);
                        kk = (double)ldexpf(exp2f((float)(l2 - li)), (int)li);
                    }
                    kk = fmin(fmax(kk, ctx.kmin), ctx.kmax);
                    k[j] = (R)kk;
                } else {
                    k[j] = R(0);
                }
            }
        }
        __device__ int comp(const Team<W>&, int s) const { return s < n ? s : -1; }
        template <class T>
        __device__ T ordered_sum(const Team<W>&, const T* x) const {
            T acc = T(0);
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (s < n) acc = acc + x[s];
            return acc;
        }
        __device__ void rhs(const Team<W>&, R, const R* y, R* f) const {
            // gathers and scatters by species index go through small local arrays
            R c[NS], acc[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                c[s] = y[s];
                acc[s] = R(0);
            }
            const MassActionNet& nt = *net;
            // small networks: fully unrolled (rate constants stay in registers)
#pragma unroll(NR <= 32 ? NR : 1)
            for (int j = 0; j < NR; ++j) {
                if (j < nt.n_reactions) {
                    const int r0 = nt.reac[j][0];
                    R r = k[j] * c[r0];
                    const bool two = nt.n_reac[j] == 2;
                    const int r1 = nt.reac[j][1];
                    if (two) r = r * c[r1];
                    acc[r0] -= r;
                    if (two) acc[r1] -= r;
                    acc[nt.prod[j][0]] += r;
                    if (nt.n_prod[j] == 2) acc[nt.prod[j][1]] += r;
                }
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) f[s] = acc[s];
        }
        // row by row: J_sl accumulates, reaction by reaction, -dr_j/dC_l for
        // each reactant occurrence of s and +dr_j/dC_l for each product
        // occurrence, dr_j/dC_l summed over the reactant occurrences of l
        __device__ R gershgorin(const Team<W>&, const R* y) const {
            const MassActionNet& nt = *net;
            R g = R(0);
            for (int s = 0; s < n; ++s) {
                R J[NS];
                for (int l = 0; l < NS; ++l) J[l] = R(0);
                for (int j = 0; j < nt.n_reactions; ++j) {
                    const int nr = nt.n_reac[j];
                    int occ = 0;  // occurrences of s: reactant count, product count
                    for (int q = 0; q < nr; ++q) occ += nt.reac[j][q] == s;
                    int pocc = 0;
                    for (int q = 0; q < nt.n_prod[j]; ++q) pocc += nt.prod[j][q] == s;
                    if (occ == 0 && pocc == 0) continue;
                    R d[2];
                    d[0] = nr == 2 ? k[j] * y[nt.reac[j][1]] : k[j];
                    d[1] = k[j] * y[nt.reac[j][0]];
                    for (int l = 0; l < n; ++l) {
                        R dl = R(0);
                        bool any = false;
                        for (int q = 0; q < nr; ++q)
                            if (nt.reac[j][q] == l) {
                                dl = dl + d[q];
                                any = true;
                            }
                        if (!any) continue;
                        for (int q = 0; q < occ; ++q) J[l] = J[l] - dl;
                        for (int q = 0; q < pocc; ++q) J[l] = J[l] + dl;
                    }
                }
                R acc = R(0);
                for (int l = 0; l < n; ++l) acc = acc + rabs(J[l]);
                g = rmax(g, acc);
            }
            return g;
        }
    };
};

}  // namespace bode
