// xmath.cuh -- logarithm, exponential and power for the plain FP64 form.
//
// Series method (only correctly rounded operations, so the value does not
// depend on which library or compiler evaluates it; the translation units
// that use it are compiled without multiply-add contraction):
//   log: x = 2^e f, f in [sqrt(1/2), sqrt(2)); t = (f - 1) / (f + 1);
//        log f = 2 artanh t = 2 t sum_{i=0..11} t^(2i) / (2i + 1);
//        log x = e ln2_hi + (e ln2_lo + log f), ln 2 split after 32 bits.
//   exp: n = nearest integer to x / ln 2, r = (x - n ln2_hi) - n ln2_lo
//        (Cody-Waite), e^r = sum_{i=0..14} r^i / i! (Horner), times 2^n.
//   pow: x^y = exp(y log x), x > 0 (0 for x == 0, y > 0).
#pragma once
#include <cmath>

namespace bode {
namespace xm {

constexpr double kLn2Hi = 0.6931471806019545;        // ln 2 rounded to 32 significant bits
constexpr double kLn2Lo = -4.2009150726810846e-11;   // ln 2 - kLn2Hi
constexpr double kLog2e = 1.4426950408889634;
constexpr double kLn10 = 2.302585092994046;
constexpr double kSqrtHalf = 0.7071067811865476;

__device__ __forceinline__ double log_series(double x) {
    if (!(x > 0.0)) return x == 0.0 ? -INFINITY : NAN;
    if (isinf(x)) return x;
    int e;
    double f = frexp(x, &e);
    if (f < kSqrtHalf) {
        f = f * 2.0;
        e = e - 1;
    }
    const double t = (f - 1.0) / (f + 1.0);
    const double t2 = t * t;
    // 1/(2i+1) for i = 11 .. 1, Horner in t^2
    double q = 0.043478260869565216;
    q = q * t2 + 0.047619047619047616;
    q = q * t2 + 0.05263157894736842;
    q = q * t2 + 0.058823529411764705;
    q = q * t2 + 0.06666666666666667;
    q = q * t2 + 0.07692307692307693;
    q = q * t2 + 0.09090909090909091;
    q = q * t2 + 0.1111111111111111;
    q = q * t2 + 0.14285714285714285;
    q = q * t2 + 0.2;
    q = q * t2 + 0.3333333333333333;
    q = q * t2 + 1.0;
    const double logf = 2.0 * t * q;
    const double ed = (double)e;
    return ed * kLn2Hi + (ed * kLn2Lo + logf);
}

__device__ __forceinline__ double exp_series(double x) {
    if (isnan(x)) return x;
    if (x > 709.0) return INFINITY;
    if (x < -745.0) return 0.0;
    const double n = rint(x * kLog2e);
    const double r = (x - n * kLn2Hi) - n * kLn2Lo;
    // 1/i! for i = 14 .. 0, Horner in r
    double q = 1.1470745597729725e-11;
    q = q * r + 1.6059043836821613e-10;
    q = q * r + 2.08767569878681e-09;
    q = q * r + 2.505210838544172e-08;
    q = q * r + 2.755731922398589e-07;
    q = q * r + 2.7557319223985893e-06;
    q = q * r + 2.48015873015873e-05;
    q = q * r + 0.0001984126984126984;
    q = q * r + 0.001388888888888889;
    q = q * r + 0.008333333333333333;
    q = q * r + 0.041666666666666664;
    q = q * r + 0.16666666666666666;
    q = q * r + 0.5;
    q = q * r + 1.0;
    q = q * r + 1.0;
    return ldexp(q, (int)n);
}

__device__ __forceinline__ double pow_series(double x, double y) {
    if (x == 0.0) return y > 0.0 ? 0.0 : INFINITY;
    return exp_series(y * log_series(x));
}

}  // namespace xm
}  // namespace bode
