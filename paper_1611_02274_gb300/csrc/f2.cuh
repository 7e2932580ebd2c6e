// f2.cuh -- two-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is carried as an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, which gives about 48 significant bits.  The
// operations are the classical error-free transformations:
//   two_sum (Knuth, TAOCP vol. 2, Sec. 4.2.2): s = fl(a + b) and the exact
//           rounding error e, a + b = s + e, in six additions;
//   fast_two_sum (Dekker 1971): the same in three additions when |a| >= |b|;
//   two_prod: p = fl(a b) and e = a b - p exactly, by one fused multiply-add.
// Sums and products of pairs combine these as in Dekker's double-length
// arithmetic: the leading words exactly, the trailing words to FP32
// accuracy, then one renormalisation.  The relative error of a product is
// a few units of 2^-48; a sum's absolute error is a few units of 2^-48
// times |a| + |b|, so heavy cancellation (production and consumption rates
// of one species) loses nothing beyond that.
//
// On this GPU the FP64 pipe runs at 1/64 of the FP32 rate; a two-float
// product costs 7 FP32 instructions and a sum 11, so state, stages and
// right-hand sides in two-float arithmetic keep nearly FP64 accuracy at a
// fraction of the FP64 cost.
//
// The compiler must not reassociate these sequences (nvcc does not without
// fast-math flags); contractions into fused multiply-adds are harmless:
// every multiply that matters is an explicit fmaf.
#pragma once

namespace bode {

struct F2 {
    float hi, lo;
    F2() = default;
    __host__ __device__ constexpr F2(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr F2(float x) : hi(x), lo(0.0f) {}
    __host__ __device__ constexpr F2(int x) : hi((float)x), lo(0.0f) {}  // small integers are exact
    // nearest pair to a double (two roundings; exact for |d| in FP32 range
    // up to the 48-bit width)
    __host__ __device__ F2(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return F2(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = a + b;
    return F2(s, b - (s - a));
}

__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    const F2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.hi, -a.lo); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return a + (-b); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 operator*(F2 a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 operator*(float a, F2 b) { return b * a; }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = a * b; }
// the pair is normalised, so the leading words order it unless they tie
__device__ __forceinline__ bool operator<(F2 a, F2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(F2 a, F2 b) { return b < a; }
__device__ __forceinline__ bool operator<=(F2 a, F2 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(F2 a, F2 b) { return !(a < b); }

__device__ __forceinline__ F2 rabs(F2 x) { return x.hi < 0.0f ? -x : x; }
__device__ __forceinline__ F2 rmax(F2 a, F2 b) { return a < b ? b : a; }
__device__ __forceinline__ float to_float(F2 x) { return x.hi + x.lo; }
__device__ __forceinline__ double to_double(F2 x) { return (double)x.hi + (double)x.lo; }

// Unnormalised forms.  A pair whose trailing word may exceed half an ulp of
// the leading one (by a few ulp) is still an exact-enough input to the
// operations above, so a product or sum that feeds another two-float
// operation can skip its renormalisation (three instructions):
//   mul_lazy(a, b)  the two_prod of the leading words plus both cross terms;
//   add_lazy(a, b)  two_sum of the leading words, trailing words added to
//                   its error (repeated lazy sums collect every rounding
//                   error in the trailing word, whose own rounding is
//                   ~2^-48 of the terms);
//   normalize(a)    one fast_two_sum, back to |lo| <= ulp(hi) / 2.
// For float and double these are the plain operations, so code written
// with them computes exactly what it computed with * and + before.
__device__ __forceinline__ F2 mul_lazy(F2 a, F2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return F2(p, e);
}
__device__ __forceinline__ F2 add_lazy(F2 a, F2 b) {
    const F2 s = two_sum(a.hi, b.hi);
    return F2(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ F2 normalize(F2 a) { return fast_two_sum(a.hi, a.lo); }
template <class T>
__device__ __forceinline__ T mul_lazy(T a, T b) { return a * b; }
template <class T>
__device__ __forceinline__ T add_lazy(T a, T b) { return a + b; }
template <class T>
__device__ __forceinline__ T normalize(T a) { return a; }

// Accumulation of a right-hand side's terms (generated network code):
// acc_first_sub / acc_first_add start an accumulator from its first term
// (0 - r and 0 + r in the plain forms, the values an accumulator started at
// zero takes), acc_add / acc_sub are lazy sums, acc_value the normalised
// result.
template <class T>
__device__ __forceinline__ T acc_first_sub(T r) { return T(0) - r; }
__device__ __forceinline__ F2 acc_first_sub(F2 r) { return -r; }
template <class T>
__device__ __forceinline__ T acc_first_add(T r) { return T(0) + r; }
__device__ __forceinline__ F2 acc_first_add(F2 r) { return r; }
template <class T>
__device__ __forceinline__ T acc_add(T a, T r) { return add_lazy(a, r); }
template <class T>
__device__ __forceinline__ T acc_sub(T a, T r) { return add_lazy(a, -r); }
template <class T>
__device__ __forceinline__ T acc_value(T a) { return normalize(a); }

// Per-system constants of a right-hand side (e.g. rate constants): an
// array in registers for the plain and FP32 forms; for the two-float forms,
// whose pairs would take twice the registers, a row of the block's shared
// memory that the integrator binds (SMEM_FLOATS floats per thread, an odd
// number of pairs so that a half-warp's 8-byte loads fall in distinct
// banks).
template <class R, int N>
struct ConstStore {
    static constexpr int SMEM_FLOATS = 0;
    R v[N];
    __device__ R& operator[](int j) { return v[j]; }
    __device__ const R& operator[](int j) const { return v[j]; }
    __device__ void bind(float*) {}
};
template <int N>
struct ConstStore<F2, N> {
    static constexpr int SMEM_FLOATS = 2 * (N | 1);
    F2* v;
    __device__ F2& operator[](int j) { return v[j]; }
    __device__ const F2& operator[](int j) const { return v[j]; }
    __device__ void bind(float* row) { v = reinterpret_cast<F2*>(row); }
};

// warp shuffles of a pair (both words from the same lane)
__device__ __forceinline__ F2 shfl_xor(unsigned m, F2 v, int o, int w) {
    return F2(__shfl_xor_sync(m, v.hi, o, w), __shfl_xor_sync(m, v.lo, o, w));
}
__device__ __forceinline__ F2 shfl_idx(unsigned m, F2 v, int s, int w) {
    return F2(__shfl_sync(m, v.hi, s, w), __shfl_sync(m, v.lo, s, w));
}
__device__ __forceinline__ F2 shfl_up(unsigned m, F2 v, int d, int w) {
    return F2(__shfl_up_sync(m, v.hi, d, w), __shfl_up_sync(m, v.lo, d, w));
}
__device__ __forceinline__ F2 shfl_down(unsigned m, F2 v, int d, int w) {
    return F2(__shfl_down_sync(m, v.hi, d, w), __shfl_down_sync(m, v.lo, d, w));
}
__device__ __forceinline__ F2 vmax(F2 a, F2 b) { return rmax(a, b); }

}  // namespace bode
