// Float-float ("double-float") arithmetic for the FP64-accuracy residuals of
// the mixed-precision solvers.
//
// On this GPU an FP64 fused multiply-add issues at about 1/60 of the FP32
// rate, so the FP64 hopping operator is bound by its arithmetic, not by
// memory.  A float-float value is the unevaluated sum hi + lo of two floats
// (about 48 significant bits, FP32 exponent range); its arithmetic costs ten
// to twenty FP32 operations per FP64 one, which still leaves it several
// times faster than FP64 here while reading the same bytes.
//
// Building blocks (error-free transformations, all published):
//   TwoSum      s + e == a + b exactly              (Knuth, TAOCP vol. 2, 4.2.2)
//   FastTwoSum  the same when |a| >= |b|            (Dekker, Numer. Math. 18, 1971)
//   TwoProduct  p + e == a * b exactly, through FMA (Ogita, Rump, Oishi,
//               SIAM J. Sci. Comput. 26, 2005)
// The round-to-nearest intrinsics keep the compiler from contracting the
// additions and products these identities rely on into FMAs.
#pragma once

#include "plq_fields.cuh"

namespace plq {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b, renormalised (the error of the high parts and both low parts are
// folded into the new low part)
__device__ __forceinline__ df operator+(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    const df t = two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
    return t;
}
__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }

// a + b without the final renormalisation: the error of the high parts and
// both low parts go into lo (8 operations instead of 14).  |lo| may grow to a
// few ulp(hi); sums of a handful of terms stay accurate to ~2^-48 of their
// inputs, and renorm() restores |lo| <= ulp(hi)/2.
__device__ __forceinline__ df add_lazy(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ df renorm(df a) { return two_sum(a.hi, a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

// a * b (the lo * lo term is below the format's precision)
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// Split of a double into hi = rn(d) and lo = rn(d - hi).
__device__ __forceinline__ df df_from_double(double d) {
    const float hi = __double2float_rn(d);
    return {hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// The same split of d * 2^es from the bit fields, for the bulk conversion
// kernels: a double -> float conversion issues on this GPU's FP64 pipe (as
// slow as an FP64 add), integer and FP32 operations do not.  hi keeps the
// sign, the (shifted) exponent and the top 23 mantissa bits of d
// (truncated); lo is the remaining 29-bit tail rounded to a float, so
// hi + lo = d 2^es to 2^-48 |d 2^es| and |lo| < ulp(hi).  The power-of-two
// shift lets callers bring fields of any magnitude into the FP32 exponent
// range; values still outside it (Inf, NaN, extreme exponents) take the
// conversion path, with sc = 2^es as a double.
__device__ __forceinline__ df df_from_double_bits(double d, int es, double sc) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int de = (int)((b >> 52) & 0x7ff);
    const int fe = de - 1023 + 127 + es;  // FP32 biased exponent of d 2^es
    if ((b << 1) == 0ull) return {__uint_as_float(sign), 0.f};  // +-0
    if (de == 0 || de == 0x7ff || fe < 1 || fe > 254) return df_from_double(d * sc);
    const unsigned long long m = b & 0xfffffffffffffull;
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(m >> 29));
    // tail * 2^(e - 52) = tail * 2^-52 * 2^(fe - 127); each factor is a normal float
    float lo = __fmul_rn(__uint2float_rn((unsigned)(m & 0x1fffffffu)), 2.220446049250313e-16f);
    lo = __fmul_rn(lo, __uint_as_float((unsigned)fe << 23));
    return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

// Accumulator of a sum of products: s collects the high parts through TwoSum,
// e every rounding error and low-order term (one renormalisation at the end).
struct dacc {
    float s, e;
};

// A = x * y (first term of a sum)
__device__ __forceinline__ dacc dacc_prod(df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return {p, e};
}

// A += x * y
__device__ __forceinline__ void dacc_fma(dacc &A, df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    const df t = two_sum(A.s, p);
    A.s = t.hi;
    A.e = __fadd_rn(A.e, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ df dacc_value(dacc A) { return two_sum(A.s, A.e); }

}  // namespace plq
