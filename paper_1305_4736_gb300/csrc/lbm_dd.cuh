// lbm_dd.cuh -- double-float arithmetic for the float64 mode on the float32 pipe.
//
// GB300 issues float32 FMAs at 128 lanes per SM cycle and float64 ones at about 1.7, so the
// float64 mode's step can run faster in double-float arithmetic: a value is an unevaluated sum
// hi + lo of two float32 numbers (48 significand bits), and each operation is built from
// error-free transformations on the float32 pipe (Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971; Knuth, TAOCP vol. 2, 4.2.2:
// TwoSum; Fast2Sum; the product error from an FMA).  Relative rounding of an operation is
// about 2^-47, against 2^-53 in float64.
//
// Values are kept unnormalised between operations: a sum or product returns the high part and
// its exact error plus the low parts, without the final Fast2Sum that would make
// |lo| <= ulp(hi) / 2.  The pair still holds the value to the same accuracy (lo stays within a
// few units of 2^-24 of the operands' magnitudes), and every operation here reads both parts,
// so only the places that look at hi alone renormalise first: the MC slope's comparisons and
// sign test, and the reciprocal's Newton step.  The populations stay float64 in HBM: a staged
// value is split into hi + lo (rounded to nearest) with integer operations, since
// float32 <-> float64 conversions run at the float64 rate on this part and the split is a phase
// of its own; an updated value is rounded back to float64 by the float64 pipe, which does that
// work beside the float32 arithmetic of the other warps.
//
// Every float32 operation here uses the _rn intrinsics, which the compiler neither contracts
// into FMAs nor reorders, so the transformations stay error-free.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct dd {
    float hi, lo;
};

// Host: the double-float value nearest to x (hi = x rounded to float, lo = the rest rounded).
inline dd dd_host(double x)
{
    const float h = (float)x;
    return dd{h, (float)(x - (double)h)};
}

__device__ __forceinline__ dd ddf(float h) { return dd{h, 0.0f}; }

// Fast2Sum (|a| >= |b| or a == 0): s + e = a + b exactly.
__device__ __forceinline__ dd fast2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b: TwoSum of the high parts, the low parts added to its error (8 operations).
__device__ __forceinline__ dd operator+(dd a, dd b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    return dd{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ dd operator-(dd a) { return dd{-a.hi, -a.lo}; }

__device__ __forceinline__ dd operator-(dd a, dd b)
{
    const float s = __fsub_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fsub_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fadd_rn(b.hi, v));
    return dd{s, __fadd_rn(e, __fsub_rn(a.lo, b.lo))};
}

// a * b: the product of the high parts and its exact error (from an FMA) plus the cross
// terms (4 operations).
__device__ __forceinline__ dd operator*(dd a, dd b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dd{p, e};
}

// a * c for a float32 constant c (3).
__device__ __forceinline__ dd operator*(dd a, float c)
{
    const float p = __fmul_rn(a.hi, c);
    float e = __fmaf_rn(a.hi, c, -p);
    e = __fmaf_rn(a.lo, c, e);
    return dd{p, e};
}
__device__ __forceinline__ dd operator*(float c, dd a) { return a * c; }

// a * 2^k (exact).
__device__ __forceinline__ dd scale2(dd a, float p2) { return dd{__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }

__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }

// a * b + c (12).
__device__ __forceinline__ dd fma_dd(dd a, dd b, dd c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(p, c.hi);
    const float v = __fsub_rn(s, p);
    const float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(c.hi, v));
    return dd{s, __fadd_rn(t, __fadd_rn(e, c.lo))};
}

// 1/x: the float32 approximate reciprocal y of x rounded to float (relative error below
// 2^-22), then one Newton step y + y (1 - x y) with 1 - x y formed in double-float and its two
// parts summed (the residual's high part alone can be of the size of its low part); relative
// error about 2^-44.
__device__ __forceinline__ dd recip(dd x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fadd_rn(x.hi, x.lo)));
    const dd r = ddf(1.0f) - x * y;
    return fast2sum(y, __fmul_rn(y, __fadd_rn(r.hi, r.lo)));
}

// The pair renormalised: |lo| <= ulp(hi) / 2 (Fast2Sum; with a low part larger than the high
// part, after a cancellation, it still returns the pair's value to within 2^-24 of that low part,
// far below the pair's own accuracy).
__device__ __forceinline__ dd norm(dd a) { return fast2sum(a.hi, a.lo); }

// Twice the MC slope, 2 minmod(2a, (a + b)/2, 2b) = sign(a) min(4|a|, 4|b|, |a + b|) when a and
// b agree in sign and 0 otherwise (Sec. III, reading A6); as mc2 of lbm_device.cuh.  a and b
// must be normalised (norm), so that their high parts carry their signs; they agree when
// a.hi b.hi > 0 (a product below 2^-149 counts as disagreement: then the smaller difference
// is below 2^-74, so the slope, at most 4 times it, is below 2^-72, far below the populations'
// 2^-47 resolution, and is taken as 0).  Two
// candidates x, y of the sign of a are ordered by the float32 value
// (x.hi - y.hi) + (x.lo - y.lo), whose sign is that of x - y (zero only for x = y or x, y within
// a few units of 2^-47 of each other, where either is the slope to the pairs' accuracy); the
// smaller magnitude is the lower value for a > 0 and the higher for a < 0.  The sum a + b is
// left unnormalised (its low part stays within a few units of its high part's last place,
// which the ordering tolerates).  Three float32 operations and a predicate per comparison;
// flipping the three pairs to magnitudes and comparing lexicographically took 4% more of the
// step.
__device__ __forceinline__ dd mc2n(dd a, dd b)
{
    const dd s = a + b;
    const bool agree = __fmul_rn(a.hi, b.hi) > 0.0f;
    const bool neg = a.hi < 0.0f;
    const float dab = __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
    const dd m = ((dab < 0.0f) != neg) ? a : b;
    const dd m4 = scale2(m, 4.0f);
    const float dms = __fadd_rn(__fsub_rn(m4.hi, s.hi), __fsub_rn(m4.lo, s.lo));
    return agree ? (((dms < 0.0f) != neg) ? m4 : s) : dd{0.0f, 0.0f};
}

// As mc2n, for pairs not yet normalised.
__device__ __forceinline__ dd mc2(dd a, dd b) { return mc2n(norm(a), norm(b)); }

// ---------------------------------------------------------------------------
// float64 -> double-float with integer operations, and back on the float64 pipe.
// ---------------------------------------------------------------------------
// x = hi + lo with hi = x rounded to 24 significand bits (half away from zero) and lo the rest
// rounded to float32 (|lo| <= 2^-25 |x|; the pair carries 48 of x's 53 bits, rounded to
// nearest).  |x| below 2^-74 (5.3e-23) is flushed to zero: populations here are O(1), so the
// absolute error stays below that.  Non-finite x and |x| >= 2^127 give +-inf or NaN in hi.
__device__ __forceinline__ dd dd_split(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned ex = (hw >> 20) & 0x7FFu;
    const unsigned sign = hw & 0x80000000u;
    // top 24 significand bits with the exponent rebiased (1023 -> 127); a carry from the
    // rounding increment moves into the exponent field, as it should
    unsigned fb = (((hw & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lw >> 29);
    const unsigned up = (lw >> 28) & 1u;
    fb += up;
    // remainder in units of 2^(ex - 1075): the low 29 bits, less 2^29 when hi was rounded up
    const int r = (int)(lw & 0x1FFFFFFFu) - (int)(up << 29);
    const float scale = __uint_as_float(((ex - 948u) & 0xFFu) << 23);   // 2^(ex - 1075) in range
    const float lo = __fmul_rn(__int2float_rn(r), scale);
    // selects, not branches: flushed, overflowing and non-finite inputs
    const bool tiny = ex < 949u, big = ex >= 1150u;
    const bool nan = ex == 2047u && ((hw & 0xFFFFFu) | lw) != 0u;
    const unsigned hbits = big ? (sign | 0x7F800000u | (nan ? 0x400000u : 0u)) : (fb | sign);
    return dd{tiny ? 0.0f : __uint_as_float(hbits),
              (tiny || big) ? 0.0f : __uint_as_float(__float_as_uint(lo) ^ sign)};
}

// hi + lo rounded to float64 (to nearest, ties to even): both parts convert to float64 exactly
// and one float64 addition rounds their sum.  These three operations run on the float64 pipe,
// which the step kernel leaves otherwise idle, alongside the float32 and integer work of the
// other warps; non-finite parts give +-inf or NaN.
__device__ __forceinline__ double dd_to_double(dd v)
{
    return __dadd_rn((double)v.hi, (double)v.lo);
}

}  // namespace lbm
