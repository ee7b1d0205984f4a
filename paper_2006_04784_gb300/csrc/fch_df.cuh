// fch_df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits. The FP64 pipe of
// this GPU runs at a small fraction of the FP32 rate; carrying FP64-class
// precision as float pairs keeps every operation on the FP32 pipe.
//
// Error-free transformations used (classical results, restated here):
//   TwoSum (Knuth): s = fl(a + b), e = (a - (s - b')) + (b - b'), b' = s - a, gives
//     a + b = s + e exactly for any floats a, b;
//   FastTwoSum (Dekker): for |a| >= |b|, s = fl(a + b), e = b - (s - a) is exact;
//   TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p), a b = p + e.
// Addition sums the high parts with TwoSum and the low parts with one rounding
// (error bounded relative to the operands); multiplication adds the cross terms to
// the exact product of the high parts; division refines a float quotient with two
// correction terms, the reciprocal takes one Newton step. Transcendental functions
// (used only by the q > 0 well and the ETD phi functions) go through double.
// Compile without fast-math: the transformations rely on IEEE rounding of each step.
#pragma once
#include <math.h>

namespace fch {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df(int i) : hi((float)i), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

struct __align__(16) df2 {
    df x, y;
};

// read-only loads of complex elements
__device__ __forceinline__ float2 ldg(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ df2 ldg(const df2 *p)
{
    const float4 v = __ldg((const float4 *)p);
    df2 r;
    r.x = df(v.x, v.y);
    r.y = df(v.z, v.w);
    return r;
}

// The sums and products of the transformations use the explicitly rounded intrinsics
// (__fadd_rn, __fsub_rn, __fmul_rn): the compiler never contracts those into fused
// multiply-adds, which would break the exactness these steps rely on (a product fused
// into the TwoSum that consumes it counts its rounding error twice).
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// Sums. The high parts are added exactly (TwoSum), the low parts with one rounding:
// an error of a few u^2 (|a| + |b|), u = 2^-24, relative to the operands rather
// than to a cancelled result. That is the norm-wise accuracy a transform's error
// analysis needs (its output error is bounded by eps log N times the input norm).
//
// The operators renormalise the sum (add_norm, 11 operations). add_lazy / sub_lazy
// leave it unrenormalised (8 operations): |lo| may exceed ulp(hi)/2, and after a
// cancellation of the high parts it may exceed |hi|; the transform butterflies use
// them and renormalise once where a transform ends (renorm restores |lo| <= ulp(hi)/2
// where |hi| >= |lo|, renorm_exact in every case). Whatever reads only the high
// word -- division, reciprocal, comparisons, signs -- renormalises its operands
// first with renorm_exact.
__device__ __forceinline__ df add_lazy(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return s;
}
__device__ __forceinline__ df sub_lazy(df a, df b)
{
    df s = two_sum(a.hi, -b.hi);
    s.lo += a.lo - b.lo;
    return s;
}
__device__ __forceinline__ df renorm(df a) { return fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ df renorm_exact(df a) { return two_sum(a.hi, a.lo); }
__device__ __forceinline__ df add_norm(df a, df b)
{
    const df s = add_lazy(a, b);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator+(df a, df b) { return add_norm(a, b); }
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return add_norm(a, -b); }

__device__ __forceinline__ df operator*(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// Product without the final renormalisation (4 operations instead of 7): the exact
// product of the high words and, in one error word, its rounding error and the two
// cross terms. The low word may exceed ulp(hi)/2 by a few units; sums and products
// take such operands (their error stays a few u^2 relative to the operands' size),
// and whatever reads only the high word renormalises first. A product neglects
// lo x lo: an operand whose high word cancelled in an unrenormalised difference (the
// value then sits in lo) is renormalised before it meets another such operand (a
// square of a small difference above all).
__device__ __forceinline__ df mul_lazy(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df(p, e);
}

// by +-1 (the DIR factors of the butterflies)
__device__ __forceinline__ df operator*(int s, df a) { return s < 0 ? -a : a; }

// Quotient by long division: three float quotient digits, each remainder
// renormalised before its leading word is read.
__device__ __forceinline__ df operator/(df a, df b)
{
    a = renorm_exact(a);
    b = renorm_exact(b);
    const float rb = 1.0f / b.hi;
    const float q1 = a.hi * rb;
    df r = renorm_exact(sub_lazy(a, b * df(q1, 0.f)));
    const float q2 = r.hi * rb;
    r = renorm_exact(sub_lazy(r, b * df(q2, 0.f)));
    const float q3 = r.hi * rb;
    const df q = fast_two_sum(q1, q2);
    return add_norm(q, df(q3, 0.f));
}

// Reciprocal by one Newton step from the float reciprocal r0 of the leading word:
// 1/d = r0 (1 + e) + O(e^2) with e = 1 - d r0 = O(2^-24), e formed to about 2^-48
// absolute (d.hi r0 split exactly by a fused multiply-add; 1 - p exact since p is
// within 2^-23 of 1), so the result carries a few u^2 relative error.
__device__ __forceinline__ df recip(df d)
{
    d = renorm_exact(d);
    const float r0 = 1.0f / d.hi;
    const float p = __fmul_rn(d.hi, r0);
    const float pe = fmaf(d.hi, r0, -p);
    const float e = ((1.0f - p) - pe) - d.lo * r0;
    return fast_two_sum(r0, r0 * e);
}
__device__ __forceinline__ float recip(float d) { return 1.0f / d; }
__device__ __forceinline__ double recip(double d) { return 1.0 / d; }

// a s for an exact power of two s (both words scale exactly; s.lo is 0)
__device__ __forceinline__ df mul_p2(df a, df s) { return df(a.hi * s.hi, a.lo * s.hi); }
__device__ __forceinline__ float mul_p2(float a, float s) { return a * s; }
__device__ __forceinline__ double mul_p2(double a, double s) { return a * s; }

// Complex product a w for a twiddle factor w, each part a sum of two products
// with one TwoSum: the high products are added exactly, their rounding errors
// (from fused multiply-adds) and the four cross terms with the low words go into
// one error word, left unrenormalised (16 operations a part instead of 25).
__device__ __forceinline__ df2 cmul_lazy(df2 a, df2 w)
{
    df2 r;
    {
        const float p1 = __fmul_rn(a.x.hi, w.x.hi), p2 = __fmul_rn(a.y.hi, w.y.hi);
        r.x = two_sum(p1, -p2);
        float e = fmaf(a.x.hi, w.x.hi, -p1) - fmaf(a.y.hi, w.y.hi, -p2);
        e = fmaf(a.x.hi, w.x.lo, e);
        e = fmaf(a.x.lo, w.x.hi, e);
        e = fmaf(-a.y.hi, w.y.lo, e);
        e = fmaf(-a.y.lo, w.y.hi, e);
        r.x.lo += e;
    }
    {
        const float p1 = __fmul_rn(a.x.hi, w.y.hi), p2 = __fmul_rn(a.y.hi, w.x.hi);
        r.y = two_sum(p1, p2);
        float e = fmaf(a.x.hi, w.y.hi, -p1) + fmaf(a.y.hi, w.x.hi, -p2);
        e = fmaf(a.x.hi, w.y.lo, e);
        e = fmaf(a.x.lo, w.y.hi, e);
        e = fmaf(a.y.hi, w.x.lo, e);
        e = fmaf(a.y.lo, w.x.hi, e);
        r.y.lo += e;
    }
    return r;
}

__device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }
__device__ __forceinline__ df &operator-=(df &a, df b) { return a = a - b; }
__device__ __forceinline__ df &operator*=(df &a, df b) { return a = a * b; }
__device__ __forceinline__ df &operator/=(df &a, df b) { return a = a / b; }

// comparisons (on renormalised operands)
__device__ __forceinline__ bool operator<(df a, df b)
{
    a = renorm_exact(a);
    b = renorm_exact(b);
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator==(df a, df b)
{
    a = renorm_exact(a);
    b = renorm_exact(b);
    return a.hi == b.hi && a.lo == b.lo;
}
__device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }

// float and double forms next to the double-float ones, so unqualified calls in
// namespace fch find every overload
__device__ __forceinline__ float fabs(float a) { return ::fabsf(a); }
__device__ __forceinline__ double fabs(double a) { return ::fabs(a); }
__device__ __forceinline__ float exp(float a) { return ::expf(a); }
__device__ __forceinline__ double exp(double a) { return ::exp(a); }
__device__ __forceinline__ float expm1(float a) { return ::expm1f(a); }
__device__ __forceinline__ double expm1(double a) { return ::expm1(a); }
__device__ __forceinline__ float copysign(float a, float b) { return ::copysignf(a, b); }
__device__ __forceinline__ double copysign(double a, double b) { return ::copysign(a, b); }

__device__ __forceinline__ df fabs(df a)
{
    a = renorm_exact(a);
    return a.hi < 0.f ? -a : a;
}
__device__ __forceinline__ df copysign(df a, df s)
{
    a = renorm_exact(a);
    s = renorm_exact(s);
    return (a.hi < 0.f) != (s.hi < 0.f) ? -a : a;
}
__device__ __forceinline__ df exp(df a) { return df(::exp((double)a)); }
__device__ __forceinline__ df expm1(df a) { return df(::expm1((double)a)); }

} // namespace fch
