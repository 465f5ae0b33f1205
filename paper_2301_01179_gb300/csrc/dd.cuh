// dd.cuh -- double-double ("FP64 pair") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 106 significant bits.  Knuth's two-sum and the FMA two-product are the exact
// error-free transformations; the operations below are the usual compositions of them
// (Dekker 1971; Hida, Li and Bailey 2001).  Used where FP64 rounding is amplified: the
// Legendre start values and the base columns of the Taylor coefficients (farfield.cu).
#pragma once
#include <cuda_runtime.h>

namespace afmm {

struct ddv {
    double hi, lo;
};

__device__ __forceinline__ ddv dd_make(double h, double l = 0.0)
{
    ddv r;
    r.hi = h;
    r.lo = l;
    return r;
}

// s + e = a + b exactly
__device__ __forceinline__ ddv dd_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return dd_make(s, e);
}

// the same when |a| >= |b|
__device__ __forceinline__ ddv dd_quick_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    return dd_make(s, __dsub_rn(b, __dsub_rn(s, a)));
}

// p + e = a * b exactly
__device__ __forceinline__ ddv dd_two_prod(double a, double b)
{
    const double p = __dmul_rn(a, b);
    return dd_make(p, __fma_rn(a, b, -p));
}

__device__ __forceinline__ ddv dd_neg(ddv a) { return dd_make(-a.hi, -a.lo); }

__device__ __forceinline__ ddv dd_add(ddv a, ddv b)
{
    ddv s = dd_two_sum(a.hi, b.hi);
    const ddv t = dd_two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = dd_quick_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return dd_quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ddv dd_sub(ddv a, ddv b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ ddv dd_add_d(ddv a, double b)
{
    ddv s = dd_two_sum(a.hi, b);
    s.lo = __dadd_rn(s.lo, a.lo);
    return dd_quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ddv dd_mul(ddv a, ddv b)
{
    ddv p = dd_two_prod(a.hi, b.hi);
    p.lo = __fma_rn(a.hi, b.lo, __fma_rn(a.lo, b.hi, p.lo));
    return dd_quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ddv dd_mul_d(ddv a, double b)
{
    ddv p = dd_two_prod(a.hi, b);
    p.lo = __fma_rn(a.lo, b, p.lo);
    return dd_quick_two_sum(p.hi, p.lo);
}

// acc + a * b, the product's errors carried into the low word before one renormalisation
__device__ __forceinline__ ddv dd_fma(ddv a, ddv b, ddv acc)
{
    const ddv p = dd_two_prod(a.hi, b.hi);
    const double cross = __fma_rn(a.hi, b.lo, __dmul_rn(a.lo, b.hi));
    ddv s = dd_two_sum(acc.hi, p.hi);
    s.lo = __dadd_rn(s.lo, __dadd_rn(__dadd_rn(acc.lo, p.lo), cross));
    return dd_quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ddv dd_div(ddv a, ddv b)
{
    const double q1 = a.hi / b.hi;
    ddv r = dd_sub(a, dd_mul_d(b, q1));
    const double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    const double q3 = r.hi / b.hi;
    return dd_add_d(dd_quick_two_sum(q1, q2), q3);
}

__device__ __forceinline__ ddv dd_div_d(ddv a, double b)
{
    const double q1 = a.hi / b;
    ddv r = dd_sub(a, dd_two_prod(q1, b));
    const double q2 = r.hi / b;
    r = dd_sub(r, dd_two_prod(q2, b));
    const double q3 = r.hi / b;
    return dd_add_d(dd_quick_two_sum(q1, q2), q3);
}

// square root: the FP64 root and one Newton correction from the exact residual
__device__ __forceinline__ ddv dd_sqrt(ddv a)
{
    if (!(a.hi > 0.0)) return dd_make(0.0);
    const double x = sqrt(a.hi);
    const ddv r = dd_sub(a, dd_two_prod(x, x));
    return dd_quick_two_sum(x, r.hi / (2.0 * x));
}

}  // namespace afmm

namespace afmm {

// 1 / d for an integer-valued d as a double-double: the FP64 quotient and its FMA residual
__device__ __forceinline__ ddv dd_recip_int(double d)
{
    const double h = 1.0 / d;
    const double r = __fma_rn(-h, d, 1.0);  // 1 - h d, exact
    return dd_quick_two_sum(h, r * h);
}

// ---- triple-float: x0 + x1 + x2, three FP32 words (about 72 significant bits), for sums of
// products on the FP32 pipe where FP64 rounding would be amplified (GB300 issues FP64 at 1/64
// of FP32).  Products are split exactly by the FP32 FMA; sums of high words by two-sum.
struct tfv {
    float x0, x1, x2;
};

__device__ __forceinline__ void tf_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a double-double split into three FP32 words (the remainder is below 2^-72 of the value)
__device__ __forceinline__ tfv tf_from_dd(ddv v)
{
    tfv t;
    t.x0 = __double2float_rn(v.hi);
    const ddv r0 = dd_add_d(v, -(double)t.x0);
    t.x1 = __double2float_rn(r0.hi);
    const ddv r1 = dd_add_d(r0, -(double)t.x1);
    t.x2 = __double2float_rn(r1.hi);
    return t;
}

__device__ __forceinline__ ddv tf_to_dd(tfv t)
{
    return dd_add_d(dd_two_sum((double)t.x0, (double)t.x1), (double)t.x2);
}

// accumulator of a sum of products: s0 collects the high products by two-sum, s1 the words
// of weight ~2^-24 (rounding residues of s0, product errors, cross products) by two-sum,
// s2 the words of weight ~2^-48 in plain FP32
struct tfacc {
    float s0, s1, s2;
};

__device__ __forceinline__ tfacc tfacc_zero()
{
    tfacc A;
    A.s0 = A.s1 = A.s2 = 0.f;
    return A;
}

// A += a * b
__device__ __forceinline__ void tf_acc(tfacc &A, const tfv &a, const tfv &b)
{
    const float p = __fmul_rn(a.x0, b.x0), e = __fmaf_rn(a.x0, b.x0, -p);
    const float q1 = __fmul_rn(a.x0, b.x1), f1 = __fmaf_rn(a.x0, b.x1, -q1);
    const float q2 = __fmul_rn(a.x1, b.x0), f2 = __fmaf_rn(a.x1, b.x0, -q2);
    const float l2 = __fmaf_rn(a.x0, b.x2, __fmaf_rn(a.x1, b.x1, __fmaf_rn(a.x2, b.x0, __fadd_rn(f1, f2))));
    float s, r, t, r1, r2, r3, r4;
    tf_two_sum(A.s0, p, s, r);
    tf_two_sum(A.s1, r, t, r1);
    tf_two_sum(t, e, t, r2);
    tf_two_sum(t, q1, t, r3);
    tf_two_sum(t, q2, t, r4);
    A.s0 = s;
    A.s1 = t;
    A.s2 = __fadd_rn(A.s2, __fadd_rn(__fadd_rn(__fadd_rn(r1, r2), __fadd_rn(r3, r4)), l2));
}

__device__ __forceinline__ ddv tfacc_to_dd(const tfacc &A)
{
    return dd_add_d(dd_two_sum((double)A.s0, (double)A.s1), (double)A.s2);
}

}  // namespace afmm

namespace afmm {

// double-double sum of products: high products by two-sum into H, all low words summed in L
struct ddacc {
    double H, L;
};

// number types of the base-column convolutions in farfield.cu: triple-float on the FP32 pipe
// (about 2^-68 of the summed magnitudes) or double-double on the FP64 pipe (about 2^-104)
template <bool DD>
struct BaseNum;

template <>
struct BaseNum<false> {
    using S = tfv;
    using A = tfacc;
    static __device__ __forceinline__ S from(ddv v) { return tf_from_dd(v); }
    static __device__ __forceinline__ ddv to(const S &s) { return tf_to_dd(s); }
    static __device__ __forceinline__ double nearest(const S &s)
    {
        return ((double)s.x0 + (double)s.x1) + (double)s.x2;
    }
    static __device__ __forceinline__ A zero() { return tfacc_zero(); }
    static __device__ __forceinline__ void acc(A &a, const S &x, const S &y) { tf_acc(a, x, y); }
    static __device__ __forceinline__ ddv fin(const A &a) { return tfacc_to_dd(a); }
};

template <>
struct BaseNum<true> {
    using S = ddv;
    using A = ddacc;
    static __device__ __forceinline__ S from(ddv v) { return v; }
    static __device__ __forceinline__ ddv to(const S &s) { return s; }
    static __device__ __forceinline__ double nearest(const S &s) { return s.hi; }
    static __device__ __forceinline__ A zero()
    {
        A a;
        a.H = a.L = 0.0;
        return a;
    }
    static __device__ __forceinline__ void acc(A &a, const S &x, const S &y)
    {
        const ddv p = dd_two_prod(x.hi, y.hi);
        const double cross = __fma_rn(x.hi, y.lo, __dmul_rn(x.lo, y.hi));
        const ddv s = dd_two_sum(a.H, p.hi);
        a.L = __dadd_rn(a.L, __dadd_rn(__dadd_rn(s.lo, p.lo), cross));
        a.H = s.hi;
    }
    static __device__ __forceinline__ ddv fin(const A &a) { return dd_quick_two_sum(a.H, a.L); }
};

}  // namespace afmm
