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
