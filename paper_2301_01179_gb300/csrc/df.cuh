// df.cuh -- FP32-pair ("double-float") arithmetic for FP64-class accuracy on the FP32 pipe.
//
// A value is hi + lo with two floats, |lo| <= ulp(hi)/2: 48 significant bits, relative
// rounding ~2^-47 per operation.  On GB300 an FP32 operation issues 61x faster than an
// FP64 one, so a df multiply (6 FP32 ops) or add (~10) costs a fraction of one FP64
// instruction.  The error-free transformations (Knuth's two-sum, the FMA two-product)
// use round-to-nearest intrinsics so the compiler cannot contract or reassociate them.
// The exponent range is FP32's; callers keep magnitudes well inside 1e-30..1e30.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace afmm {

struct dfv {
    float hi, lo;
};

__device__ __forceinline__ dfv df_make(float h, float l)
{
    dfv r;
    r.hi = h;
    r.lo = l;
    return r;
}

__device__ __forceinline__ dfv two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float v = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return df_make(s, e);
}

__device__ __forceinline__ dfv quick_two_sum(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

__device__ __forceinline__ dfv df_add(dfv a, dfv b)
{
    dfv s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, e);
}

__device__ __forceinline__ dfv df_neg(dfv a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ dfv df_sub(dfv a, dfv b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfv df_mul(dfv a, dfv b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}

// a * b - c: the product's exact error by FMA, one two-sum with -c.hi, one renormalisation
// (one rounding fewer than df_sub(df_mul(a, b), c))
__device__ __forceinline__ dfv df_fms(dfv a, dfv b, dfv c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fsub_rn(p, c.hi);
    const float v = __fsub_rn(s, p);
    const float err = __fsub_rn(__fsub_rn(p, __fsub_rn(s, v)), __fadd_rn(c.hi, v));  // (p - (s - v)) + (-c.hi - v)
    const float t = __fadd_rn(__fsub_rn(e, c.lo), err);
    return quick_two_sum(s, t);
}

__device__ __forceinline__ dfv df_mulf(dfv a, float b)
{
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}

// a * 2^k exactly (k small): scale both parts
__device__ __forceinline__ dfv df_scale2(dfv a, float p2) { return df_make(a.hi * p2, a.lo * p2); }

// a / b: FP32 quotient from the hardware reciprocal (MUFU, ~1 ulp), then one df residual
// correction; the residual step removes the approximation error of the first quotient
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ dfv df_div(dfv a, dfv b)
{
    float rb = rcp_approx(b.hi);
    float q1 = __fmul_rn(a.hi, rb);
    dfv r = df_sub(a, df_mulf(b, q1));
    float q2 = __fmul_rn(r.hi, rb);
    dfv q = quick_two_sum(q1, q2);
    // second correction for full df accuracy
    dfv r2 = df_sub(a, df_mul(b, q));
    return df_add(q, df_make(__fmul_rn(r2.hi, rb), 0.f));
}

// 1 / b: the FP32 reciprocal r0 of b.hi (MUFU, ~1 ulp) refined by one Newton step carrying
// the quadratic term, r = r0 + r0 (e + e^2) with e = 1 - b r0 (FMA-exact to 2^-47 of e), so
// the relative error is O(e^3 + 2^-47): the accuracy of df_div at a fifth of its operations
__device__ __forceinline__ dfv df_rcp(dfv b)
{
    const float r0 = rcp_approx(b.hi);
    float e = __fmaf_rn(-b.hi, r0, 1.0f);
    e = __fmaf_rn(-b.lo, r0, e);
    const float t = __fmul_rn(r0, __fmaf_rn(e, e, e));
    return quick_two_sum(r0, t);
}

// sqrt by one correction of an FP32 seed from the hardware reciprocal square root (Karp):
// x = rsqrt(a_hi), y = a_hi x, sqrt(a) ~ y + (a - y^2) x / 2
__device__ __forceinline__ dfv df_sqrt(dfv a)
{
    if (!(a.hi > 0.f)) return df_make(0.f, 0.f);
    float x = rsqrtf(a.hi);
    float y = __fmul_rn(a.hi, x);
    float p = __fmul_rn(y, y);
    float pe = __fmaf_rn(y, y, -p);
    float d = __fsub_rn(__fsub_rn(a.hi, p), pe);
    d = __fadd_rn(d, a.lo);
    return two_sum(y, __fmul_rn(d, __fmul_rn(0.5f, x)));
}

__device__ __forceinline__ double df_to_double(dfv a) { return (double)a.hi + (double)a.lo; }

// FP64 -> df with integer operations (the FP64<->FP32 conversions run on the FP64 pipe on
// GB300): hi keeps the top 24 bits of the significand (rounded), lo = v - hi is exact in
// FP64 and keeps the next 24.  Values outside the normal FP32 range fall back to the
// conversion instructions.
__device__ __forceinline__ float f64_to_f32_bits(double v, double &back)
{
    long long b = __double_as_longlong(v);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e < -125 || e > 126) {
        float f = __double2float_rn(v);
        back = (double)f;
        return f;
    }
    unsigned long long sgn = (unsigned long long)b & 0x8000000000000000ull;
    unsigned long long m = (unsigned long long)b & 0x000fffffffffffffull;
    unsigned long long m23 = (m + (1ull << 28)) >> 29;  // round to 23 fraction bits
    if (m23 == (1ull << 23)) {
        m23 = 0;
        ++e;
    }
    unsigned int fb = (unsigned int)(sgn >> 32) | ((unsigned int)(e + 127) << 23) | (unsigned int)m23;
    back = __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) | (m23 << 29)));
    return __uint_as_float(fb);
}

__device__ __forceinline__ dfv df_from_double(double v)
{
    // zero tests on the bit patterns (integer pipe, not the FP64 pipe)
    if ((__double_as_longlong(v) << 1) == 0) return df_make(0.f, 0.f);
    double hb;
    float h = f64_to_f32_bits(v, hb);
    double r = v - hb;  // exact
    double lb;
    float l = (__double_as_longlong(r) << 1) == 0 ? 0.f : f64_to_f32_bits(r, lb);
    return df_make(h, l);
}

// accumulate a * b into the (sum, error) pair (S, E): exact two-product and two-sum
__device__ __forceinline__ void df_acc(float &S, float &E, dfv a, dfv b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s = __fadd_rn(S, p);
    float v = __fsub_rn(s, S);
    float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, v)), __fsub_rn(p, v));
    E = __fadd_rn(E, __fadd_rn(err, pe));
    S = s;
}

// ---- two FP32-pair values per instruction (packed f32x2 arithmetic, sm_100 and later) ----
// A df2 holds two independent FP32 pairs: (hi.x, lo.x) and (hi.y, lo.y).  Each operation
// below performs, on both components, exactly the FP32 operations of its scalar
// counterpart above (same order, same roundings), so packed and scalar results are
// bitwise equal; one packed instruction issues the work of two FP32 instructions.
struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a), rb = *reinterpret_cast<unsigned long long *>(&b),
                       rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2 *>(&rd);
}
__device__ __forceinline__ float2 fneg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ df2 df2_make(float2 hi, float2 lo)
{
    df2 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
// (a, b) from two scalar pairs; the broadcast form (a, a)
__device__ __forceinline__ df2 df2_pack(dfv a, dfv b) { return df2_make(make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)); }
__device__ __forceinline__ df2 df2_bcast(dfv a) { return df2_pack(a, a); }
// float4 (x.hi, y.hi, x.lo, y.lo) <-> df2
__device__ __forceinline__ df2 df2_from4(float4 v) { return df2_make(make_float2(v.x, v.y), make_float2(v.z, v.w)); }
__device__ __forceinline__ float4 df2_to4(df2 v) { return make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y); }
__device__ __forceinline__ dfv df2_x(df2 v) { return df_make(v.hi.x, v.lo.x); }
__device__ __forceinline__ dfv df2_y(df2 v) { return df_make(v.hi.y, v.lo.y); }

__device__ __forceinline__ void quick_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = fadd2(a, b);
    e = fsub2(b, fsub2(s, a));
}

__device__ __forceinline__ df2 df2_add(df2 a, df2 b)
{
    const float2 s = fadd2(a.hi, b.hi);
    const float2 v = fsub2(s, a.hi);
    const float2 e = fadd2(fsub2(a.hi, fsub2(s, v)), fsub2(b.hi, v));
    const float2 t = fadd2(e, fadd2(a.lo, b.lo));
    df2 r;
    quick_two_sum2(s, t, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df2 df2_mul(df2 a, df2 b)
{
    const float2 p = fmul2(a.hi, b.hi);
    float2 e = ffma2(a.hi, b.hi, fneg2(p));
    e = ffma2(a.hi, b.lo, e);
    e = ffma2(a.lo, b.hi, e);
    df2 r;
    quick_two_sum2(p, e, r.hi, r.lo);
    return r;
}

// a * b + c componentwise, given nb = -b.hi: the product's exact error by FMA, one two-sum
// with c's high part, one renormalisation (one rounding fewer than df2_add(df2_mul(a, b), c))
__device__ __forceinline__ df2 df2_fma(df2 a, df2 b, float2 nb, df2 c)
{
    const float2 np = fmul2(a.hi, nb);  // -p, p = fl(a.hi b.hi)
    float2 e = ffma2(a.hi, b.hi, np);  // a.hi b.hi - p, exact
    e = ffma2(a.hi, b.lo, e);
    e = ffma2(a.lo, b.hi, e);
    const float2 s = fsub2(c.hi, np);  // c.hi + p
    const float2 v = fsub2(s, c.hi);
    const float2 err = fsub2(fsub2(c.hi, fsub2(s, v)), fadd2(np, v));  // (c.hi - (s - v)) + (p - v)
    const float2 t = fadd2(fadd2(e, c.lo), err);
    df2 r;
    quick_two_sum2(s, t, r.hi, r.lo);
    return r;
}

// (S, E) += a * b componentwise, as df_acc
__device__ __forceinline__ void df2_acc(float2 &S, float2 &E, df2 a, df2 b)
{
    const float2 p = fmul2(a.hi, b.hi);
    float2 pe = ffma2(a.hi, b.hi, fneg2(p));
    pe = ffma2(a.hi, b.lo, pe);
    pe = ffma2(a.lo, b.hi, pe);
    const float2 s = fadd2(S, p);
    const float2 v = fsub2(s, S);
    const float2 err = fadd2(fsub2(S, fsub2(s, v)), fsub2(p, v));
    E = fadd2(E, fadd2(err, pe));
    S = s;
}

// Negation-free forms.  np = -(a.hi * b.hi), formed by the caller from a negated operand
// (-a.hi * b.hi or a.hi * -b.hi, exact sign change under round-to-nearest).  df2_mul_np
// returns a * b as df2_mul does (p + e and its error, with s - p computed as s + np) and
// also -hi of the result, for products that feed df2_acc_np.
__device__ __forceinline__ df2 df2_mul_np(df2 a, df2 b, float2 np, float2 &nhi)
{
    float2 e = ffma2(a.hi, b.hi, np);  // a.hi b.hi - p, exact
    e = ffma2(a.hi, b.lo, e);
    e = ffma2(a.lo, b.hi, e);
    df2 r;
    r.hi = fsub2(e, np);               // p + e
    r.lo = fsub2(e, fadd2(r.hi, np));  // e - (s - p)
    nhi = fsub2(np, e);                // -(p + e)
    return r;
}

// a * b left unnormalised for a product that only feeds other pair products: hi = fl(a.hi
// b.hi) (= -np exactly, np given), lo = its exact error plus the cross terms (|lo| about
// 2^-23 |hi|; the dropped a.lo b.lo and the later lo * lo terms stay near 2^-46 of the
// product).  The negated high part is np itself.
__device__ __forceinline__ df2 df2_mul_nr(df2 a, df2 b, float2 np)
{
    float2 e = ffma2(a.hi, b.hi, np);  // a.hi b.hi - p, exact
    e = ffma2(a.hi, b.lo, e);
    e = ffma2(a.lo, b.hi, e);
    df2 r;
    r.hi = fmul2(a.hi, b.hi);
    r.lo = e;
    return r;
}

// df2_acc(S, E, a, b) given nbh = -b.hi: the same roundings, no negation
__device__ __forceinline__ void df2_acc_n(float2 &S, float2 &E, df2 a, df2 b, float2 nbh)
{
    const float2 np = fmul2(a.hi, nbh);  // -p
    float2 pe = ffma2(a.hi, b.hi, np);
    pe = ffma2(a.hi, b.lo, pe);
    pe = ffma2(a.lo, b.hi, pe);
    const float2 s = fsub2(S, np);  // S + p
    const float2 v = fsub2(s, S);
    const float2 err = fsub2(fsub2(S, fsub2(s, v)), fadd2(np, v));  // (S - (s - v)) + (p - v)
    E = fadd2(E, fadd2(err, pe));
    S = s;
}

// a * b + c * d componentwise, given na = -a.hi and nc = -c.hi: both products with their
// exact errors (FMA), one two-sum of the high parts (in negated form, exact under
// round-to-nearest), the low parts added, one renormalisation; returns the sum and sets
// nhi = -(its high part)
__device__ __forceinline__ df2 df2_dot2_np(df2 a, float2 na, df2 b, df2 c, float2 nc, df2 d, float2 &nhi)
{
    const float2 np1 = fmul2(na, b.hi);  // -p1
    float2 e1 = ffma2(a.hi, b.hi, np1);  // a.hi b.hi - p1, exact
    e1 = ffma2(a.hi, b.lo, e1);
    e1 = ffma2(a.lo, b.hi, e1);
    const float2 np2 = fmul2(nc, d.hi);  // -p2
    float2 e2 = ffma2(c.hi, d.hi, np2);
    e2 = ffma2(c.hi, d.lo, e2);
    e2 = ffma2(c.lo, d.hi, e2);
    const float2 ns = fadd2(np1, np2);  // -(p1 + p2), rounded
    const float2 v = fsub2(ns, np1);
    const float2 nerr = fadd2(fsub2(np1, fsub2(ns, v)), fsub2(np2, v));  // -(p1 + p2 - s)
    const float2 lo = fsub2(fadd2(e1, e2), nerr);
    df2 r;
    r.hi = fsub2(lo, ns);                  // s + lo
    r.lo = fsub2(lo, fadd2(r.hi, ns));     // lo - (hi - s)
    nhi = fsub2(ns, lo);
    return r;
}

}  // namespace afmm
