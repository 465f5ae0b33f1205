// pair_df.cuh -- the per-pair modal Green's function sequence of pair.cuh, in FP32-pair
// (double-float) arithmetic: same start values (G^(0) = 1/(2 AGM(rho_+, rho_-)), G^(1) from
// the AGM half-difference sum), same scaled Legendre recursion (Eq. gfunc:recursion), same
// forward / Miller choice, ~48-bit precision.  The cancelling coordinate differences r - r1
// and z - z1 (and r + r1) come from exact FP32 triples of the coordinates by error-free
// FP32 sums, so the kernels issue no FP64 arithmetic per pair.
//
// Precision budget: the forward sweep's rounding grows like exp(n acosh chi) while Q_{n-1/2}
// decays like exp(-n acosh chi); measured against the pair's G^(0) (the scale of the
// max-normalised per-mode error) the error is ~2^-47 N exp(s/2) / s with s = 2 N acosh chi,
// which the forward switch df_fwd_switch (s <= 8) keeps near 1e-12; pairs beyond it use
// Miller's sweep.
#pragma once
#include "common.cuh"
#include "df.cuh"

namespace afmm {

struct PairDF {
    dfv x;     // z_field - z_source
    dfv dr;    // r - r1
    dfv sr;    // r + r1
    dfv rm2;   // rho_-^2 (rho_+^2 for coincident / inactive pairs)
    dfv rp2;   // rho_+^2
    dfv chi;   // 1 + rho_-^2 / (2 r r1)
    float t;   // chi - 1 (FP32, regime decision only)
    float zero;
};

// (a0 + a1 + a2) + (b0 + b1 + b2) as an FP32 pair, for exact FP32 triples of coordinates:
// the high and middle words by exact two-sums, the rest summed in FP32.  When the high words
// cancel (Sterbenz), the pair holds the difference to ~2^-47 of itself plus ~2^-72 of the
// coordinates: the accuracy of the FP64 difference split into a pair, without FP64 work.
__device__ __forceinline__ dfv sum_f32x3(float a0, float a1, float a2, float b0, float b1, float b2)
{
    const dfv p = two_sum(a0, b0);
    const dfv q = two_sum(a1, b1);
    const dfv h = two_sum(p.hi, q.hi);
    const float l = __fadd_rn(__fadd_rn(p.lo, q.lo), __fadd_rn(h.lo, __fadd_rn(a2, b2)));
    return quick_two_sum(h.hi, l);
}

// pair_geom_df from the exact FP32 triples of the sorted points (tg: the field point's two
// float4, sg: the source's; layout (r0, r1, z0, z1), (r2, z2, 1/r hi, 1/r lo))
__device__ __forceinline__ void pair_geom_f32x3(const float4 tg0, const float4 tg1, const float4 sg0,
                                                const float4 sg1, dfv inv2w, bool active, PairDF &g)
{
    g.x = sum_f32x3(tg0.z, tg0.w, tg1.y, -sg0.z, -sg0.w, -sg1.y);
    g.dr = sum_f32x3(tg0.x, tg0.y, tg1.x, -sg0.x, -sg0.y, -sg1.x);
    g.sr = sum_f32x3(tg0.x, tg0.y, tg1.x, sg0.x, sg0.y, sg1.x);
    dfv x2 = df_mul(g.x, g.x);
    dfv rm2 = df_add(df_mul(g.dr, g.dr), x2);
    dfv rp2 = df_add(df_mul(g.sr, g.sr), x2);
    bool coinc = !(rm2.hi > 0.f) || !active;
    g.zero = coinc ? 0.f : 1.f;
    if (coinc) rm2 = rp2;
    g.rm2 = rm2;
    g.rp2 = rp2;
    dfv t = df_mul(rm2, inv2w);
    g.t = t.hi;
    g.chi = df_add(df_make(1.f, 0.f), t);
}

// The sequence of one lane in a slot of the near-field ring: y_n at mode pair n / 2 of a
// [pair][32 lanes] float4 array (y_2m.hi, y_2m+1.hi, y_2m.lo, y_2m+1.lo), so that a
// consumer loads two modes of one pair as one packed operand.  y points at the lane's
// float4 of pair 0.
struct SeqSlot {
    float *y;
    __device__ __forceinline__ void put(int n, dfv v) const
    {
        float *e = y + (n >> 1) * 128 + (n & 1);
        e[0] = v.hi;
        e[2] = v.lo;
    }
    __device__ __forceinline__ dfv get(int n) const
    {
        const float *e = y + (n >> 1) * 128 + (n & 1);
        return df_make(e[0], e[2]);
    }
};

// Regime of the sweep (Appendix A): forward iff 2 N acosh(chi) <= fwd_switch (and
// acosh(chi) <= 0.96), else Miller's backward sweep.
__device__ __forceinline__ float acosh_chi(float t) { return log1pf(t + sqrtf(t * (t + 2.0f))); }  // t = chi - 1

// the same test on t = chi - 1 against tlim = min(cosh(fwd_switch / (2 max(N, 1))), cosh(0.96)) - 1
// (host-side), without the logarithm
__device__ __forceinline__ bool pair_forward(float t, float tlim) { return t <= tlim; }

// AGM of (rho_+, rho_-) with the half-difference sum csum for G^(1) (Eq. gfunc:Q0 and the
// start values of Appendix A); returns the mean a: G^(0) = 1 / (2 a)
__device__ __forceinline__ dfv pair_agm_df(const PairDF &g, dfv &csum)
{
    dfv a = df_sqrt(g.rp2), b = df_sqrt(g.rm2);
    csum = df_make(0.f, 0.f);
    float w = 1.f;
    for (int it = 0; it < 40; ++it) {
        dfv c = df_scale2(df_sub(a, b), 0.5f);
        csum = df_add(csum, df_scale2(df_mul(c, c), w));
        w *= 2.f;
        dfv an = df_scale2(df_add(a, b), 0.5f);
        b = df_sqrt(df_mul(a, b));
        a = an;
        if (c.hi <= 1e-7f * a.hi) break;
    }
    return a;
}

// The sweep of the scaled recursion (Eq. gfunc:recursion) from the start values G0 and
// csum: writes y_n (n = 0..N) into the slot and returns the factor s with G_n = s c_n y_n
// times zero (0 for a pair that must not contribute).  With FOLD the backward lanes apply
// s in place, so that the slot holds y_n = G_n / c_n on every lane (a forward lane's s is
// 1) and the return value is not needed.  gam2: recursion constants gam_n as FP32 pairs,
// gam4 the same by mode pair (shared memory).
//
// Forward lanes: two steps per iteration, gam_n chi and gam_{n+1} chi as one packed
// product, one 16-byte store per mode pair; every lane of a warp that has a forward lane
// runs it (a backward lane's values, possibly overflowing, are overwritten by its own
// sweep).  Backward lanes (Miller): from y_L = 0, y_{L-1} = 2^-e (e ~ the sweep's growth in
// bits, at most 100) down to y_0, rescaled exactly by 2^-100 whenever |y| passes 2^60,
// then normalised in place by G0 / y_0.  The start is
// L = max(N + 2, N / 2 + ceil(extra / acosh chi) + 2): the relative error of y_n,
// e^{-2 a (L - n)} (a = acosh chi), is then below e^{-2 extra} measured against the
// pair's G^(0), since |G^(n) / G^(0)| ~ e^{-n a}.
template <bool FOLD>
__device__ __forceinline__ dfv pair_sweep_df(dfv chi, float t, float zero, dfv inv2w, int N, bool fwd, float extra,
                                             dfv G0, dfv csum, const float2 *__restrict__ gam2,
                                             const float4 *__restrict__ gam4, const SeqSlot ys)
{
    const bool allf = __all_sync(0xffffffffu, fwd);
    if (allf || __any_sync(0xffffffffu, fwd)) {
        float4 *yp = reinterpret_cast<float4 *>(ys.y);
        dfv ym2 = G0, ym1 = df_mul(df_mul(G0, csum), inv2w);
        if (N == 0) ym1 = df_make(0.f, 0.f);  // pad of pair 0
        yp[0] = make_float4(ym2.hi, ym1.hi, ym2.lo, ym1.lo);
        const df2 CHI = df2_bcast(chi);
        int n = 2;
        for (; n + 1 <= N; n += 2) {
            const df2 GC = df2_mul(df2_from4(gam4[n >> 1]), CHI);
            const dfv ya = df_fms(df2_x(GC), ym1, ym2);
            const dfv yb = df_fms(df2_y(GC), ya, ym1);
            yp[(n >> 1) * 32] = make_float4(ya.hi, yb.hi, ya.lo, yb.lo);
            ym2 = ya;
            ym1 = yb;
        }
        if (n == N) {  // N even: the last mode alone, with the pad
            const dfv ya = df_fms(df_mul(df_make(gam2[n].x, gam2[n].y), chi), ym1, ym2);
            yp[(n >> 1) * 32] = make_float4(ya.hi, 0.f, ya.lo, 0.f);
        }
        if (allf) return df_make(zero, 0.f);
    }
    // a forward lane's zero is 1: a pair that must not contribute (coincident, or a padding
    // source) has chi - 1 >= 2 and takes the backward branch
    if (fwd) return df_make(zero, 0.f);
    // backward lane
    const float af = acosh_chi(t);
    const float lf = ceilf(extra / fmaxf(af, 1e-6f) - 0.5f * (float)N);  // L - N - 2 >= extra / a - N / 2
    const int ext = lf < 0.f ? 0 : (lf > (float)AFMM_REC_TAB ? AFMM_REC_TAB : (int)lf);
    int L = N + ext + 2;
    if (L > AFMM_REC_TAB - 1) L = AFMM_REC_TAB - 1;
    // y_L = 0, y_{L-1} = 2^-e with e ~ log2 of the sweep's growth e^{a (L - 1)} (at most 100),
    // so that y_0 ends near 1 and the normalisation G0 / y_0 (which multiplies the gradient
    // factors) stays far inside the FP32 range; a power of two scales the whole sweep exactly
    const int e2 = (int)fminf(100.f, rintf(af * (float)(L - 1) * 1.44269504f));
    dfv y0 = df_make(0.f, 0.f);
    dfv y1 = df_make(__int_as_float((127 - e2) << 23), 0.f);
    for (int n = L; n >= 2; --n) {
        const float2 gm = gam2[n];
        const dfv yn = df_fms(df_mul(df_make(gm.x, gm.y), chi), y1, y0);  // y_{n-2}
        y0 = y1;
        y1 = yn;
        const int idx = n - 2;
        if (idx <= N) ys.put(idx, yn);
        // above 2^60: rescale by 2^-100 (exact); the margin 2^68 to the FP32 range covers the
        // growth of one step, ~2 chi, up to chi ~ 1e20 (points near the axis)
        if (fabsf(yn.hi) > 1.1529215e18f) {
            const float s100 = 7.8886091e-31f;
            y0 = df_scale2(y0, s100);
            y1 = df_scale2(y1, s100);
            for (int m = idx; m <= N; ++m) ys.put(m, df_scale2(ys.get(m), s100));
        }
    }
    const dfv y0n = ys.get(0);
    dfv sc = df_div(G0, y0n);
    sc = df_make(sc.hi * zero, sc.lo * zero);
    if (FOLD)
        for (int m = 0; m <= N; ++m) ys.put(m, df_mul(ys.get(m), sc));
    return sc;
}

}  // namespace afmm
