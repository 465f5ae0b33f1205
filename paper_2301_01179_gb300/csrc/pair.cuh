// pair.cuh -- the modal Green's function G^(n)(r, r1, x), n = 0..N, for one (field point,
// source) pair in FP64 (Eq. analysis:gfunc; Appendix A Eqs. gfunc:recursion, gfunc:Q0).
//
// Start values.  With rho_pm^2 = (r +- r1)^2 + x^2, Gauss's arithmetic-geometric mean
// M = AGM(rho_+, rho_-) gives the ring potential directly:
//     G^(0) = Q_{-1/2}(chi) / (2 pi sqrt(r r1)) = 1 / (2 M)
// (Q_{-1/2} = mu K(mu), K = pi / (2 AGM(1, k')), mu = 2 sqrt(r r1) / rho_+, k' = rho_-/rho_+).
// With c_1 = (rho_+ - rho_-)/2, c_{m+1} = (a_m - b_m)/2 the AGM half-differences, Legendre's
// E = K (1 - sum_{m>=0} 2^{m-1} c_m^2 / rho_+^2) turns Q_{1/2} = chi mu K - (1+chi) mu E into
//     G^(1) = G^(0) * sum_{m>=1} 2^{m-1} c_m^2 / (2 r r1)
// with no cancellation (every term is positive).
//
// Recursion.  Eq. gfunc:recursion in the scaled variable y_n = G_n / c_n (see RecTab):
// forward y_n = gam_n chi y_{n-1} - y_{n-2} where the forward direction is stable
// (2 N acosh chi <= fwd_switch and acosh chi <= 0.96), otherwise Miller's backward
// recursion from (y_L, y_{L-1}) = (0, tiny), L = N + ceil(miller_extra / acosh chi) + 2,
// normalised by the known G^(0).  Both regimes run as one loop body so that a warp whose
// lanes disagree on the regime executes max(N, L) steps, not N + L.
#pragma once
#include "common.cuh"

namespace afmm {

struct PairGeom {
    double x;      // z_field - z_source
    double rm2;    // rho_-^2 (replaced by rho_+^2 for coincident / inactive pairs)
    double rp2;    // rho_+^2
    double chi;    // 1 + rho_-^2 / (2 r r1)
    double zero;   // 0 for a coincident or inactive pair, 1 otherwise
};

__device__ __forceinline__ void pair_geom(double rt, double zt, double r1, double z1, double inv2w, bool active,
                                          PairGeom &g)
{
    double x = zt - z1, dr = rt - r1, sr = rt + r1;
    double rm2 = fma(dr, dr, x * x);
    double rp2 = fma(sr, sr, x * x);
    bool coinc = !(rm2 > 0.0) || !active;
    g.zero = coinc ? 0.0 : 1.0;
    if (coinc) rm2 = rp2;
    g.x = x;
    g.rm2 = rm2;
    g.rp2 = rp2;
    g.chi = fma(rm2, inv2w, 1.0);
}

// Runs the start values and the recursion for one pair; writes y_n (n = 0..N) to
// ys[n * stride] and returns the factor s with G_n = s * c_n * ys[n].
// gam: recursion table (shared memory copy), N: highest mode.
__device__ __forceinline__ double pair_sequence(const PairGeom &g, double inv2w, int N, const PairParams &pp,
                                                const double *__restrict__ gam, double *ys, int stride)
{
    // regime decision in FP32 (only selects an algorithm; both are accurate)
    float tf = (float)(g.chi - 1.0);
    float af = log1pf(tf + sqrtf(tf * (tf + 2.0f)));  // acosh(chi)
    int Nr = N < 1 ? 1 : N;
    bool fwd = (2.0f * (float)Nr * af <= (float)pp.fwd_switch) && (af <= 0.96f);
    // AGM of (rho_+, rho_-) with the half-difference sum for G^(1)
    double a = sqrt(g.rp2), b = sqrt(g.rm2);
    double csum = 0.0, w = 1.0;
    for (int it = 0; it < 40; ++it) {
        double c = 0.5 * (a - b);
        csum = fma(w * c, c, csum);
        w *= 2.0;
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
        if (c <= 1.5e-8 * a) break;
    }
    double G0 = 0.5 / a;
    // unified sweep: forward lanes go up from (y0, y1), Miller lanes go down from (0, tiny)
    int L = N + 2;
    if (!fwd) {
        float lf = ceilf((float)pp.miller_extra / fmaxf(af, 1e-6f));
        int ext = lf > (float)(AFMM_REC_TAB) ? AFMM_REC_TAB : (int)lf;
        L = N + ext + 2;
        if (L > AFMM_REC_TAB - 1) L = AFMM_REC_TAB - 1;
    }
    double y0, y1;
    if (fwd) {
        y0 = G0;
        y1 = G0 * csum * inv2w;
        ys[0] = y0;
        if (N >= 1) ys[stride] = y1;
    } else {
        y0 = 0.0;     // y_L
        y1 = 1e-280;  // y_{L-1}
    }
    int steps = fwd ? N - 1 : L - 1;
    // warp-uniform trip count (lanes past their own count idle through the body)
    int smax = steps;
    for (int o = 16; o > 0; o >>= 1) smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    double chi = g.chi;
    for (int s = 0; s < smax; ++s) {
        if (s < steps) {
            int n = fwd ? s + 2 : L - s;           // forward: y_n from y_{n-1}, y_{n-2}
            double yn = fma(gam[n] * chi, y1, -y0); // backward: y_{n-2} from y_{n-1}, y_n
            y0 = y1;
            y1 = yn;
            int idx = fwd ? n : n - 2;
            if (idx <= N) ys[idx * stride] = yn;
            if (!fwd && (__double2hiint(yn) & 0x7ff00000) > 0x73d00000) {  // |y| > ~1e250
                y0 *= 1e-250;
                y1 *= 1e-250;
                for (int m = idx; m <= N; ++m)
                    if (m >= 0) ys[m * stride] *= 1e-250;
            }
        }
    }
    if (fwd) return g.zero;
    return g.zero * (G0 / ys[0]);
}

}  // namespace afmm
