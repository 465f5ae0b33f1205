// nearfield.cu -- direct sums of S^(n) G^(n) over (field point, source) pairs (Eq.
// analysis:sum): the FMM's near field over the 3x3 neighbour leaves (the D list, Sec. 2.2;
// Algorithm 1 last step, together with the local expansion of Eq. analysis:local), and the
// all-pairs direct evaluation.
//
// AFMM_FP64 and AFMM_MIXED run k_near_ws: warp-specialised blocks (producer warps compute
// the pairs' Legendre sequences into a ring of shared-memory slots, consumer warps own a
// range of modes and accumulate), FP32-pair arithmetic on the FP32 pipe, packed f32x2 mode
// pairs in the accumulation.  AFMM_FP64_NATIVE runs the FP64 kernels k_near / k_near2
// (one warp per work unit, per-mode accumulators in shared memory).
#include <cstring>
#include "common.cuh"
#include "pair.cuh"
#include "pair_df.cuh"
#include "mbar.cuh"

namespace afmm {

struct NearArgs {
    // field role (sorted)
    const double *fr, *fz;
    int64_t nfield;
    // source role (sorted), amplitudes [nmodes][nsrc] pre-multiplied by c_n
    const double *sr, *sz, *q_re, *q_im;
    // FP32-pair kernel: sorted coordinates as exact FP32 triples with 1 / r as an FP32 pair,
    // [n][2] float4 (r0, r1, z0, z1), (r2, z2, 1/r hi, 1/r lo); field role and source role
    const float4 *geo_f, *geo_s;
    int64_t nsrc;
    int nmodes, N;
    // work
    const NearUnit *units;
    int64_t nunits;
    const int32_t *nbr;  // [nbox][9] (near mode)
    const int2 *srng;    // source-role ranges per leaf (near mode)
    // adaptive tree (near mode): the unit's source-role ranges are nl_rng[nl_off[g] ..
    // nl_off[g + 1]) with g = nl_base[level] + box; the L2P takes the leaf's key and locals
    // from its level's tables
    const int64_t *nl_off;
    const int2 *nl_rng;
    int64_t nl_base[AFMM_MAX_LEVEL + 1];
    const uint32_t *lv_key[AFMM_MAX_LEVEL + 1];
    const float2 *lv_locd_re[AFMM_MAX_LEVEL + 1], *lv_locd_im[AFMM_MAX_LEVEL + 1];
    const float *lv_loc32_re[AFMM_MAX_LEVEL + 1], *lv_loc32_im[AFMM_MAX_LEVEL + 1];
    double side;         // the domain square's side (box size h = side / 2^level)
    int direct;          // 1: all sources, split into nsplit chunks
    int nsplit;
    int64_t split_len;
    // FP64 path in FP32 pairs: amplitudes per source by mode pair, re then im,
    // [nsrc][n / 2][2] float4 (q_2m.hi, q_2m+1.hi, q_2m.lo, q_2m+1.lo); leaf locals as (hi, lo)
    const float4 *qdf;
    const float2 *locdf_re, *locdf_im;
    float df_fwd_switch;
    float df_tlim;  // forward iff chi - 1 <= df_tlim (the switch on t = chi - 1)
    // MIXED precision: FP32 amplitudes per source by mode pair, [nsrc][n / 2] float4
    // (re_2m, re_2m+1, im_2m, im_2m+1), FP32 local expansions, compensated FP32 sums
    const float4 *q32;
    const float *loc32_re, *loc32_im;
    int mode_lo, mode_hi;  // FP32-pair kernel: the modes [mode_lo, mode_hi) of this launch
    int *err;              // plan error word (bounded waits that ran out)
    int accumulate;        // FP32-pair kernel: add to the outputs (k_l2p wrote the local expansion)
    int inject_timeout;    // test hook: slot 0 is never handed over
    // local expansion at the leaves (near mode, optional)
    const double *loc_re, *loc_im;
    const uint32_t *leaf_key;
    int M, ncoef;
    double r0, z0, h;
    // outputs (caller layout [nmodes][nfield] through out_perm, or split partials)
    const int32_t *out_perm;
    double *o_re, *o_im, *o_dr_re, *o_dr_im, *o_dz_re, *o_dz_im;
    double *part;  // split partials [nsplit][ncomp][nmodes][nfield]
    PairParams pp;
};

// Local expansion value and gradient at offset (u, v) in box units (locals stored as plain
// scaled Taylor coefficients F_kl = h^{k+l} Phi_kl, index k(M+1) - k(k-1)/2 + l).
template <bool GRAD>
__device__ __forceinline__ void l2p_eval(const double *__restrict__ F, int M, double u, double v, double &val,
                                         double &du, double &dv)
{
    double pu = 0.0, pdu = 0.0, pdv = 0.0;
    for (int k = M; k >= 0; --k) {
        int base = k * (M + 1) - k * (k - 1) / 2;
        double pk = 0.0, pkd = 0.0;
        for (int l = M - k; l >= 0; --l) {
            if (GRAD) pkd = fma(pkd, v, pk);
            pk = fma(pk, v, F[base + l]);
        }
        if (GRAD) {
            pdu = fma(pdu, u, pu);
            pdv = fma(pdv, u, pkd);
        }
        pu = fma(pu, u, pk);
    }
    val = pu;
    du = pdu;
    dv = pdv;
}

template <bool GRAD>
__global__ void __launch_bounds__(AFMM_NEAR_WARPS * 32) k_near(const NearArgs a, const RecTab tab)
{
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int nm = a.nmodes, N = a.N;
    double *gam = smem;                    // [AFMM_REC_TAB]
    double *rho = gam + AFMM_REC_TAB;      // [nm] c_{n-1}/c_n
    const int ncomp = GRAD ? 6 : 2;
    double *wbase = rho + AFMM_MAX_MODES + (size_t)warp * ((ncomp + 1) * nm + 1) * 32;
    double *acc = wbase;                   // [ncomp][nm][32]
    double *ys = wbase + (size_t)ncomp * nm * 32;  // [nm + 1][32]
    const int Nq = GRAD && N < 1 ? 1 : N;          // the gradient of mode 0 needs G^(1)
    for (int i = threadIdx.x; i < AFMM_REC_TAB; i += blockDim.x) gam[i] = tab.gam[i];
    for (int i = threadIdx.x; i < nm; i += blockDim.x) rho[i] = i == 0 ? 1.0 : tab.c[i - 1] / tab.c[i];
    __syncthreads();

    const int64_t unit = (int64_t)blockIdx.x * nw + warp;
    if (unit >= a.nunits) return;
    int64_t t0, t1, split = 0;
    int box = -1;
    if (a.direct) {
        int64_t tu = unit / a.nsplit;
        split = unit % a.nsplit;
        t0 = tu * 32;
        t1 = min(t0 + 32, a.nfield);
    } else {
        NearUnit u = a.units[unit];
        box = u.box;
        t0 = u.begin;
        t1 = u.end;
    }
    const int64_t t = t0 + lane;
    const bool active = t < t1;
    const int64_t tc = active ? t : t0;
    const double rt = a.fr[tc], zt = a.fz[tc];
    const double inv2r = 0.5 / rt;

    for (int c = 0; c < ncomp; ++c)
        for (int n = 0; n < nm; ++n) acc[((size_t)c * nm + n) * 32 + lane] = 0.0;

    // source ranges: 9 neighbour leaves, or one split of all sources
    int nrange = a.direct ? 1 : 9;
    for (int rg = 0; rg < nrange; ++rg) {
        int64_t s0, s1;
        if (a.direct) {
            s0 = split * a.split_len;
            s1 = min(s0 + a.split_len, a.nsrc);
        } else {
            int32_t nb = a.nbr[(int64_t)box * 9 + rg];
            if (nb < 0) continue;
            int2 r = a.srng[nb];
            s0 = r.x;
            s1 = r.y;
        }
        for (int64_t s = s0; s < s1; ++s) {
            const double r1 = a.sr[s], z1 = a.sz[s];
            const double inv2w = inv2r / r1;
            PairGeom g;
            pair_geom(rt, zt, r1, z1, inv2w, true, g);  // a lane past the last target: never written
            double sc = pair_sequence(g, inv2w, Nq, a.pp, gam, ys + lane, 32);
            if (!GRAD) {
                for (int n = 0; n < nm; ++n) {
                    double gn = sc * ys[n * 32 + lane];
                    double qr = a.q_re[(size_t)n * a.nsrc + s], qi = a.q_im[(size_t)n * a.nsrc + s];
                    acc[(size_t)n * 32 + lane] = fma(qr, gn, acc[(size_t)n * 32 + lane]);
                    acc[((size_t)nm + n) * 32 + lane] = fma(qi, gn, acc[((size_t)nm + n) * 32 + lane]);
                }
            } else {
                // dG_n/dx = nu_n x W_n, dG_n/dr = -G_n/(2r) + nu_n (r^2 - r1^2 - x^2)/(2r) W_n,
                // W_n = G_n A + G_{n-1} B, A = 1/rho_+^2 + 1/rho_-^2, B = 1/rho_+^2 - 1/rho_-^2,
                // G_{-1} = G_1 (Appendix A).  nu_n and 1/(2r) are applied per field point.
                double inv = 1.0 / (g.rp2 * g.rm2);
                double ip = g.rm2 * inv, im = g.rp2 * inv;
                double A = ip + im, B = ip - im;
                double qfac = fma(rt - r1, rt + r1, -g.x * g.x);
                double yprev = ys[32 + lane];  // y_{-1} := y_1 (G^(-1) = G^(1), c_1 = 1)
                for (int n = 0; n < nm; ++n) {
                    double yn = ys[n * 32 + lane];
                    double gn = sc * yn;
                    double wt = sc * fma(yn, A, rho[n] * yprev * B);
                    yprev = yn;
                    double xw = g.x * wt, qw = qfac * wt;
                    double qr = a.q_re[(size_t)n * a.nsrc + s], qi = a.q_im[(size_t)n * a.nsrc + s];
                    size_t o = (size_t)n * 32 + lane, st = (size_t)nm * 32;
                    acc[o] = fma(qr, gn, acc[o]);
                    acc[o + st] = fma(qi, gn, acc[o + st]);
                    acc[o + 2 * st] = fma(qr, qw, acc[o + 2 * st]);
                    acc[o + 3 * st] = fma(qi, qw, acc[o + 3 * st]);
                    acc[o + 4 * st] = fma(qr, xw, acc[o + 4 * st]);
                    acc[o + 5 * st] = fma(qi, xw, acc[o + 5 * st]);
                }
            }
        }
    }
    if (!active) return;
    // local expansion at the field point (far field)
    double u = 0.0, v = 0.0;
    if (a.loc_re) {
        uint32_t k = a.leaf_key[box];
        double cr = a.r0 + ((double)morton_ir(k) + 0.5) * a.h, cz = a.z0 + ((double)morton_iz(k) + 0.5) * a.h;
        u = (rt - cr) / a.h;
        v = (zt - cz) / a.h;
    }
    const int64_t dst = a.out_perm ? a.out_perm[t] : t;
    const size_t st = (size_t)nm * 32;
    for (int n = 0; n < nm; ++n) {
        // (amplitudes carry c_n and the sequence is G_n / c_n, so the sums are plain)
        size_t o = (size_t)n * 32 + lane;
        double c0 = acc[o], c1 = acc[o + st], c2 = 0, c3 = 0, c4 = 0, c5 = 0;
        if (GRAD) {
            c2 = acc[o + 2 * st];
            c3 = acc[o + 3 * st];
            c4 = acc[o + 4 * st];
            c5 = acc[o + 5 * st];
        }
        double pr = c0, pi = c1;
        double dr_r = 0, dr_i = 0, dz_r = 0, dz_i = 0;
        if (GRAD) {
            double nu = n - 0.5;
            dr_r = (nu * c2 - pr) * inv2r;
            dr_i = (nu * c3 - pi) * inv2r;
            dz_r = nu * c4;
            dz_i = nu * c5;
        }
        if (a.loc_re) {
            const double *Fr = a.loc_re + ((size_t)box * nm + n) * a.ncoef;
            const double *Fi = a.loc_im + ((size_t)box * nm + n) * a.ncoef;
            double vr, dur, dvr, vi, dui, dvi;
            l2p_eval<GRAD>(Fr, a.M, u, v, vr, dur, dvr);
            l2p_eval<GRAD>(Fi, a.M, u, v, vi, dui, dvi);
            pr += vr;
            pi += vi;
            if (GRAD) {
                double ih = 1.0 / a.h;
                dr_r += dur * ih;
                dr_i += dui * ih;
                dz_r += dvr * ih;
                dz_i += dvi * ih;
            }
        }
        if (a.part) {
            size_t base = (size_t)split * ncomp;
            size_t nfm = (size_t)a.nfield;
            a.part[((base + 0) * nm + n) * nfm + t] = pr;
            a.part[((base + 1) * nm + n) * nfm + t] = pi;
            if (GRAD) {
                a.part[((base + 2) * nm + n) * nfm + t] = dr_r;
                a.part[((base + 3) * nm + n) * nfm + t] = dr_i;
                a.part[((base + 4) * nm + n) * nfm + t] = dz_r;
                a.part[((base + 5) * nm + n) * nfm + t] = dz_i;
            }
        } else {
            size_t od = (size_t)n * a.nfield + dst;
            if (a.o_re) a.o_re[od] = pr;
            if (a.o_im) a.o_im[od] = pi;
            if (GRAD) {
                a.o_dr_re[od] = dr_r;
                a.o_dr_im[od] = dr_i;
                a.o_dz_re[od] = dz_r;
                a.o_dz_im[od] = dz_i;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Cooperative near-field kernel: the WB warps of a block share one unit of <= 32 field
// points.  Sources are taken WB at a time: in phase 1 warp w evaluates the pair sequence of
// source w of the chunk for all 32 field points and leaves it in shared memory; in phase 2
// warp w accumulates its contiguous share of the modes over the chunk's sources.  Each lane
// thus holds accumulators for nm / WB modes instead of nm, which lifts occupancy from 3 to
// 8 warps per SM (FP64 with gradient, N = 32) so the FP64 pipe stays busy.
// ------------------------------------------------------------------------------------
#define NEAR2_WB 4

template <bool GRAD>
__global__ void __launch_bounds__(NEAR2_WB * 32) k_near2(const NearArgs a, const RecTab tab)
{
    extern __shared__ double smem[];
    constexpr int WB = NEAR2_WB;
    constexpr int NPP = GRAD ? 5 : 1;  // per-pair scalars: scale (, x, qfac, A, B)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nm = a.nmodes, N = a.N;
    const int Nq = GRAD && N < 1 ? 1 : N;
    const int nmq = Nq + 1;                     // sequence rows per pair
    const int ncomp = GRAD ? 6 : 2;
    const int mper = (nm + WB - 1) / WB;        // modes per warp
    double *gam = smem;                         // [AFMM_REC_TAB]
    double *rho = gam + AFMM_REC_TAB;           // [AFMM_MAX_MODES] c_{n-1}/c_n
    double *ys = rho + AFMM_MAX_MODES;          // [WB][nmq][32]
    double *pp = ys + (size_t)WB * nmq * 32;    // [WB][NPP][32]
    double *acc = pp + (size_t)WB * NPP * 32;   // [WB][ncomp][mper][32]
    __shared__ int rb[10], rcum[10];
    for (int i = threadIdx.x; i < AFMM_REC_TAB; i += blockDim.x) gam[i] = tab.gam[i];
    for (int i = threadIdx.x; i < nm; i += blockDim.x) rho[i] = i == 0 ? 1.0 : tab.c[i - 1] / tab.c[i];

    const int64_t unit = blockIdx.x;
    int64_t t0, t1, split = 0;
    int box = -1;
    if (a.direct) {
        int64_t tu = unit / a.nsplit;
        split = unit % a.nsplit;
        t0 = tu * 32;
        t1 = min(t0 + 32, a.nfield);
    } else {
        NearUnit u = a.units[unit];
        box = u.box;
        t0 = u.begin;
        t1 = u.end;
    }
    // source ranges (flattened): 9 neighbour leaves, or one split of all sources
    if (threadIdx.x == 0) {
        int cum = 0;
        if (a.direct) {
            int64_t s0 = split * a.split_len, s1 = min(s0 + a.split_len, a.nsrc);
            rb[0] = (int)s0;
            rcum[0] = 0;
            cum = (int)(s1 > s0 ? s1 - s0 : 0);
            for (int k = 1; k < 10; ++k) {
                rb[k] = 0;
                rcum[k] = cum;
            }
        } else {
            for (int k = 0; k < 9; ++k) {
                int32_t nb = a.nbr[(int64_t)box * 9 + k];
                int2 r = nb >= 0 ? a.srng[nb] : make_int2(0, 0);
                rb[k] = r.x;
                rcum[k] = cum;
                cum += r.y - r.x;
            }
            rb[9] = 0;
            rcum[9] = cum;
        }
    }
    const int64_t t = t0 + lane;
    const bool active = t < t1;
    const int64_t tc = active ? t : t0;
    const double rt = a.fr[tc], zt = a.fz[tc];
    const double inv2r = 0.5 / rt;
    double *myacc = acc + (size_t)warp * ncomp * mper * 32;
    for (int i = lane; i < ncomp * mper * 32; i += 32) myacc[i] = 0.0;
    const int n0 = warp * mper, n1 = min(nm, n0 + mper);
    __syncthreads();
    const int total = rcum[9];
    for (int c0 = 0; c0 < total; c0 += WB) {
        // ---- phase 1: warp w evaluates source c0 + w for the unit's field points
        const int k = c0 + warp;
        if (k < total) {
            int rg = 0;
            while (rg < 8 && rcum[rg + 1] <= k) ++rg;
            const int64_t s = rb[rg] + (k - rcum[rg]);
            const double r1 = a.sr[s], z1 = a.sz[s];
            const double inv2w = inv2r / r1;
            PairGeom g;
            pair_geom(rt, zt, r1, z1, inv2w, true, g);  // a lane past the last target: never written
            double *yw = ys + (size_t)warp * nmq * 32;
            double sc = pair_sequence(g, inv2w, Nq, a.pp, gam, yw + lane, 32);
            double *pw = pp + (size_t)warp * NPP * 32;
            pw[lane] = sc;
            if (GRAD) {
                double inv = 1.0 / (g.rp2 * g.rm2);
                double ip = g.rm2 * inv, im = g.rp2 * inv;
                pw[32 + lane] = g.x;
                pw[64 + lane] = fma(rt - r1, rt + r1, -g.x * g.x);
                pw[96 + lane] = sc * (ip + im);  // scaled A
                pw[128 + lane] = sc * (ip - im); // scaled B
            }
        }
        __syncthreads();
        // ---- phase 2: warp w accumulates modes [n0, n1) over the chunk's sources
        const int kmax = min(WB, total - c0);
        for (int kk = 0; kk < kmax; ++kk) {
            const int kq = c0 + kk;
            int rg = 0;
            while (rg < 8 && rcum[rg + 1] <= kq) ++rg;
            const int64_t s = rb[rg] + (kq - rcum[rg]);
            const double *yk = ys + (size_t)kk * nmq * 32;
            const double *pk = pp + (size_t)kk * NPP * 32;
            const double sc = pk[lane];
            double gx = 0, qf = 0, As = 0, Bs = 0, yprev = 0;
            if (GRAD) {
                gx = pk[32 + lane];
                qf = pk[64 + lane];
                As = pk[96 + lane];
                Bs = pk[128 + lane];
                yprev = n0 == 0 ? yk[32 + lane] : yk[(n0 - 1) * 32 + lane];  // y_{-1} := y_1
            }
            for (int n = n0; n < n1; ++n) {
                const double yn = yk[n * 32 + lane];
                const size_t o = (size_t)(n - n0) * 32 + lane, st = (size_t)mper * 32;
                double qr = a.q_re[(size_t)n * a.nsrc + s], qi = a.q_im[(size_t)n * a.nsrc + s];
                double gn = sc * yn;
                myacc[o] = fma(qr, gn, myacc[o]);
                myacc[o + st] = fma(qi, gn, myacc[o + st]);
                if (GRAD) {
                    double wt = fma(yn, As, rho[n] * yprev * Bs);
                    yprev = yn;
                    double xw = gx * wt, qw = qf * wt;
                    myacc[o + 2 * st] = fma(qr, qw, myacc[o + 2 * st]);
                    myacc[o + 3 * st] = fma(qi, qw, myacc[o + 3 * st]);
                    myacc[o + 4 * st] = fma(qr, xw, myacc[o + 4 * st]);
                    myacc[o + 5 * st] = fma(qi, xw, myacc[o + 5 * st]);
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    double u = 0.0, v = 0.0;
    if (a.loc_re) {
        uint32_t kk = a.leaf_key[box];
        double cr = a.r0 + ((double)morton_ir(kk) + 0.5) * a.h, cz = a.z0 + ((double)morton_iz(kk) + 0.5) * a.h;
        u = (rt - cr) / a.h;
        v = (zt - cz) / a.h;
    }
    const int64_t dst = a.out_perm ? a.out_perm[t] : t;
    const size_t st = (size_t)mper * 32;
    for (int n = n0; n < n1; ++n) {
        size_t o = (size_t)(n - n0) * 32 + lane;
        double c[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < ncomp; ++q)
            c[q] = myacc[o + q * st];
        double pr = c[0], pi = c[1];
        double dr_r = 0, dr_i = 0, dz_r = 0, dz_i = 0;
        if (GRAD) {
            double nu = n - 0.5;
            dr_r = (nu * c[2] - pr) * inv2r;
            dr_i = (nu * c[3] - pi) * inv2r;
            dz_r = nu * c[4];
            dz_i = nu * c[5];
        }
        if (a.loc_re) {
            const double *Fr = a.loc_re + ((size_t)box * nm + n) * a.ncoef;
            const double *Fi = a.loc_im + ((size_t)box * nm + n) * a.ncoef;
            double vr, dur, dvr, vi, dui, dvi;
            l2p_eval<GRAD>(Fr, a.M, u, v, vr, dur, dvr);
            l2p_eval<GRAD>(Fi, a.M, u, v, vi, dui, dvi);
            pr += vr;
            pi += vi;
            if (GRAD) {
                double ih = 1.0 / a.h;
                dr_r += dur * ih;
                dr_i += dui * ih;
                dz_r += dvr * ih;
                dz_i += dvi * ih;
            }
        }
        if (a.part) {
            size_t base = (size_t)split * ncomp;
            size_t nfm = (size_t)a.nfield;
            a.part[((base + 0) * nm + n) * nfm + t] = pr;
            a.part[((base + 1) * nm + n) * nfm + t] = pi;
            if (GRAD) {
                a.part[((base + 2) * nm + n) * nfm + t] = dr_r;
                a.part[((base + 3) * nm + n) * nfm + t] = dr_i;
                a.part[((base + 4) * nm + n) * nfm + t] = dz_r;
                a.part[((base + 5) * nm + n) * nfm + t] = dz_i;
            }
        } else {
            size_t od = (size_t)n * a.nfield + dst;
            if (a.o_re) a.o_re[od] = pr;
            if (a.o_im) a.o_im[od] = pi;
            if (GRAD) {
                a.o_dr_re[od] = dr_r;
                a.o_dr_im[od] = dr_i;
                a.o_dz_re[od] = dz_r;
                a.o_dz_im[od] = dz_i;
            }
        }
    }
}

static size_t near2_smem(int nm, int grad)
{
    int Nq = (grad && nm < 2) ? 1 : nm - 1;
    int ncomp = grad ? 6 : 2, npp = grad ? 5 : 1;
    int mper = (nm + NEAR2_WB - 1) / NEAR2_WB;
    return sizeof(double) * ((size_t)AFMM_REC_TAB + AFMM_MAX_MODES + (size_t)NEAR2_WB * (Nq + 1) * 32 +
                             (size_t)NEAR2_WB * npp * 32 + (size_t)NEAR2_WB * ncomp * mper * 32);
}

// ------------------------------------------------------------------------------------
// Near field in FP32-pair arithmetic (AFMM_FP64 and AFMM_MIXED), warp-specialised.
//
// A block takes one work unit: up to 32 field points of one leaf against the sources of
// its 3 x 3 neighbour leaves (the D list of Sec. 2.2), or one source split of the direct
// sum.  The unit's (field point, source) pairs are cut into slots of 32 lanes (lane = field
// point; when the unit has c <= 16 points, T = 2^ceil(log2 c) lanes per source and 32 / T
// sources per slot).  The warps split into two roles:
//   producers  take the next slot from a shared counter and compute each lane's pair: the
//              coordinate differences (FP64, split exactly), the AGM start values, the
//              forward or Miller sweep of the scaled Legendre recursion (Eq.
//              gfunc:recursion) and the gradient factors, into a ring of B slots;
//   consumers  own MPER modes each (register accumulators) and walk the slots in order,
//              adding q^(n) G^(n) (Eq. analysis:sum) and the gradient terms.
// A full and an empty mbarrier per ring slot hand the slots over; every wait is bounded
// (1 s), after which the block records the timeout in the plan's error word and ends.  The
// sequential, latency-bound recursion of the producers thus runs beside the consumers'
// independent multiply-adds instead of alternating with them at block barriers.
//
// The consumers work on mode pairs (2m, 2m+1) with packed f32x2 instructions: the slot
// stores y_n interleaved by mode pair (SeqSlot), the amplitudes are stored the same way,
// and the per-pair factors in broadcast form, so every operand is a ready register pair.
// The packed operations are the scalar FP32-pair operations lane by lane: the results are
// those of the same sums in scalar FP32-pair arithmetic.
// ------------------------------------------------------------------------------------
constexpr int NWS_THREADS = 512;                             // 16 warps per block
constexpr int NWS_BMAX = 24;                                 // ring slots (upper bound)
constexpr int NWS_SRC_STAGE = 1024;                          // unit source lists staged in shared memory
constexpr unsigned long long NWS_WAIT_NS = 1000000000ull;    // a hand-over wait gives up after 1 s

// Lane 0 waits on the barrier (suspended in hardware between polls; bounded by the timer);
// the warp learns the outcome and, through __syncwarp, is ordered after lane 0's acquire.
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, int lane, int *err, volatile int *abort_flag)
{
    int ok = 1;
    if (lane == 0 && !mbar_try(bar, parity)) {
        const unsigned long long t0 = global_ns();
        for (;;) {
            if (mbar_try_sleep(bar, parity, 20000u)) break;
            if (*abort_flag) {
                ok = 0;
                break;
            }
            if (global_ns() - t0 > NWS_WAIT_NS) {
                ok = 0;
                *abort_flag = 1;
                if (err) *(volatile int *)err = 1;
                break;
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

__device__ __forceinline__ float4 bcast4(dfv v) { return make_float4(v.hi, v.hi, v.lo, v.lo); }

// Kahan-compensated FP32 sums of two components at once: S the sums, C the running
// compensations (true sums ~ S - C)
__device__ __forceinline__ void kahan2(float2 &S, float2 &C, float2 v)
{
    const float2 y = fsub2(v, C);
    const float2 t = fadd2(S, y);
    C = fsub2(fsub2(t, S), y);
    S = t;
}

// the range k (< nrg) of a flattened source list holding position i: rcum[k] <= i < rcum[k + 1]
// (empty ranges are skipped); a linear scan for the 9 ranges of the uniform tree, a binary
// search over the longer lists of the adaptive tree
__device__ __forceinline__ int ws_range_of(const int *rcum, int nrg, int i)
{
    if (nrg <= 9) {
        int rg = 0;
        while (rg < nrg - 1 && rcum[rg + 1] <= i) ++rg;
        return rg;
    }
    int lo = 0, hi = nrg - 1;  // the largest k with rcum[k] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rcum[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// MPER: modes per consumer warp (even); MIX: MIXED precision (same FP32-pair sequence,
// FP32 products with Kahan-compensated FP32 sums, FP32 locals)
template <bool GRAD, int MPER, bool MIX>
__global__ void __launch_bounds__(NWS_THREADS, 1) k_near_ws(const NearArgs a, const RecTab tab, int ncons, int nbuf)
{
    static_assert(MPER % 2 == 0, "consumers work on mode pairs");
    extern __shared__ __align__(16) unsigned char smem_ws[];
    // The FP64 path folds the backward sweeps' scale into the sequence (one product less
    // per mode pair for the consumers); MIXED keeps it as a per-pair factor: its consumers'
    // FP32 products gain little from the fold, while the in-place scaling costs its
    // producers N + 1 pair products per backward lane (measured on 65 modes near the axis).
    constexpr bool FOLD = !MIX;
    constexpr int PB = FOLD ? 0 : 1;                 // row of the gradient factors
    constexpr int NPP = PB + (GRAD ? 4 : 0);         // per-pair factors: (scale,) x, qfac, A, B
    constexpr int NC = GRAD ? 6 : 2;   // accumulated components
    constexpr int NP = MPER / 2;       // mode pairs per consumer
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nm = a.nmodes, N = a.N;
    const int Nq = GRAD && N < 1 ? 1 : N;  // the gradient of mode 0 needs y_1
    const int npair = (Nq + 2) / 2;        // mode pairs of y_0 .. y_Nq
    const int npq_all = (nm + 1) / 2;      // mode pairs of the amplitude copies
    float2 *gam2 = reinterpret_cast<float2 *>(smem_ws);                 // [AFMM_REC_TAB]
    float4 *gam4 = reinterpret_cast<float4 *>(gam2 + AFMM_REC_TAB);     // [pair] gam_2m, gam_2m+1
    float4 *rho4 = gam4 + (AFMM_MAX_MODES / 2 + 1);                     // [pair] rho_n = c_{n-1} / c_n
    unsigned char *ring = reinterpret_cast<unsigned char *>(rho4 + AFMM_MAX_MODES / 2 + 1);
    const size_t slot_bytes = (size_t)(npair + NPP) * 32 * sizeof(float4) + 32 * sizeof(int);
    __shared__ uint64_t s_full[NWS_BMAX], s_empty[NWS_BMAX];
    __shared__ int rb[AFMM_NEAR_MAXRG + 1], rcum[AFMM_NEAR_MAXRG + 1];
    __shared__ int s_nrg;
    __shared__ int s_next;
    __shared__ int s_src[NWS_SRC_STAGE];
    __shared__ volatile int s_abort;
    for (int i = threadIdx.x; i < AFMM_REC_TAB; i += blockDim.x) {
        dfv g = df_from_double(tab.gam[i]);
        gam2[i] = make_float2(g.hi, g.lo);
    }
    for (int m = threadIdx.x; m < AFMM_MAX_MODES / 2 + 1; m += blockDim.x) {
        const dfv g0 = df_from_double(tab.gam[2 * m]), g1 = df_from_double(tab.gam[2 * m + 1]);
        gam4[m] = make_float4(g0.hi, g1.hi, g0.lo, g1.lo);
    }
    for (int m = threadIdx.x; 2 * m < nm; m += blockDim.x) {
        const int n = 2 * m;
        const dfv r0 = df_from_double(n == 0 ? 1.0 : tab.c[n - 1] / tab.c[n]);
        const dfv r1 = n + 1 < nm ? df_from_double(tab.c[n] / tab.c[n + 1]) : df_make(0.f, 0.f);
        rho4[m] = make_float4(r0.hi, r1.hi, r0.lo, r1.lo);
    }
    const int64_t unit = blockIdx.x;
    int64_t t0, t1, split = 0;
    int box = -1, ulevel = 0;
    if (a.direct) {
        int64_t tu = unit / a.nsplit;
        split = unit % a.nsplit;
        t0 = tu * 32;
        t1 = min(t0 + 32, a.nfield);
    } else {
        NearUnit u = a.units[unit];
        box = u.box;
        t0 = u.begin;
        t1 = u.end;
        ulevel = u.level;
    }
    if (threadIdx.x == 0) {
        // the unit's sources as nrg ranges [rb[k], rb[k] + rcum[k + 1] - rcum[k]), flattened
        int cum = 0, nrg = 9;
        if (a.direct) {
            int64_t s0 = split * a.split_len, s1 = min(s0 + a.split_len, a.nsrc);
            rb[0] = (int)s0;
            rcum[0] = 0;
            cum = (int)(s1 > s0 ? s1 - s0 : 0);
            for (int k = 1; k < 10; ++k) {
                rb[k] = 0;
                rcum[k] = cum;
            }
        } else if (a.nl_off) {  // adaptive tree: the leaf's near list (at most AFMM_NEAR_MAXRG)
            const int64_t g = a.nl_base[ulevel] + box, o0 = a.nl_off[g];
            nrg = (int)(a.nl_off[g + 1] - o0);
            for (int k = 0; k < nrg; ++k) {
                const int2 r = a.nl_rng[o0 + k];
                rb[k] = r.x;
                rcum[k] = cum;
                cum += r.y - r.x;
            }
            rb[nrg] = 0;
            rcum[nrg] = cum;
        } else {
            for (int k = 0; k < 9; ++k) {
                int32_t nb = a.nbr[(int64_t)box * 9 + k];
                int2 r = nb >= 0 ? a.srng[nb] : make_int2(0, 0);
                rb[k] = r.x;
                rcum[k] = cum;
                cum += r.y - r.x;
            }
            rb[9] = 0;
            rcum[9] = cum;
        }
        s_nrg = nrg;
        s_next = 0;
        s_abort = 0;
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(&s_full[b], 1);
            mbar_init(&s_empty[b], (uint32_t)ncons);
        }
    }
    // lane packing: the unit's c targets take T = 2^ceil(log2 c) lanes, and the 32 / T lane
    // groups (slices) take consecutive sources of a slot; the slices are summed at the end
    const int cnt = (int)(t1 - t0);
    const int lgT = cnt <= 1 ? 0 : 32 - __clz(cnt - 1);
    const int S = 32 >> lgT;
    const int tl = lane & ((1 << lgT) - 1), slice = lane >> lgT;
    const int64_t t = t0 + tl;
    const bool active = t < t1;
    const int64_t tc = active ? t : t0;
    const double rt = a.fr[tc], zt = a.fz[tc];
    __syncthreads();
    const int nrg = s_nrg;
    const int total = rcum[nrg];
    const int nslots = (total + S - 1) / S;
    if (total <= NWS_SRC_STAGE) {  // the unit's source list, in slot order
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int rg = ws_range_of(rcum, nrg, i);
            s_src[i] = rb[rg] + (i - rcum[rg]);
        }
        __syncthreads();
    }

    if (warp >= ncons) {
        // ---------------- producer ----------------
        const float4 tg0 = a.geo_f[2 * tc], tg1 = a.geo_f[2 * tc + 1];
        const dfv inv2r = df_scale2(df_make(tg1.z, tg1.w), 0.5f);  // 1 / (2 r)
        const float extra = (float)a.pp.miller_extra;
        for (;;) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&s_next, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= nslots) break;
            const int b = k % nbuf;
            if (!ws_wait(&s_empty[b], ((uint32_t)(k / nbuf) & 1u) ^ 1u, lane, a.err, &s_abort)) break;
            float4 *y4 = reinterpret_cast<float4 *>(ring + (size_t)b * slot_bytes);
            float4 *p4 = y4 + (size_t)npair * 32;
            int kk = k * S + slice;
            const bool valid = kk < total;
            if (!valid) kk = total - 1;
            int64_t s;
            if (total <= NWS_SRC_STAGE) {
                s = s_src[kk];
            } else {
                const int rg = ws_range_of(rcum, nrg, kk);
                s = rb[rg] + (kk - rcum[rg]);
            }
            const float4 sg0 = a.geo_s[2 * s], sg1 = a.geo_s[2 * s + 1];
            const dfv inv2w = df_mul(inv2r, df_make(sg1.z, sg1.w));  // 1 / (2 r r1)
            PairDF g;
            // a lane past the unit's last target repeats the first target's pair (tc): its sums
            // are never written, and its sequence takes the same regime as a real pair's
            // instead of a full backward sweep
            pair_geom_f32x3(tg0, tg1, sg0, sg1, inv2w, valid, g);
            SeqSlot ys;
            ys.y = reinterpret_cast<float *>(y4 + lane);
            if ((Nq & 1) == 0) ys.put(Nq + 1, df_make(0.f, 0.f));  // pad of the last mode pair
            const bool fwd = pair_forward(g.t, a.df_tlim);
            dfv csum;
            const dfv G0 = df_scale2(df_rcp(pair_agm_df(g, csum)), 0.5f);  // 1 / (2 AGM)
            const dfv sc = pair_sweep_df<FOLD>(g.chi, g.t, g.zero, inv2w, Nq, fwd, extra, G0, csum, gam2, gam4, ys);
            reinterpret_cast<int *>(p4 + NPP * 32)[lane] = (int)s;
            if (!FOLD) p4[lane] = bcast4(sc);
            if (GRAD) {
                const dfv inv = df_rcp(df_mul(g.rp2, g.rm2));
                const dfv ip = df_mul(g.rm2, inv), im = df_mul(g.rp2, inv);
                dfv As = df_add(ip, im), Bs = df_sub(ip, im);
                if (!FOLD) {
                    As = df_mul(sc, As);
                    Bs = df_mul(sc, Bs);
                }
                const dfv qf = df_sub(df_mul(g.dr, g.sr), df_mul(g.x, g.x));
                p4[32 * PB + lane] = bcast4(g.x);
                p4[32 * (PB + 1) + lane] = bcast4(qf);
                p4[32 * (PB + 2) + lane] = bcast4(As);
                p4[32 * (PB + 3) + lane] = bcast4(Bs);
            }
            __syncwarp();
            if (lane == 0 && !(a.inject_timeout && k == 0)) mbar_arrive(&s_full[b]);
        }
        return;
    }

    // ---------------- consumer: modes n0 .. n0 + MPER - 1 ----------------
    const int n0 = a.mode_lo + warp * MPER;  // mode_lo is even
    const int m0 = n0 / 2;
    const int nhi = a.mode_hi;
    float2 aS[NC][NP], aE[NC][NP];  // .x mode 2m, .y mode 2m + 1
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < NP; ++j) aS[c][j] = aE[c][j] = make_float2(0.f, 0.f);
    for (int k = 0; k < nslots; ++k) {
        const int b = k % nbuf;
        if (!ws_wait(&s_full[b], (uint32_t)(k / nbuf) & 1u, lane, a.err, &s_abort)) return;
        const unsigned char *sl = ring + (size_t)b * slot_bytes;
        const float4 *y4 = reinterpret_cast<const float4 *>(sl);
        const float4 *p4 = y4 + (size_t)npair * 32;
        const int64_t s = reinterpret_cast<const int *>(p4 + NPP * 32)[lane];
        // the slot holds y_n = G_n / c_n (the amplitudes carry c_n), so the potential's
        // products need no per-pair factor
        const df2 Z2 = df2_bcast(df_make(0.f, 0.f));
        df2 GX = Z2, QF = Z2, AS = Z2, BS = Z2;
        dfv yprev = df_make(0.f, 0.f);
        const float2 SCf = FOLD ? Z2.hi : make_float2(p4[lane].x, p4[lane].y);  // MIXED: the scale
        if (GRAD) {
            GX = df2_from4(p4[32 * PB + lane]);
            QF = df2_from4(p4[32 * (PB + 1) + lane]);
            AS = df2_from4(p4[32 * (PB + 2) + lane]);
            BS = df2_from4(p4[32 * (PB + 3) + lane]);
            // y_{n0 - 1}: the second mode of the previous pair; y_{-1} := y_1
            yprev = df2_y(df2_from4(y4[(m0 == 0 ? 0 : m0 - 1) * 32 + lane]));
        }
        // The last consumer of an odd number of mode pairs has one pair fewer and takes a
        // warp-uniform branch that skips it: that warp shares its SM sub-partition with two
        // other consumers (9 consumer warps over 4 sub-partitions), so halving its work
        // evens the sub-partitions' FMA-pipe load.  Full warps run the pairs unrolled, so
        // the compiler interleaves their chains.
        const bool fullp = 2 * (m0 + NP - 1) < nhi;
        if (MIX) {
            // FP32 products of the pairs' high words, Kahan-compensated sums (aE: compensation)
            const float2 GXf = GX.hi, QFf = QF.hi, nBS = fneg2(BS.hi);
            auto step = [&](const int j) {
                const int m = m0 + j;
                const df2 Y = df2_from4(y4[m * 32 + lane]);
                const float4 Q4 = a.q32[(size_t)s * npq_all + m];
                const float2 QR = make_float2(Q4.x, Q4.y), QI = make_float2(Q4.z, Q4.w);
                const float2 G = fmul2(SCf, Y.hi);
                kahan2(aS[0][j], aE[0][j], fmul2(QR, G));
                kahan2(aS[1][j], aE[1][j], fmul2(QI, G));
                if (GRAD) {
                    // y_n A + rho_n y_{n-1} B cancels for near pairs (A ~ -B): FP32 pairs
                    const df2 YP = df2_pack(yprev, df2_x(Y));
                    yprev = df2_y(Y);
                    const df2 R = df2_from4(rho4[m]);
                    const float2 nT = fmul2(R.hi, fneg2(YP.hi));
                    const df2 T = df2_mul_nr(R, YP, nT);  // rho_n y_{n-1}, only feeds a product
                    const float2 wt = df2_fma(T, BS, nBS, df2_mul(Y, AS)).hi;
                    const float2 xw = fmul2(GXf, wt), qw = fmul2(QFf, wt);
                    kahan2(aS[2 % NC][j], aE[2 % NC][j], fmul2(QR, qw));
                    kahan2(aS[3 % NC][j], aE[3 % NC][j], fmul2(QI, qw));
                    kahan2(aS[4 % NC][j], aE[4 % NC][j], fmul2(QR, xw));
                    kahan2(aS[5 % NC][j], aE[5 % NC][j], fmul2(QI, xw));
                }
            };
            if (fullp) {
#pragma unroll
                for (int j = 0; j < NP; ++j) step(j);
            } else {
#pragma unroll
                for (int j = 0; j < NP; ++j)
                    if (2 * (m0 + j) < nhi) step(j);
            }
        } else {
            // negated high words of the per-slot factors (the products below need no
            // negation instructions: see df2_mul_np, df2_acc_n)
            const float2 NEG = make_float2(-1.f, -1.f);
            float2 nyprev = make_float2(-yprev.hi, 0.f);  // -(high word of yprev)
            auto step = [&](const int j) {
                const int m = m0 + j;
                const df2 Y = df2_from4(y4[m * 32 + lane]);
                const float4 *qs = a.qdf + ((size_t)s * npq_all + m) * 2;
                const df2 QR = df2_from4(qs[0]);
                const df2 QI = df2_from4(qs[1]);
                const float2 nY = fmul2(Y.hi, NEG);
                df2_acc_n(aS[0][j], aE[0][j], QR, Y, nY);
                df2_acc_n(aS[1][j], aE[1][j], QI, Y, nY);
                if (GRAD) {
                    // w_n = y_n A + rho_n y_{n-1} B, the derivative recursion's weight
                    const df2 YP = df2_pack(yprev, df2_x(Y));
                    const float2 nYP = make_float2(nyprev.x, nY.x);
                    yprev = df2_y(Y);
                    nyprev.x = nY.y;
                    float2 nWT;
                    const df2 R = df2_from4(rho4[m]);
                    // T, XW and QW only feed pair products: left unnormalised (df2_mul_nr)
                    const float2 nT = fmul2(R.hi, nYP);
                    const df2 T = df2_mul_nr(R, YP, nT);
                    const df2 WT = df2_dot2_np(Y, nY, AS, T, nT, BS, nWT);
                    const float2 nXW = fmul2(nWT, GX.hi), nQW = fmul2(nWT, QF.hi);
                    const df2 XW = df2_mul_nr(WT, GX, nXW);
                    const df2 QW = df2_mul_nr(WT, QF, nQW);
                    df2_acc_n(aS[2 % NC][j], aE[2 % NC][j], QR, QW, nQW);
                    df2_acc_n(aS[3 % NC][j], aE[3 % NC][j], QI, QW, nQW);
                    df2_acc_n(aS[4 % NC][j], aE[4 % NC][j], QR, XW, nXW);
                    df2_acc_n(aS[5 % NC][j], aE[5 % NC][j], QI, XW, nXW);
                }
            };
            if (fullp) {
#pragma unroll
                for (int j = 0; j < NP; ++j) step(j);
            } else {
#pragma unroll
                for (int j = 0; j < NP; ++j)
                    if (2 * (m0 + j) < nhi) step(j);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[b]);
    }
    // sum the slices in FP64 (every lane of target tl gets the sums); cs is indexed by the
    // mode at run time below (local memory: once per unit, off the slot loop)
    double cs[NC][MPER];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int jp = 0; jp < NP; ++jp) {
            double v0 = MIX ? (double)aS[q][jp].x - (double)aE[q][jp].x : (double)aS[q][jp].x + (double)aE[q][jp].x;
            double v1 = MIX ? (double)aS[q][jp].y - (double)aE[q][jp].y : (double)aS[q][jp].y + (double)aE[q][jp].y;
            for (int o = 1 << lgT; o < 32; o <<= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            }
            cs[q][2 * jp] = v0;
            cs[q][2 * jp + 1] = v1;
        }
    if (!active || slice != 0) return;
    // write, or add to the local-expansion values that k_l2p wrote (FMM near field)
    const bool add = a.accumulate != 0;
    const int64_t dst = a.out_perm ? a.out_perm[t] : t;
#pragma unroll 1
    for (int j = 0; j < MPER; ++j) {
        const int n = n0 + j;
        if (n >= nhi) continue;
        const double pr = cs[0][j];
        const double pi = cs[1][j];
        double dr_r = 0, dr_i = 0, dz_r = 0, dz_i = 0;
        if (GRAD) {
            double nu = n - 0.5;
            dr_r = (nu * cs[2 % NC][j] - pr) * (0.5 / rt);
            dr_i = (nu * cs[3 % NC][j] - pi) * (0.5 / rt);
            dz_r = nu * cs[4 % NC][j];
            dz_i = nu * cs[5 % NC][j];
        }
        if (a.part) {
            size_t base = (size_t)split * NC;
            size_t nfm = (size_t)a.nfield;
            a.part[((base + 0) * nm + n) * nfm + t] = pr;
            a.part[((base + 1) * nm + n) * nfm + t] = pi;
            if (GRAD) {
                a.part[((base + 2) * nm + n) * nfm + t] = dr_r;
                a.part[((base + 3) * nm + n) * nfm + t] = dr_i;
                a.part[((base + 4) * nm + n) * nfm + t] = dz_r;
                a.part[((base + 5) * nm + n) * nfm + t] = dz_i;
            }
        } else {
            const size_t od = (size_t)n * a.nfield + dst;
            if (a.o_re) a.o_re[od] = add ? a.o_re[od] + pr : pr;
            if (a.o_im) a.o_im[od] = add ? a.o_im[od] + pi : pi;
            if (GRAD) {
                a.o_dr_re[od] = add ? a.o_dr_re[od] + dr_r : dr_r;
                a.o_dr_im[od] = add ? a.o_dr_im[od] + dr_i : dr_i;
                a.o_dz_re[od] = add ? a.o_dz_re[od] + dz_r : dz_r;
                a.o_dz_im[od] = add ? a.o_dz_im[od] + dz_i : dz_i;
            }
        }
    }
}

// Local expansion (Eq. analysis:local) at the field points of the near-field units, the
// L2P of Algorithm 1: value and gradient, written to the outputs before k_near_ws adds the
// near sums.  One block of 4 warps per unit (<= 32 field points of one leaf): warp w takes
// modes w, w + 4, ...; the leaf's coefficients of a mode (re and im) are staged in shared
// memory by coalesced loads, and each lane runs the packed (re, im) Horner scheme at its
// point.  AFMM_FP64: FP32-pair locals and arithmetic; MIXED: FP32.
constexpr int L2P_WARPS = 4;
constexpr int L2P_MAXC = (AFMM_MAX_ORDER + 1) * (AFMM_MAX_ORDER + 2) / 2;

template <bool GRAD, bool MIX>
__global__ void __launch_bounds__(L2P_WARPS * 32) k_l2p(const NearArgs a)
{
    __shared__ float4 sF[L2P_WARPS][L2P_MAXC];  // (re.hi, im.hi, re.lo, im.lo), or (re, im, -, -)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const NearUnit un = a.units[blockIdx.x];
    const int box = un.box, nm = a.nmodes, M = a.M, nc = a.ncoef;
    const int64_t t = un.begin + lane;
    const bool active = t < un.end;
    const int64_t tc = active ? t : un.begin;
    const double rt = a.fr[tc], zt = a.fz[tc];
    // the leaf's level: d on the uniform tree, the unit's own on the adaptive tree
    const bool ad = a.nl_off != nullptr;
    const double h = ad ? a.side / (double)(1 << un.level) : a.h;
    const uint32_t kk = ad ? a.lv_key[un.level][box] : a.leaf_key[box];
    const float2 *locdf_re = ad ? a.lv_locd_re[un.level] : a.locdf_re;
    const float2 *locdf_im = ad ? a.lv_locd_im[un.level] : a.locdf_im;
    const float *loc32_re = ad ? a.lv_loc32_re[un.level] : a.loc32_re;
    const float *loc32_im = ad ? a.lv_loc32_im[un.level] : a.loc32_im;
    const double cr = a.r0 + ((double)morton_ir(kk) + 0.5) * h, cz = a.z0 + ((double)morton_iz(kk) + 0.5) * h;
    const double ud = (rt - cr) / h, vd = (zt - cz) / h, ih = 1.0 / h;
    const int64_t dst = a.out_perm ? a.out_perm[tc] : tc;
    float4 *F = sF[warp];
    for (int n = warp; n < nm; n += L2P_WARPS) {
        const size_t off = ((size_t)box * nm + n) * nc;
        for (int c = lane; c < nc; c += 32) {
            if (MIX)
                F[c] = make_float4(loc32_re[off + c], loc32_im[off + c], 0.f, 0.f);
            else {
                const float2 r = locdf_re[off + c], i = locdf_im[off + c];
                F[c] = make_float4(r.x, i.x, r.y, i.y);
            }
        }
        __syncwarp();
        double pr, pi, dr_r = 0, dr_i = 0, dz_r = 0, dz_i = 0;
        if (MIX) {
            const float2 U = make_float2((float)ud, (float)ud), V = make_float2((float)vd, (float)vd);
            const float2 Z = make_float2(0.f, 0.f);
            float2 pu = Z, pdu = Z, pdv = Z;
            for (int k = M; k >= 0; --k) {
                const int base = k * (M + 1) - k * (k - 1) / 2;
                float2 pk = Z, pkd = Z;
                for (int l = M - k; l >= 0; --l) {
                    if (GRAD) pkd = ffma2(pkd, V, pk);
                    const float4 f = F[base + l];
                    pk = ffma2(pk, V, make_float2(f.x, f.y));
                }
                if (GRAD) {
                    pdu = ffma2(pdu, U, pu);
                    pdv = ffma2(pdv, U, pkd);
                }
                pu = ffma2(pu, U, pk);
            }
            pr = pu.x;
            pi = pu.y;
            if (GRAD) {
                dr_r = pdu.x * ih;
                dr_i = pdu.y * ih;
                dz_r = pdv.x * ih;
                dz_i = pdv.y * ih;
            }
        } else {
            const df2 U = df2_bcast(df_from_double(ud)), V = df2_bcast(df_from_double(vd));
            const float2 nU = fneg2(U.hi), nV = fneg2(V.hi);
            const df2 Z = df2_make(make_float2(0.f, 0.f), make_float2(0.f, 0.f));
            df2 pu = Z, pdu = Z, pdv = Z;
            for (int k = M; k >= 0; --k) {
                const int base = k * (M + 1) - k * (k - 1) / 2;
                df2 pk = Z, pkd = Z;
                for (int l = M - k; l >= 0; --l) {
                    if (GRAD) pkd = df2_fma(pkd, V, nV, pk);
                    pk = df2_fma(pk, V, nV, df2_from4(F[base + l]));
                }
                if (GRAD) {
                    pdu = df2_fma(pdu, U, nU, pu);
                    pdv = df2_fma(pdv, U, nU, pkd);
                }
                pu = df2_fma(pu, U, nU, pk);
            }
            pr = df_to_double(df2_x(pu));
            pi = df_to_double(df2_y(pu));
            if (GRAD) {
                dr_r = df_to_double(df2_x(pdu)) * ih;
                dr_i = df_to_double(df2_y(pdu)) * ih;
                dz_r = df_to_double(df2_x(pdv)) * ih;
                dz_i = df_to_double(df2_y(pdv)) * ih;
            }
        }
        if (active) {
            const size_t od = (size_t)n * a.nfield + dst;
            if (a.o_re) a.o_re[od] = pr;
            if (a.o_im) a.o_im[od] = pi;
            if (GRAD) {
                a.o_dr_re[od] = dr_r;
                a.o_dr_im[od] = dr_i;
                a.o_dz_re[od] = dz_r;
                a.o_dz_im[od] = dz_i;
            }
        }
        __syncwarp();
    }
}

// shared memory of k_near_ws: tables + ring of nbuf slots
static size_t nws_slot_bytes(int nm, int grad, int mix)
{
    const int Nq = (grad && nm < 2) ? 1 : nm - 1;
    const int npair = (Nq + 2) / 2, npp = (mix ? 1 : 0) + (grad ? 4 : 0);  // as NPP in k_near_ws
    return (size_t)(npair + npp) * 32 * 16 + 32 * sizeof(int);
}
static size_t nws_table_bytes()
{
    return sizeof(float2) * AFMM_REC_TAB + sizeof(float4) * 2 * (AFMM_MAX_MODES / 2 + 1);
}

// Modes per consumer warp: the smallest even MPER with at most 11 consumers (>= 5 producers)
static int nws_mper(int nm, bool grad)
{
    if (!grad) {
        // potential only: two accumulations per mode, light consumers; at most 6 consumer
        // warps, so that 10 or more warps compute sequences
        for (int mp = 4; mp <= 16; mp += 4)
            if ((nm + mp - 1) / mp <= 6) return mp;
        return 0;
    }
    // with the gradient: at most 9 consumer warps, at least 7 producers (measured best on
    // 33 modes: 9 x 4 against 11 x 3 or 6 x 6; on 65 modes 9 x 8 against 11 x 6)
    for (int mp = 2; mp <= 8; mp += 2)
        if ((nm + mp - 1) / mp <= 9) return mp;
    return 0;
}

// modes per launch: 9 x 8 with the gradient, 6 x 16 without
static int nws_modes_per_launch(bool grad) { return grad ? 72 : 96; }

template <bool GRAD, int MPER, bool MIX>
static afmm_status launch_near_ws_k(const NearArgs &a, const RecTab &tab, cudaStream_t st)
{
    const int ncons = (a.mode_hi - a.mode_lo + MPER - 1) / MPER;
    const size_t slot = nws_slot_bytes(a.nmodes, GRAD, MIX), tabs = nws_table_bytes();
    const size_t budget = 200 * 1024;
    int nbuf = (int)((budget - tabs) / slot);
    if (nbuf > NWS_BMAX) nbuf = NWS_BMAX;
    if (nbuf < 2) return AFMM_EUNSUPPORTED;
    // at most nbuf producers: a producer then never waits on a ring slot two rounds behind
    // (nbuf + 1 producers would all have to be stuck on slots of the same consumer backlog),
    // so the parity of each wait is unambiguous
    int nprod = NWS_THREADS / 32 - ncons;
    if (nprod > nbuf) nprod = nbuf;
    const size_t sm = tabs + (size_t)nbuf * slot;
    AFMM_CUDA(cudaFuncSetAttribute(k_near_ws<GRAD, MPER, MIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_near_ws<GRAD, MPER, MIX><<<(unsigned)a.nunits, 32 * (ncons + nprod), sm, st>>>(a, tab, ncons, nbuf);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

template <bool GRAD, bool MIX>
static afmm_status launch_near_ws(const NearArgs &a, const RecTab &tab, cudaStream_t st)
{
    const int mp = nws_mper(a.mode_hi - a.mode_lo, GRAD);
    if constexpr (!GRAD) {
        if (mp == 12) return launch_near_ws_k<GRAD, 12, MIX>(a, tab, st);
        if (mp == 16) return launch_near_ws_k<GRAD, 16, MIX>(a, tab, st);
    }
    switch (mp) {
    case 2: return launch_near_ws_k<GRAD, 2, MIX>(a, tab, st);
    case 4: return launch_near_ws_k<GRAD, 4, MIX>(a, tab, st);
    case 6: return launch_near_ws_k<GRAD, 6, MIX>(a, tab, st);
    case 8: return launch_near_ws_k<GRAD, 8, MIX>(a, tab, st);
    default: return AFMM_EUNSUPPORTED;
    }
}

// strengths into sorted order, times c_n: the FP64 copy [mode][point] (far field) and the
// FP32-pair copy [point][mode pair][re, im] (near field: a source's amplitudes of all modes
// in one contiguous run); one thread per (mode pair, point)
__global__ void k_permute_df(const double *__restrict__ q_re, const double *__restrict__ q_im,
                             const int32_t *__restrict__ perm, int64_t n, int nm, const RecTab tab,
                             double *__restrict__ qs_re, double *__restrict__ qs_im, float4 *__restrict__ qd_ri)
{
    const int64_t npq = (nm + 1) / 2;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * npq) return;
    const int m = (int)(i / n);
    const int64_t j = i % n;
    dfv r[2], im[2];
    for (int h = 0; h < 2; ++h) {
        const int mode = 2 * m + h;
        r[h] = im[h] = df_make(0.f, 0.f);
        if (mode >= nm) continue;
        const size_t src = (size_t)mode * n + perm[j];
        const double c = tab.c[mode];
        const double vr = q_re[src] * c, vi = q_im[src] * c;
        qs_re[(size_t)mode * n + j] = vr;
        qs_im[(size_t)mode * n + j] = vi;
        r[h] = df_from_double(vr);
        im[h] = df_from_double(vi);
    }
    // per source, all mode pairs contiguous: [j][m][re, im] (one 32-byte sector per thread)
    float4 *qd = qd_ri + ((size_t)j * npq + m) * 2;
    qd[0] = make_float4(r[0].hi, r[1].hi, r[0].lo, r[1].lo);
    qd[1] = make_float4(im[0].hi, im[1].hi, im[0].lo, im[1].lo);
}

// sorted-order sums [comp][mode][t] into the caller's layout: out_c[mode][perm[t]]; one
// thread per element in plane order, so that each plane's scattered writes meet in L2
struct UnpermOut {
    double *o[6];
};
__global__ void k_unpermute(const double *__restrict__ S, const int32_t *__restrict__ perm, int nm, int64_t nf,
                            int ncomp, UnpermOut uo)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)ncomp * nm * nf) return;
    const int64_t plane = i / nf, t = i - plane * nf;
    const int c = (int)(plane / nm), n = (int)(plane - (int64_t)c * nm);
    double *dst = uo.o[c];
    if (dst) dst[(size_t)n * nf + perm[t]] = S[i];
}

// sum of split partials into the caller layout
__global__ void k_split_reduce(const double *__restrict__ part, int nsplit, int ncomp, int nm, int64_t nfield,
                               const int32_t *__restrict__ perm, double *o0, double *o1, double *o2, double *o3,
                               double *o4, double *o5)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)ncomp * nm * nfield;
    if (i >= tot) return;
    int comp = (int)(i / ((int64_t)nm * nfield));
    int64_t rem = i % ((int64_t)nm * nfield);
    int n = (int)(rem / nfield);
    int64_t t = rem % nfield;
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += part[(((size_t)k * ncomp + comp) * nm + n) * nfield + t];
    double *o = comp == 0 ? o0 : comp == 1 ? o1 : comp == 2 ? o2 : comp == 3 ? o3 : comp == 4 ? o4 : o5;
    if (o) o[(size_t)n * nfield + (perm ? perm[t] : t)] = s;
}

// strengths into sorted order, times c_n: qs[n][i] = q[n][perm[i]] * c_n
__global__ void k_permute(const double *__restrict__ q_re, const double *__restrict__ q_im,
                          const int32_t *__restrict__ perm, int64_t n, int nm, const RecTab tab,
                          double *__restrict__ qs_re, double *__restrict__ qs_im)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nm) return;
    int m = (int)(i / n);
    int64_t j = i % n;
    size_t src = (size_t)m * n + perm[j];
    double c = tab.c[m];
    qs_re[i] = q_re[src] * c;
    qs_im[i] = q_im[src] * c;
}

// unit evaluator: thread per pair, G (and gradient) for all modes
__global__ void k_green(int64_t np, const double *__restrict__ r, const double *__restrict__ r1,
                        const double *__restrict__ x, int nm, const RecTab tab, PairParams pp, double *G, double *Gr,
                        double *Gx)
{
    extern __shared__ double smem[];
    double *gam = smem;
    double *ys = gam + AFMM_REC_TAB;  // [max(nm, 2)][blockDim]
    for (int i = threadIdx.x; i < AFMM_REC_TAB; i += blockDim.x) gam[i] = tab.gam[i];
    __syncthreads();
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool active = p < np;
    int64_t pc = active ? p : 0;
    double rt = r[pc], rs = r1[pc], xx = x[pc];
    double inv2w = 0.5 / (rt * rs);
    PairGeom g;
    pair_geom(rt, xx, rs, 0.0, inv2w, active, g);
    int N = nm - 1;
    int Nq = N < 1 ? 1 : N;  // the gradient of mode 0 needs G^(1)
    double sc = pair_sequence(g, inv2w, Nq, pp, gam, ys + threadIdx.x, blockDim.x);
    if (!active) return;
    const int B = blockDim.x;
    for (int n = 0; n < nm; ++n) G[(size_t)n * np + p] = sc * tab.c[n] * ys[n * B + threadIdx.x];
    if (Gr) {
        double inv = 1.0 / (g.rp2 * g.rm2);
        double ip = g.rm2 * inv, im = g.rp2 * inv;
        double A = ip + im, Bc = ip - im;
        double qf = fma(rt - rs, rt + rs, -xx * xx);
        for (int n = 0; n < nm; ++n) {
            double gn = sc * tab.c[n] * ys[n * B + threadIdx.x];
            int m = n == 0 ? 1 : n - 1;
            double gm = sc * tab.c[m] * ys[m * B + threadIdx.x];
            double wv = gn * A + gm * Bc;
            double nu = n - 0.5;
            Gx[(size_t)n * np + p] = nu * xx * wv;
            Gr[(size_t)n * np + p] = (-gn + nu * qf * wv) / (2.0 * rt);
        }
    }
}

static size_t near_smem(int nm, int grad, int warps)
{
    int ncomp = grad ? 6 : 2;
    return sizeof(double) * ((size_t)AFMM_REC_TAB + AFMM_MAX_MODES + (size_t)warps * ((ncomp + 1) * nm + 1) * 32);
}

static int near_warps(int nm, int grad)
{
    for (int w = AFMM_NEAR_WARPS; w >= 1; --w)
        if (near_smem(nm, grad, w) <= 227 * 1024) return w;
    return 0;
}

static inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b > 0 ? (n + b - 1) / b : 1); }

// strengths into sorted order, times c_n, rounded to FP32 (MIXED precision), per point by
// mode pair: [point][mode pair] (re_2m, re_2m+1, im_2m, im_2m+1); one thread per (mode
// pair, point)
__global__ void k_permute32(const double *__restrict__ q_re, const double *__restrict__ q_im,
                            const int32_t *__restrict__ perm, int64_t n, int nm, const RecTab tab,
                            float4 *__restrict__ qs_ri)
{
    const int64_t npq = (nm + 1) / 2;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * npq) return;
    const int m = (int)(i / n);
    const int64_t j = i % n;
    float r[2] = {0.f, 0.f}, im[2] = {0.f, 0.f};
    for (int h = 0; h < 2; ++h) {
        const int mode = 2 * m + h;
        if (mode >= nm) continue;
        const size_t src = (size_t)mode * n + perm[j];
        const double c = tab.c[mode];
        r[h] = (float)(q_re[src] * c);
        im[h] = (float)(q_im[src] * c);
    }
    qs_ri[(size_t)j * npq + m] = make_float4(r[0], r[1], im[0], im[1]);
}

afmm_status launch_permute(afmm_plan p, int dir, const double *q_re, const double *q_im)
{
    int64_t n = dir == 0 ? p->ns : p->nf;
    const int32_t *perm = dir == 0 ? p->s_perm : p->t_perm;
    const int64_t npq = (p->nmodes + 1) / 2;
    if (p->precision == AFMM_MIXED)
        k_permute32<<<nblk(n * npq), 256, 0, p->stream>>>(q_re, q_im, perm, n, p->nmodes, *p->rec, p->qs32);
    else if (p->precision == AFMM_FP64)
        k_permute_df<<<nblk(n * npq), 256, 0, p->stream>>>(q_re, q_im, perm, n, p->nmodes, *p->rec, p->qs_re, p->qs_im,
                                                            p->qsdf);
    else
        k_permute<<<nblk(n * p->nmodes), 256, 0, p->stream>>>(q_re, q_im, perm, n, p->nmodes, *p->rec, p->qs_re,
                                                               p->qs_im);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

// dir 0: field points <- sources; dir 1: sources <- field points (transposed problem).
// direct = 1: all pairs (split over sources when the field set is small).
afmm_status launch_near(afmm_plan p, int dir, int with_local, int grad, double *phi_re, double *phi_im, double *dr_re,
                        double *dr_im, double *dz_re, double *dz_im, int direct)
{
    NearArgs a;
    memset(&a, 0, sizeof(a));
    const bool fw = dir == 0;
    a.fr = fw ? p->t_r : p->s_r;
    a.fz = fw ? p->t_z : p->s_z;
    a.nfield = fw ? p->nf : p->ns;
    a.sr = fw ? p->s_r : p->t_r;
    a.sz = fw ? p->s_z : p->t_z;
    a.geo_f = fw ? p->t_geo : p->s_geo;
    a.geo_s = fw ? p->s_geo : p->t_geo;
    a.nsrc = fw ? p->ns : p->nf;
    const bool mix = p->precision == AFMM_MIXED;
    a.q_re = p->qs_re;
    a.q_im = p->qs_im;
    a.q32 = p->qs32;
    a.nmodes = p->nmodes;
    a.N = p->N;
    a.pp = p->pp;
    a.out_perm = fw ? p->t_perm : p->s_perm;
    a.o_re = phi_re;
    a.o_im = phi_im;
    a.o_dr_re = dr_re;
    a.o_dr_im = dr_im;
    a.o_dz_re = dz_re;
    a.o_dz_im = dz_im;
    int d = p->d;
    if (direct) {
        int64_t tunits = (a.nfield + 31) / 32;
        int64_t want = 152 * 8;  // warps in flight to fill the GPU
        int nsplit = 1;
        if (tunits < want) {
            int64_t ns_ = (want + tunits - 1) / tunits;
            int64_t maxs = (a.nsrc + 63) / 64;
            int64_t room = p->part_cap / ((int64_t)(grad ? 6 : 2) * a.nmodes * a.nfield);
            if (ns_ > maxs) ns_ = maxs;
            if (ns_ > room) ns_ = room;
            nsplit = ns_ < 1 ? 1 : (int)ns_;
        }
        a.direct = 1;
        a.nsplit = nsplit;
        a.split_len = (a.nsrc + nsplit - 1) / nsplit;
        a.nunits = tunits * nsplit;
        a.part = nsplit > 1 ? p->part_buf : nullptr;
    } else {
        a.units = p->near_unit[dir];
        a.nunits = p->n_near_unit[dir];
        a.nbr = p->lv[d].nbr;
        a.srng = fw ? p->lv[d].srng : p->lv[d].trng;
        if (p->adaptive) {
            if (p->precision == AFMM_FP64_NATIVE) return AFMM_EUNSUPPORTED;
            a.nl_off = p->nl_off;
            a.nl_rng = p->nl_rng[dir];
            for (int l = 0; l <= AFMM_MAX_LEVEL; ++l) {
                a.nl_base[l] = p->nl_base[l];
                a.lv_key[l] = p->lv[l].key;
                a.lv_locd_re[l] = p->lv[l].locd_re;
                a.lv_locd_im[l] = p->lv[l].locd_im;
                a.lv_loc32_re[l] = p->lv[l].loc32_re;
                a.lv_loc32_im[l] = p->lv[l].loc32_im;
            }
            a.side = p->L;
        }
        if (with_local) {
            a.loc_re = mix ? nullptr : p->lv[d].loc_re;
            a.loc_im = mix ? nullptr : p->lv[d].loc_im;
            a.loc32_re = mix ? p->lv[d].loc32_re : nullptr;
            a.loc32_im = mix ? p->lv[d].loc32_im : nullptr;
            a.leaf_key = p->lv[d].key;
            a.M = p->M;
            a.ncoef = p->ncoef;
            a.r0 = p->r0;
            a.z0 = p->z0;
            a.h = p->L / (double)(1 << d);
        }
    }
    if (a.nunits == 0) return AFMM_OK;
    // The FP32-pair kernels write their sums in sorted point order (each unit's points are a
    // contiguous run, so the writes and the near field's additions to the L2P values are
    // coalesced); one pass then scatters them into the caller's layout, plane by plane, so
    // that the scattered writes of a plane meet in L2.  Split direct sums keep their own
    // reduction into the caller's layout.
    double *user[6] = {phi_re, phi_im, dr_re, dr_im, dz_re, dz_im};
    const int ncomp = grad ? 6 : 2;
    const bool sorted = p->precision != AFMM_FP64_NATIVE && !a.part && p->osort;
    if (sorted) {
        const size_t P = (size_t)a.nmodes * a.nfield;
        double **o[6] = {&a.o_re, &a.o_im, &a.o_dr_re, &a.o_dr_im, &a.o_dz_re, &a.o_dz_im};
        for (int c = 0; c < 6; ++c) *o[c] = (c < ncomp && user[c]) ? p->osort + c * P : nullptr;
        a.out_perm = nullptr;
    }
    size_t sm = near2_smem(p->nmodes, grad);
    unsigned grid = (unsigned)a.nunits;
    const int T = NEAR2_WB * 32;
    if (p->precision == AFMM_FP64_NATIVE && sm > 227 * 1024) return AFMM_EUNSUPPORTED;
    if (p->precision == AFMM_FP64 || mix) {
        // FP32-pair sequence (GB300's FP64 issues at 1/64 of FP32, so the pair arithmetic is
        // the fast way to the FP64-class sequence); FP64: FP32-pair sums, MIXED: compensated
        // FP32 sums.  Amplitudes are interleaved by mode pair.
        if (mix) {
            a.q32 = p->qs32;
        } else {
            a.qdf = p->qsdf;
            if (with_local && !direct) {  // the leaf locals are kept as FP32 pairs
                a.locdf_re = p->lv[d].locd_re;
                a.locdf_im = p->lv[d].locd_im;
                a.loc_re = nullptr;
                a.loc_im = nullptr;
            }
        }
        a.df_fwd_switch = (float)p->df_fwd_switch;
        a.df_tlim = (float)fmin(cosh(p->df_fwd_switch / (2.0 * (p->N < 1 ? 1 : p->N))), cosh(0.96)) - 1.0f;
        a.err = p->err_dev;
        a.inject_timeout = p->inject_near_timeout;
        const bool loc = mix ? a.loc32_re != nullptr : a.locdf_re != nullptr;
        if (loc) {  // the leaf's local expansion first; the near kernel adds its sums
            if (grad && mix)
                k_l2p<true, true><<<(unsigned)a.nunits, L2P_WARPS * 32, 0, p->stream>>>(a);
            else if (grad)
                k_l2p<true, false><<<(unsigned)a.nunits, L2P_WARPS * 32, 0, p->stream>>>(a);
            else if (mix)
                k_l2p<false, true><<<(unsigned)a.nunits, L2P_WARPS * 32, 0, p->stream>>>(a);
            else
                k_l2p<false, false><<<(unsigned)a.nunits, L2P_WARPS * 32, 0, p->stream>>>(a);
            AFMM_LAUNCH_CHECK();
            a.accumulate = 1;
        }
        if (p->timing) cudaEventRecord(p->ev[AFMM_EV_L2P], p->stream);
        // larger mode counts than one launch's consumer warps hold take several launches
        // over mode ranges (each recomputes the pair sequences)
        const int per = nws_modes_per_launch(grad != 0);
        for (int lo = 0; lo < p->nmodes; lo += per) {
            a.mode_lo = lo;
            a.mode_hi = p->nmodes < lo + per ? p->nmodes : lo + per;
            if (grad && mix)
                AFMM_TRY((launch_near_ws<true, true>(a, *p->rec, p->stream)));
            else if (grad)
                AFMM_TRY((launch_near_ws<true, false>(a, *p->rec, p->stream)));
            else if (mix)
                AFMM_TRY((launch_near_ws<false, true>(a, *p->rec, p->stream)));
            else
                AFMM_TRY((launch_near_ws<false, false>(a, *p->rec, p->stream)));
        }
    } else {
        // the FP64 kernels evaluate the local expansions themselves (no separate L2P phase)
        if (p->timing) cudaEventRecord(p->ev[AFMM_EV_L2P], p->stream);
        if (grad) {
            AFMM_CUDA(cudaFuncSetAttribute(k_near2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_near2<true><<<grid, T, sm, p->stream>>>(a, *p->rec);
        } else {
            AFMM_CUDA(cudaFuncSetAttribute(k_near2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            k_near2<false><<<grid, T, sm, p->stream>>>(a, *p->rec);
        }
    }
    if (p->precision == AFMM_FP64_NATIVE) AFMM_LAUNCH_CHECK();
    if (sorted) {
        UnpermOut uo;
        for (int c = 0; c < 6; ++c) uo.o[c] = c < ncomp ? user[c] : nullptr;
        const int32_t *perm = dir == 0 ? p->t_perm : p->s_perm;
        const int64_t tot = (int64_t)ncomp * a.nmodes * a.nfield;
        k_unpermute<<<nblk(tot), 256, 0, p->stream>>>(p->osort, perm, a.nmodes, a.nfield, ncomp, uo);
        AFMM_LAUNCH_CHECK();
    }
    if (a.part) {
        int ncomp = grad ? 6 : 2;
        int64_t tot = (int64_t)ncomp * a.nmodes * a.nfield;
        k_split_reduce<<<nblk(tot), 256, 0, p->stream>>>(a.part, a.nsplit, ncomp, a.nmodes, a.nfield, a.out_perm,
                                                         phi_re, phi_im, dr_re, dr_im, dz_re, dz_im);
        AFMM_LAUNCH_CHECK();
    }
    return AFMM_OK;
}

afmm_status launch_green(int64_t npairs, const double *r, const double *r1, const double *x, int n_modes, double *G,
                         double *Gr, double *Gx, cudaStream_t st)
{
    RecTab tab;
    make_rec_tab(&tab);
    PairParams pp;
    pp.fwd_switch = default_fwd_switch(n_modes - 1);
    pp.miller_extra = 15.0;
    const int B = 64;
    size_t sm = sizeof(double) * ((size_t)AFMM_REC_TAB + (size_t)(n_modes < 2 ? 2 : n_modes) * B);
    AFMM_CUDA(cudaFuncSetAttribute(k_green, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_green<<<nblk(npairs, B), B, sm, st>>>(npairs, r, r1, x, n_modes, tab, pp, G, Gr, Gx);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

}  // namespace afmm

namespace afmm {

// ------------------------------------------------------------------------------------
// afmm_direct_static: the all-pairs direct sum without any device allocation.
//
// Some callers cannot call cudaMalloc: a service that must keep a fixed device-memory
// footprint after start-up, code that runs while another framework's caching allocator
// has reserved almost all device memory, and code that must not risk the implicit device
// synchronisation cudaMalloc/cudaFree can cause.  For them the direct sum takes its
// scratch (the strengths scaled by the recursion constants, and the per-split partial
// sums when the field set is small) from one file-scope device array of fixed size.
// Every GPU that loads this library holds that array until the process exits.
// ------------------------------------------------------------------------------------
static __device__ __align__(256) double g_static_scratch[AFMM_STATIC_SCRATCH_DOUBLES];

// Host code may not take the address of g_static_scratch directly (it names a host-side
// stand-in); the device address comes from cudaGetSymbolAddress on every call, in the
// caller's current context, so that nothing stale survives a cudaDeviceReset or a change
// of context.  The lookup is a host-side query, cheap next to the kernels.
static afmm_status static_scratch(double **out)
{
    void *ptr = nullptr;
    AFMM_CUDA(cudaGetSymbolAddress(&ptr, g_static_scratch));
    *out = (double *)ptr;
    return AFMM_OK;
}

// qs[n][i] = q[n][i] * c_n (caller order, no permutation)
__global__ void k_scale_strengths(const double *__restrict__ q_re, const double *__restrict__ q_im, int64_t n, int nm,
                                  const RecTab tab, double *__restrict__ qs_re, double *__restrict__ qs_im)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nm) return;
    double c = tab.c[i / n];
    qs_re[i] = q_re[i] * c;
    qs_im[i] = q_im[i] * c;
}

}  // namespace afmm

extern "C" afmm_status afmm_direct_static(int64_t ns, const double *src_r, const double *src_z, int64_t nf,
                                          const double *tgt_r, const double *tgt_z, int n_modes, const double *q_re,
                                          const double *q_im, double *phi_re, double *phi_im, void *stream)
{
    using namespace afmm;
    if (ns < 1 || nf < 1 || n_modes < 1 || n_modes > AFMM_MAX_MODES) return AFMM_EINVAL;
    if (!src_r || !src_z || !tgt_r || !tgt_z || !q_re || !q_im || !phi_re || !phi_im) return AFMM_EINVAL;
    const int64_t need = 2 * (int64_t)n_modes * ns;  // scaled strengths
    if (need > AFMM_STATIC_SCRATCH_DOUBLES) return AFMM_EINVAL;
    double *scr = nullptr;
    AFMM_TRY(static_scratch(&scr));
    cudaStream_t st = (cudaStream_t)stream;
    RecTab tab;
    make_rec_tab(&tab);
    double *qs_re = scr, *qs_im = scr + (size_t)n_modes * ns;
    k_scale_strengths<<<nblk(ns * n_modes), 256, 0, st>>>(q_re, q_im, ns, n_modes, tab, qs_re, qs_im);
    AFMM_LAUNCH_CHECK();

    NearArgs a;
    memset(&a, 0, sizeof(a));
    a.fr = tgt_r;
    a.fz = tgt_z;
    a.nfield = nf;
    a.sr = src_r;
    a.sz = src_z;
    a.nsrc = ns;
    a.q_re = qs_re;
    a.q_im = qs_im;
    a.nmodes = n_modes;
    a.N = n_modes - 1;
    a.pp.fwd_switch = default_fwd_switch(n_modes - 1);
    a.pp.miller_extra = 15.0;
    a.out_perm = nullptr;
    a.o_re = phi_re;
    a.o_im = phi_im;
    // split the sources when the field set is too small to fill the GPU, as far as the
    // rest of the array holds the partial sums (every partial is written, none is read
    // before it is written, so nothing has to start at zero)
    int64_t tunits = (nf + 31) / 32, want = 152 * 8;
    int64_t room = (AFMM_STATIC_SCRATCH_DOUBLES - need) / (2 * (int64_t)n_modes * nf);
    int64_t nsplit = 1;
    if (tunits < want) {
        nsplit = (want + tunits - 1) / tunits;
        int64_t maxs = (ns + 63) / 64;
        if (nsplit > maxs) nsplit = maxs;
        if (nsplit > room) nsplit = room;
        if (nsplit < 1) nsplit = 1;
    }
    a.direct = 1;
    a.nsplit = (int)nsplit;
    a.split_len = (ns + nsplit - 1) / nsplit;
    a.nunits = tunits * nsplit;
    a.part = nsplit > 1 ? scr + need : nullptr;
    int w = near_warps(n_modes, 0);
    if (w == 0) return AFMM_EUNSUPPORTED;
    size_t sm = near_smem(n_modes, 0, w);
    AFMM_CUDA(cudaFuncSetAttribute(k_near<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_near<false><<<(unsigned)((a.nunits + w - 1) / w), w * 32, sm, st>>>(a, tab);
    AFMM_LAUNCH_CHECK();
    if (a.part) {
        int64_t tot = (int64_t)2 * n_modes * nf;
        k_split_reduce<<<nblk(tot), 256, 0, st>>>(a.part, a.nsplit, 2, n_modes, nf, nullptr, phi_re, phi_im, nullptr,
                                                  nullptr, nullptr, nullptr);
        AFMM_LAUNCH_CHECK();
    }
    return AFMM_OK;
}

