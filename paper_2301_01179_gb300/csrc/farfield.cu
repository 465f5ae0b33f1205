// farfield.cu -- the far-field half of Algorithm 1: leaf moments (Eq. analysis:moments),
// upward shifts (Eq. analysis:shift), Green's-function Taylor expansions per radial station
// (Appendix A), source-to-local operators FO/BO/FI/BI (Eq. analysis:s2l, Sec. 2.2) and
// downward local shifts (Eq. analysis:l2l).
//
// Representation (scaled by the box size h of the level; mathematically identical to the
// paper's moments S_ij and local coefficients Phi_kl):
//   moments  Shat_ij = sum_q S_q U^i W^j / j!,   U = (r_q - c_r)/h, W = -(z_q - c_z)/h
//            ( = (-1)^j S_ij / (j! h^{i+j}) )
//   locals   F_kl = h^{k+l} Phi_kl      (Phi(r, z) = sum F_kl u^k v^l, u = (r-c_r)/h, ...)
//   expansion Ehat_{a,b,c} = c! h^{a+b+c} gbar_{a,b,c}(r_big, r_small, |x|)
// so that the FO operator is  F_kl += (1/l!) sum_ij Shat_ij Ehat_{k,i,j+l}:  BO flips the sign
// of odd c (G is even in x), FI/BI exchange the first two indices of Ehat (G is symmetric in
// r <-> r1).  Every S2L application is then a plain FP64 FMA contraction.
//
// The expansions are generated per level for every occupied radial station and the twelve
// offsets (|dr|, |dz|) in 0..3, not both <= 1 (Sec. 2.2: "twelve" expansions per station),
// in box units (Eq. gfunc:scaled): gbar at (R_s + |dr|, R_s, |dz|), R_s = r_small / h.
#include <cstring>
#include <vector>
#include "common.cuh"
#include "pair.cuh"
#include "df.cuh"
#include "dd.cuh"

namespace afmm {

__host__ __device__ inline int cix(int i, int j, int M) { return i * (M + 1) - i * (i - 1) / 2 + j; }

// ------------------------------------------------------------------------------------
// shift tables (host): the child sits at +-h_child/2 from the parent centre, i.e. at
// alpha = (bit - 1/2)/2 parent-box units.
//  M2M (hat moments):   Shat^p_ij = sum_{q<=i, v<=j} Ar[br][i][q] Bz[bz][j][v] Shat^c_{i-q,j-v}
//        Ar[i][q] = C(i,q) alpha^q 2^{q-i},  Bz[j][v] = beta^v / v! 2^{v-j}, beta = -alpha_z
//  L2L (plain locals):  F^c_im = sum_{k>=i} Lr[br][i][k] sum_{l>=m} Lz[bz][m][l] F^p_kl
//        Lr[i][k] = C(k,i) 2^{-i} alpha^{k-i},  Lz[m][l] = C(l,m) 2^{-m} gamma^{l-m}
// layout: tab[((which * 2 + bit) * (M+1) + i) * (M+1) + q]
// ------------------------------------------------------------------------------------
afmm_status make_shift_tables(afmm_plan p)
{
    int M = p->M, W = M + 1;
    std::vector<double> m2m(2 * 2 * W * W, 0.0), l2l(2 * 2 * W * W, 0.0);
    auto C = [](int n, int k) {
        double b = 1.0;
        for (int t = 1; t <= k; ++t) b = b * (n - k + t) / t;
        return b;
    };
    for (int bit = 0; bit < 2; ++bit) {
        double al = (bit - 0.5) / 2.0;  // (c_child - c_parent) / h_parent
        for (int i = 0; i <= M; ++i)
            for (int q = 0; q <= M; ++q) {
                // M2M radial
                if (q <= i) m2m[((0 * 2 + bit) * W + i) * W + q] = C(i, q) * pow(al, q) * pow(2.0, q - i);
                // M2M axial, W = -(z - c)/h: beta = -al
                double be = -al, fv = 1.0;
                for (int t = 2; t <= q; ++t) fv *= t;
                if (q <= i) m2m[((1 * 2 + bit) * W + i) * W + q] = pow(be, q) / fv * pow(2.0, q - i);
                // L2L radial / axial (gamma = al for z as well)
                if (q >= i) {
                    l2l[((0 * 2 + bit) * W + i) * W + q] = C(q, i) * pow(2.0, -i) * pow(al, q - i);
                    l2l[((1 * 2 + bit) * W + i) * W + q] = C(q, i) * pow(2.0, -i) * pow(al, q - i);
                }
            }
    }
    AFMM_TRY(dalloc_t(p, &p->m2m_tab, m2m.size()));
    AFMM_TRY(dalloc_t(p, &p->l2l_tab, l2l.size()));
    AFMM_CUDA(cudaMemcpyAsync(p->m2m_tab, m2m.data(), m2m.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    AFMM_CUDA(cudaMemcpyAsync(p->l2l_tab, l2l.data(), l2l.size() * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    // the same tables as FP32 pairs (hi = nearest float, lo = the rest) for the FP64 path
    std::vector<float2> m2mf(m2m.size()), l2lf(l2l.size());
    for (size_t i = 0; i < m2m.size(); ++i) {
        float h = (float)m2m[i], g = (float)l2l[i];
        m2mf[i] = make_float2(h, (float)(m2m[i] - (double)h));
        l2lf[i] = make_float2(g, (float)(l2l[i] - (double)g));
    }
    AFMM_TRY(dalloc_t(p, &p->m2m_tab_df, m2mf.size()));
    AFMM_TRY(dalloc_t(p, &p->l2l_tab_df, l2lf.size()));
    AFMM_CUDA(cudaMemcpyAsync(p->m2m_tab_df, m2mf.data(), m2mf.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    AFMM_CUDA(cudaMemcpyAsync(p->l2l_tab_df, l2lf.data(), l2lf.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    AFMM_CUDA(cudaStreamSynchronize(p->stream));  // the host vectors die here
    return AFMM_OK;
}

// ------------------------------------------------------------------------------------
// P2M: hat moments of every leaf box (zero for boxes without source-role points)
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void k_p2m(const uint32_t *__restrict__ key, const int2 *__restrict__ rng, int64_t nbox,
                      const double *__restrict__ sr, const double *__restrict__ sz, const T *__restrict__ q_re,
                      const T *__restrict__ q_im, int64_t nsrc, int nm, int M, double r0, double z0, double h,
                      const RecTab tab, T *__restrict__ mom_re, T *__restrict__ mom_im)
{
    extern __shared__ double sm_raw[];
    T *sm = reinterpret_cast<T *>(sm_raw);
    const int nc = (M + 1) * (M + 2) / 2;
    T *mono = sm;                        // [32][nc]
    T *acc = mono + 32 * nc;             // [2][nm][nc]
    T *invf = acc + 2 * (size_t)nm * nc;  // [M+1] 1/j!
    const int npq = (nm + 1) / 2;
    int64_t b = blockIdx.x;
    if (b >= nbox) return;
    for (int i = threadIdx.x; i < 2 * nm * nc; i += blockDim.x) acc[i] = (T)0;
    if (threadIdx.x == 0) {
        double f = 1.0;
        for (int j = 0; j <= M; ++j) {
            if (j > 0) f *= j;
            invf[j] = (T)(1.0 / f);
        }
    }
    uint32_t k = key[b];
    double cr = r0 + ((double)morton_ir(k) + 0.5) * h, cz = z0 + ((double)morton_iz(k) + 0.5) * h;
    int2 R = rng[b];
    __syncthreads();
    for (int s0 = R.x; s0 < R.y; s0 += 32) {
        int cnt = min(32, R.y - s0);
        // monomials U^i W^j / j! of the chunk's points
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            T U = (T)((sr[s0 + t] - cr) / h), Wv = (T)(-(sz[s0 + t] - cz) / h);
            T ui = (T)1;
            for (int i = 0; i <= M; ++i) {
                T wj = ui;
                for (int j = 0; i + j <= M; ++j) {
                    mono[t * nc + cix(i, j, M)] = wj * invf[j];
                    wj *= Wv;
                }
                ui *= U;
            }
        }
        __syncthreads();
        for (int o = threadIdx.x; o < nm * nc; o += blockDim.x) {
            int n = o / nc, c = o % nc;
            T ar = acc[o], ai = acc[nm * nc + o];
            for (int t = 0; t < cnt; ++t) {
                T m = mono[t * nc + c];
                ar = fma(amp_at(q_re, n, s0 + t, nsrc, npq), m, ar);
                ai = fma(amp_at(q_im, n, s0 + t, nsrc, npq), m, ai);
            }
            acc[o] = ar;
            acc[nm * nc + o] = ai;
        }
        __syncthreads();
    }
    // amplitudes carry the recursion constant c_n: divide it out
    for (int o = threadIdx.x; o < nm * nc; o += blockDim.x) {
        int n = o / nc;
        T ic = (T)(1.0 / tab.c[n]);
        mom_re[(size_t)b * nm * nc + o] = acc[o] * ic;
        mom_im[(size_t)b * nm * nc + o] = acc[nm * nc + o] * ic;
    }
}

// ------------------------------------------------------------------------------------
// M2M: parent hat moments from the children (separable radial then axial shift)
// ------------------------------------------------------------------------------------
template <typename R>
__global__ void k_m2m(const int2 *__restrict__ child, const uint32_t *__restrict__ ckey, int64_t npar, int nm, int M,
                      const double *__restrict__ tab, const R *__restrict__ cre, const R *__restrict__ cim,
                      R *__restrict__ pre, R *__restrict__ pim)
{
    extern __shared__ double sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int nc = (M + 1) * (M + 2) / 2, W = M + 1;
    R *X = sm;          // [2][nc]
    R *T = X + 2 * nc;  // [4][W][W] tables
    for (int i = threadIdx.x; i < 4 * W * W; i += blockDim.x) T[i] = (R)tab[i];
    int64_t P = blockIdx.x;
    const int n = blockIdx.y;  // one block per (parent, mode)
    __syncthreads();
    if (P >= npar) return;
    int2 ch = child[P];
    if (ch.x >= ch.y) return;  // a leaf of the adaptive tree keeps its P2M moments
    {
        R accr[2] = {0, 0}, acci[2] = {0, 0};  // outputs o = tid, tid + blockDim (nc <= 2 * blockDim)
        for (int c = ch.x; c < ch.y; ++c) {
            uint32_t k = ckey[c];
            int br = morton_ir(k) & 1, bz = morton_iz(k) & 1;
            const R *Ar = T + (0 * 2 + br) * W * W, *Bz = T + (1 * 2 + bz) * W * W;
            const R *sr_ = cre + ((size_t)c * nm + n) * nc, *si_ = cim + ((size_t)c * nm + n) * nc;
            // X_{i,j} = sum_q Ar[i][q] S_{i-q, j}
            for (int o = threadIdx.x; o < nc; o += blockDim.x) {
                int i = 0, rem = o;
                while (rem >= M + 1 - i) { rem -= M + 1 - i; ++i; }
                int j = rem;
                R xr = 0, xi = 0;
                for (int q = 0; q <= i; ++q) {
                    R a = Ar[i * W + q];
                    int s = cix(i - q, j, M);
                    xr = fma(a, sr_[s], xr);
                    xi = fma(a, si_[s], xi);
                }
                X[o] = xr;
                X[nc + o] = xi;
            }
            __syncthreads();
            for (int h = 0; h < 2; ++h) {
                int o = threadIdx.x + h * blockDim.x;
                if (o >= nc) break;
                int i = 0, rem = o;
                while (rem >= M + 1 - i) { rem -= M + 1 - i; ++i; }
                int j = rem;
                for (int v = 0; v <= j; ++v) {
                    R bcoef = Bz[j * W + v];
                    int s = cix(i, j - v, M);
                    accr[h] = fma(bcoef, X[s], accr[h]);
                    acci[h] = fma(bcoef, X[nc + s], acci[h]);
                }
            }
            __syncthreads();
        }
        for (int h = 0; h < 2; ++h) {
            int o = threadIdx.x + h * blockDim.x;
            if (o >= nc) break;
            pre[((size_t)P * nm + n) * nc + o] = accr[h];
            pim[((size_t)P * nm + n) * nc + o] = acci[h];
        }
    }
}

// ------------------------------------------------------------------------------------
// L2L: child locals from the parent (overwrites; level-2 locals start at zero)
// ------------------------------------------------------------------------------------
template <typename R>
__global__ void k_l2l(const int32_t *__restrict__ parent, const uint32_t *__restrict__ key, int64_t nbox, int nm, int M,
                      const double *__restrict__ tab, const R *__restrict__ fre_p, const R *__restrict__ fim_p,
                      R *__restrict__ fre, R *__restrict__ fim)
{
    extern __shared__ double sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int nc = (M + 1) * (M + 2) / 2, W = M + 1;
    R *Y = sm;          // [2][nc]
    R *T = Y + 2 * nc;  // [4][W][W]
    for (int i = threadIdx.x; i < 4 * W * W; i += blockDim.x) T[i] = (R)tab[i];
    int64_t b = blockIdx.x;
    __syncthreads();
    if (b >= nbox) return;
    int32_t P = parent ? parent[b] : -1;
    uint32_t k = key[b];
    int br = morton_ir(k) & 1, bz = morton_iz(k) & 1;
    const R *Lr = T + (0 * 2 + br) * W * W, *Lz = T + (1 * 2 + bz) * W * W;
    const int n = blockIdx.y;  // one block per (box, mode)
    {
        R *or_ = fre + ((size_t)b * nm + n) * nc, *oi_ = fim + ((size_t)b * nm + n) * nc;
        if (P < 0) {
            for (int o = threadIdx.x; o < nc; o += blockDim.x) or_[o] = oi_[o] = (R)0;
            return;
        }
        const R *pr = fre_p + ((size_t)P * nm + n) * nc, *pi = fim_p + ((size_t)P * nm + n) * nc;
        // Y_{k,m} = sum_{l >= m} Lz[m][l] F_{k,l}
        for (int o = threadIdx.x; o < nc; o += blockDim.x) {
            int kk = 0, rem = o;
            while (rem >= M + 1 - kk) { rem -= M + 1 - kk; ++kk; }
            int m = rem;
            R yr = 0, yi = 0;
            for (int l = m; kk + l <= M; ++l) {
                R c = Lz[m * W + l];
                int s = cix(kk, l, M);
                yr = fma(c, pr[s], yr);
                yi = fma(c, pi[s], yi);
            }
            Y[o] = yr;
            Y[nc + o] = yi;
        }
        __syncthreads();
        // F^c_{i,m} = sum_{k >= i} Lr[i][k] Y_{k,m}
        for (int o = threadIdx.x; o < nc; o += blockDim.x) {
            int i = 0, rem = o;
            while (rem >= M + 1 - i) { rem -= M + 1 - i; ++i; }
            int m = rem;
            R fr = 0, fi = 0;
            for (int kk = i; kk + m <= M; ++kk) {
                R c = Lr[i * W + kk];
                int s = cix(kk, m, M);
                fr = fma(c, Y[s], fr);
                fi = fma(c, Y[nc + s], fi);
            }
            or_[o] = fr;
            oi_[o] = fi;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// FP64 path: moments and locals as FP32 pairs ([re, im] arrays of float2), the same
// operators as k_p2m / k_m2m / k_l2l above in pair arithmetic (GB300's FP64 issues at 1/61
// of FP32).  Sums are (hi, err) pairs updated by exact two-sums.
// ------------------------------------------------------------------------------------
__global__ void k_p2m_df(const uint32_t *__restrict__ key, const int2 *__restrict__ rng, int64_t nbox,
                         const double *__restrict__ sr, const double *__restrict__ sz, const float4 *__restrict__ qri,
                         int64_t nsrc, int nm, int M, double r0, double z0, double h,
                         const RecTab tab, float2 *__restrict__ mom_re, float2 *__restrict__ mom_im, int CH)
{
    extern __shared__ float4 smq[];
    const int nc = (M + 1) * (M + 2) / 2, npq = (nm + 1) / 2;
    float4 *qst = smq;                     // [CH][nm] the chunk's amplitudes (re.hi, re.lo, im.hi, im.lo)
    float2 *mono = reinterpret_cast<float2 *>(qst + (size_t)CH * nm);  // [CH][nc] U^i W^j / j!
    float2 *acc = mono + CH * nc;          // [2][nm][nc] (hi, err)
    float2 *invf = acc + 2 * (size_t)nm * nc;  // [M+1] 1/j!
    float2 *ic = invf + (M + 1);           // [nm] 1/c_n
    const int64_t b = blockIdx.x;
    if (b >= nbox) return;
    for (int i = threadIdx.x; i < 2 * nm * nc; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    for (int j = threadIdx.x; j <= M; j += blockDim.x) {
        double f = 1.0;
        for (int t = 2; t <= j; ++t) f *= t;
        const dfv v = df_from_double(1.0 / f);
        invf[j] = make_float2(v.hi, v.lo);
    }
    for (int n = threadIdx.x; n < nm; n += blockDim.x) {
        const dfv v = df_from_double(1.0 / tab.c[n]);
        ic[n] = make_float2(v.hi, v.lo);
    }
    const uint32_t k = key[b];
    const double cr = r0 + ((double)morton_ir(k) + 0.5) * h, cz = z0 + ((double)morton_iz(k) + 0.5) * h;
    const double ih = 1.0 / h;
    const int2 R = rng[b];
    __syncthreads();
    for (int s0 = R.x; s0 < R.y; s0 += CH) {
        const int cnt = min(CH, R.y - s0);
        // the chunk's amplitudes: one contiguous run of the per-source copy, split by mode
        const float4 *qc = qri + (size_t)s0 * npq * 2;
        for (int e = threadIdx.x; e < cnt * npq; e += blockDim.x) {
            const int t = e / npq, m = e - t * npq;
            const float4 qr = qc[2 * (size_t)e], qi = qc[2 * (size_t)e + 1];
            qst[t * nm + 2 * m] = make_float4(qr.x, qr.z, qi.x, qi.z);
            if (2 * m + 1 < nm) qst[t * nm + 2 * m + 1] = make_float4(qr.y, qr.w, qi.y, qi.w);
        }
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const dfv U = df_from_double((sr[s0 + t] - cr) * ih), Wv = df_from_double(-(sz[s0 + t] - cz) * ih);
            dfv ui = df_make(1.f, 0.f);
            for (int i = 0; i <= M; ++i) {
                dfv wj = ui;
                for (int j = 0; i + j <= M; ++j) {
                    const dfv m = df_mul(wj, df_make(invf[j].x, invf[j].y));
                    mono[t * nc + cix(i, j, M)] = make_float2(m.hi, m.lo);
                    wj = df_mul(wj, Wv);
                }
                ui = df_mul(ui, U);
            }
        }
        __syncthreads();
        // two outputs per thread at a time: four independent accumulation chains (each
        // output's sum keeps its order)
        for (int o0 = threadIdx.x; o0 < nm * nc; o0 += 2 * blockDim.x) {
            const int o1 = o0 + blockDim.x;
            const bool h1 = o1 < nm * nc;
            const int n0 = o0 / nc, c0 = o0 % nc, n1 = h1 ? o1 / nc : n0, c1 = h1 ? o1 % nc : c0;
            float2 ar0 = acc[o0], ai0 = acc[nm * nc + o0];
            float2 ar1 = h1 ? acc[o1] : make_float2(0.f, 0.f), ai1 = h1 ? acc[nm * nc + o1] : make_float2(0.f, 0.f);
            for (int t = 0; t < cnt; ++t) {
                const float2 m2a = mono[t * nc + c0], m2b = mono[t * nc + c1];
                const dfv ma = df_make(m2a.x, m2a.y), mb = df_make(m2b.x, m2b.y);
                const float4 qa = qst[t * nm + n0], qb = qst[t * nm + n1];
                df_acc(ar0.x, ar0.y, df_make(qa.x, qa.y), ma);
                df_acc(ai0.x, ai0.y, df_make(qa.z, qa.w), ma);
                df_acc(ar1.x, ar1.y, df_make(qb.x, qb.y), mb);
                df_acc(ai1.x, ai1.y, df_make(qb.z, qb.w), mb);
            }
            acc[o0] = ar0;
            acc[nm * nc + o0] = ai0;
            if (h1) {
                acc[o1] = ar1;
                acc[nm * nc + o1] = ai1;
            }
        }
        __syncthreads();
    }
    // the amplitudes carry the recursion constant c_n: divide it out
    for (int o = threadIdx.x; o < nm * nc; o += blockDim.x) {
        const int n = o / nc;
        const dfv c = df_make(ic[n].x, ic[n].y);
        const dfv vr = df_mul(two_sum(acc[o].x, acc[o].y), c), vi = df_mul(two_sum(acc[nm * nc + o].x, acc[nm * nc + o].y), c);
        mom_re[(size_t)b * nm * nc + o] = make_float2(vr.hi, vr.lo);
        mom_im[(size_t)b * nm * nc + o] = make_float2(vi.hi, vi.lo);
    }
}

#define SHIFT_MB 8  // modes per block of the FP32-pair shifts (the table is staged once)

// M2M in FP32 pairs: one block per (parent, 8 modes)
__global__ void k_m2m_df(const int2 *__restrict__ child, const uint32_t *__restrict__ ckey, int64_t npar, int nm, int M,
                         const float2 *__restrict__ tab, const float2 *__restrict__ cre, const float2 *__restrict__ cim,
                         float2 *__restrict__ pre, float2 *__restrict__ pim)
{
    extern __shared__ float2 smf[];
    const int nc = (M + 1) * (M + 2) / 2, W = M + 1;
    float2 *X = smf;          // [2][nc]
    float2 *T = X + 2 * nc;   // [4][W][W]
    for (int i = threadIdx.x; i < 4 * W * W; i += blockDim.x) T[i] = tab[i];
    const int64_t P = blockIdx.x;
    __syncthreads();
    if (P >= npar) return;
    const int2 ch = child[P];
    if (ch.x >= ch.y) return;  // a leaf of the adaptive tree keeps its P2M moments
    for (int n = blockIdx.y * SHIFT_MB; n < nm && n < (blockIdx.y + 1) * SHIFT_MB; ++n) {
    float2 accr[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, acci[2] = {accr[0], accr[1]};
    for (int c = ch.x; c < ch.y; ++c) {
        const uint32_t k = ckey[c];
        const int br = morton_ir(k) & 1, bz = morton_iz(k) & 1;
        const float2 *Ar = T + (0 * 2 + br) * W * W, *Bz = T + (1 * 2 + bz) * W * W;
        const float2 *sr_ = cre + ((size_t)c * nm + n) * nc, *si_ = cim + ((size_t)c * nm + n) * nc;
        // X_{i,j} = sum_q Ar[i][q] S_{i-q, j}
        for (int o = threadIdx.x; o < nc; o += blockDim.x) {
            int i = 0, rem = o;
            while (rem >= M + 1 - i) { rem -= M + 1 - i; ++i; }
            const int j = rem;
            float xr = 0.f, er = 0.f, xi = 0.f, ei = 0.f;
            for (int q = 0; q <= i; ++q) {
                const dfv av = df_make(Ar[i * W + q].x, Ar[i * W + q].y);
                const int s = cix(i - q, j, M);
                df_acc(xr, er, av, df_make(sr_[s].x, sr_[s].y));
                df_acc(xi, ei, av, df_make(si_[s].x, si_[s].y));
            }
            const dfv vr = two_sum(xr, er), vi = two_sum(xi, ei);
            X[o] = make_float2(vr.hi, vr.lo);
            X[nc + o] = make_float2(vi.hi, vi.lo);
        }
        __syncthreads();
        for (int hh = 0; hh < 2; ++hh) {
            const int o = threadIdx.x + hh * blockDim.x;
            if (o >= nc) break;
            int i = 0, rem = o;
            while (rem >= M + 1 - i) { rem -= M + 1 - i; ++i; }
            const int j = rem;
            for (int v = 0; v <= j; ++v) {
                const dfv bc = df_make(Bz[j * W + v].x, Bz[j * W + v].y);
                const int s = cix(i, j - v, M);
                df_acc(accr[hh].x, accr[hh].y, bc, df_make(X[s].x, X[s].y));
                df_acc(acci[hh].x, acci[hh].y, bc, df_make(X[nc + s].x, X[nc + s].y));
            }
        }
        __syncthreads();
    }
    for (int hh = 0; hh < 2; ++hh) {
        const int o = threadIdx.x + hh * blockDim.x;
        if (o >= nc) break;
        const dfv vr = two_sum(accr[hh].x, accr[hh].y), vi = two_sum(acci[hh].x, acci[hh].y);
        pre[((size_t)P * nm + n) * nc + o] = make_float2(vr.hi, vr.lo);
        pim[((size_t)P * nm + n) * nc + o] = make_float2(vi.hi, vi.lo);
    }
    }
}

// L2L in FP32 pairs: one block per (box, 8 modes); overwrites (level-2 locals start at zero)
__global__ void k_l2l_df(const int32_t *__restrict__ parent, const uint32_t *__restrict__ key, int64_t nbox, int nm,
                         int M, const float2 *__restrict__ tab, const float2 *__restrict__ fre_p,
                         const float2 *__restrict__ fim_p, float2 *__restrict__ fre, float2 *__restrict__ fim)
{
    extern __shared__ float2 smf[];
    const int nc = (M + 1) * (M + 2) / 2, W = M + 1;
    float2 *Y = smf;          // [2][nc]
    float2 *T = Y + 2 * nc;   // [4][W][W]
    for (int i = threadIdx.x; i < 4 * W * W; i += blockDim.x) T[i] = tab[i];
    const int64_t b = blockIdx.x;
    __syncthreads();
    if (b >= nbox) return;
    const int32_t P = parent ? parent[b] : -1;
    for (int n = blockIdx.y * SHIFT_MB; n < nm && n < (blockIdx.y + 1) * SHIFT_MB; ++n) {
    float2 *or_ = fre + ((size_t)b * nm + n) * nc, *oi_ = fim + ((size_t)b * nm + n) * nc;
    if (P < 0) {
        for (int o = threadIdx.x; o < nc; o += blockDim.x) or_[o] = oi_[o] = make_float2(0.f, 0.f);
        continue;
    }
    const uint32_t k = key[b];
    const int br = morton_ir(k) & 1, bz = morton_iz(k) & 1;
    const float2 *Lr = T + (0 * 2 + br) * W * W, *Lz = T + (1 * 2 + bz) * W * W;
    const float2 *pr = fre_p + ((size_t)P * nm + n) * nc, *pi = fim_p + ((size_t)P * nm + n) * nc;
    // Y_{k,m} = sum_{l >= m} Lz[m][l] F_{k,l}
    for (int o = threadIdx.x; o < nc; o += blockDim.x) {
        int kk = 0, rem = o;
        while (rem >= M + 1 - kk) { rem -= M + 1 - kk; ++kk; }
        const int m = rem;
        float yr = 0.f, er = 0.f, yi = 0.f, ei = 0.f;
        for (int l = m; kk + l <= M; ++l) {
            const dfv c = df_make(Lz[m * W + l].x, Lz[m * W + l].y);
            const int s = cix(kk, l, M);
            df_acc(yr, er, c, df_make(pr[s].x, pr[s].y));
            df_acc(yi, ei, c, df_make(pi[s].x, pi[s].y));
        }
        const dfv vr = two_sum(yr, er), vi = two_sum(yi, ei);
        Y[o] = make_float2(vr.hi, vr.lo);
        Y[nc + o] = make_float2(vi.hi, vi.lo);
    }
    __syncthreads();
    // F^c_{i,m} = sum_{k >= i} Lr[i][k] Y_{k,m}
    for (int o = threadIdx.x; o < nc; o += blockDim.x) {
        int i = 0, rem = o;
        while (rem >= M + 1 - i) { rem -= M + 1 - i; ++i; }
        const int m = rem;
        float fr = 0.f, er = 0.f, fi = 0.f, ei = 0.f;
        for (int kk = i; kk + m <= M; ++kk) {
            const dfv c = df_make(Lr[i * W + kk].x, Lr[i * W + kk].y);
            const int s = cix(kk, m, M);
            df_acc(fr, er, c, df_make(Y[s].x, Y[s].y));
            df_acc(fi, ei, c, df_make(Y[nc + s].x, Y[nc + s].y));
        }
        const dfv vr = two_sum(fr, er), vi = two_sum(fi, ei);
        or_[o] = make_float2(vr.hi, vr.lo);
        oi_[o] = make_float2(vi.hi, vi.lo);
    }
    __syncthreads();  // Y is rewritten for the next mode
    }
}

// ------------------------------------------------------------------------------------
// Green's-function Taylor coefficients gbar^(n)_{a,b,c}(r, r1, x), a <= A, b <= B,
// a + b + c <= P, all modes, one point per block.
//   1. G^(n) from the AGM start values and the Legendre recursion (double-double);
//   2. x-derivatives gbar_{0,0,k} by the coupled recursion of Eq. gfunc:derivatives:x;
//   3. gbar_{1,0,k}, gbar_{0,1,k}, gbar_{1,1,k} from the closed forms (Appendix A);
//      steps 2 and 3 in double-double (see the reading in gbar_block);
//   4. the Laplace equation (Eq. gfunc:laplace) in the source radius raises b and in the
//      field radius raises a.  Expanding r^2 G_rr + r G_r - n^2 G + r^2 G_xx = 0 in the
//      radial offset gives, for each Taylor coefficient,
//        (a+1)(a+2) r^2 g_{a+2} + (a+1)(2a+1) r g_{a+1} + (a^2 - n^2) g_a
//          + (c+1)(c+2) [r^2 g_{a,c+2} + 2 r g_{a-1,c+2} + g_{a-2,c+2}] = 0
//      (the same with r1, b for the source side); this three-term form is used here.
// out[((n * (A+1) + a) * (B+1) + b) * (P+1) + c], scaled by scale * c! when fact != 0.
// ------------------------------------------------------------------------------------
struct ExpJob {
    double r, r1, x;   // evaluation point (box units for S2L)
    double *out;       // slab base for this point (modes consecutive)
};

// Number types of the warp-parallel Laplace fill: FP64, or FP32 pairs (the FP64 path)
struct NumF64 {
    using T = double;
    using S = double;  // storage
    static __device__ __forceinline__ T from(double x) { return x; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T mulf(T a, float b) { return a * (double)b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T down2(T a) { return __shfl_down_sync(0xffffffffu, a, 2); }
    static __device__ __forceinline__ T idx(int src, T a) { return __shfl_sync(0xffffffffu, a, src); }
    static __device__ __forceinline__ T ld(const S *p) { return *p; }
    static __device__ __forceinline__ void st(S *p, T v) { *p = v; }
};
struct NumDF {
    using T = dfv;
    using S = float2;
    static __device__ __forceinline__ T from(double x) { return df_from_double(x); }
    static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
    static __device__ __forceinline__ T mulf(T a, float b) { return df_mulf(a, b); }
    static __device__ __forceinline__ T neg(T a) { return df_neg(a); }
    static __device__ __forceinline__ T zero() { return df_make(0.f, 0.f); }
    static __device__ __forceinline__ T down2(T a)
    {
        return df_make(__shfl_down_sync(0xffffffffu, a.hi, 2), __shfl_down_sync(0xffffffffu, a.lo, 2));
    }
    static __device__ __forceinline__ T idx(int src, T a)
    {
        return df_make(__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src));
    }
    static __device__ __forceinline__ T ld(const S *p)
    {
        const float2 v = *p;
        return df_make(v.x, v.y);
    }
    static __device__ __forceinline__ void st(S *p, T v) { *p = make_float2(v.hi, v.lo); }
};

// Step 4 of gbar_block, warp-parallel (P <= 32 NH - 1): lane l holds the Taylor coefficients
// c = l + 32 h, h < NH, of one row (a, b) of one mode.  The Laplace recursion of a row needs
// rows b+1, b, b-1, b-2 (resp. a+1 .. a-2) at c and c+2 only, so a warp walks the rows with a
// register window and a shuffle for c+2 (across the halves when NH = 2):  phase A raises b for
// a = 0, 1 (one warp per (mode, a)); phase B raises a for each b (one warp per (mode, b)),
// reading the phase-A rows and writing every entry scaled by scale * c!.  Same recursions and
// coefficients as the serial fill below.
template <class O, int NH>
__device__ __forceinline__ void fill_down2(const typename O::T (&x)[NH], typename O::T (&d)[NH], int lane)
{
    // d[h] = the value at c + 2 (zero beyond the last half)
    d[0] = O::down2(x[0]);
    if constexpr (NH == 2) {
        const typename O::T w = O::idx((lane + 2) & 31, x[1]);
        if (lane >= 30) d[0] = w;
        d[1] = O::down2(x[1]);
        if (lane >= 30) d[1] = O::zero();
    }
}

template <class O, int NH>
__device__ void gbar_fill_warp(double r, double r1, int N, int P, int A, int Bm, int Q, const double *g00,
                               const double *g10, const double *g01, const double *g11, typename O::S *out,
                               double scale, int fact, typename O::S *dtab)
{
    using T = typename O::T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int cc[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) cc[h] = lane + 32 * h;
    const int SA = (Bm + 1) * Q;
    // 1 / (r1^2 (b+1)(b+2)) and 1 / (r^2 (a+1)(a+2)), once per block (FP64 division is slow)
    typename O::S *denB = dtab, *denA = dtab + Q;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        O::st(denB + i, O::from(1.0 / (r1 * r1 * (i + 1.0) * (i + 2.0))));
        O::st(denA + i, O::from(1.0 / (r * r * (i + 1.0) * (i + 2.0))));
    }
    __syncthreads();
    const T r1d = O::from(r1), r1s = O::from(r1 * r1), r1x2 = O::from(2.0 * r1);
    const T rd = O::from(r), rs = O::from(r * r), rx2 = O::from(2.0 * r);
    float cc2[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) cc2[h] = (float)((cc[h] + 1) * (cc[h] + 2));
    // phase A: rows (a, b), a <= 1, unscaled
    const int na = A >= 1 ? 2 : 1;
    for (int task = warp; task < (N + 1) * na; task += nw) {
        const int n = task / na, a = task % na;
        typename O::S *E = out + (size_t)n * (A + 1) * SA + (size_t)a * SA;
        const float n2 = (float)(n * n);
        const double *gb0 = a == 0 ? g00 : g10, *gb1 = a == 0 ? g01 : g11;
        T R0[NH], R1[NH], Rm1[NH], Rm2[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const int c = cc[h];
            R0[h] = c <= P - a ? O::from(gb0[n * Q + c]) : O::zero();                    // b = 0
            R1[h] = (Bm >= 1 && c <= P - a - 1) ? O::from(gb1[n * Q + c]) : O::zero();  // b = 1
            Rm1[h] = Rm2[h] = O::zero();                                                 // b - 1, b - 2
            if (c <= P - a) O::st(E + c, R0[h]);
            if (Bm >= 1 && c <= P - a - 1) O::st(E + Q + c, R1[h]);
        }
        for (int b = 0; b + 2 <= Bm && a + b + 2 <= P; ++b) {
            const T den = O::ld(denB + b);
            T d0[NH], dm1[NH], dm2[NH];
            fill_down2<O, NH>(R0, d0, lane);
            fill_down2<O, NH>(Rm1, dm1, lane);
            fill_down2<O, NH>(Rm2, dm2, lane);
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                T sv = O::add(O::mulf(O::mul(r1d, R1[h]), (float)((b + 1) * (2 * b + 1))), O::mulf(R0[h], (float)(b * b) - n2));
                T t = O::mul(r1s, d0[h]);
                if (b >= 1) t = O::add(t, O::mul(r1x2, dm1[h]));
                if (b >= 2) t = O::add(t, dm2[h]);
                sv = O::add(sv, O::mulf(t, cc2[h]));
                const T R2 = O::neg(O::mul(sv, den));
                if (a + b + 2 + cc[h] <= P) O::st(E + (size_t)(b + 2) * Q + cc[h], R2);
                Rm2[h] = Rm1[h];
                Rm1[h] = R0[h];
                R0[h] = R1[h];
                R1[h] = R2;
            }
        }
    }
    __syncthreads();
    // phase B: raise a for each (mode, b); write every entry scaled
    T fc[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        double fcd = scale;
        if (fact)
            for (int k = 2; k <= cc[h]; ++k) fcd *= k;
        fc[h] = O::from(fcd);
    }
    for (int task = warp; task < (N + 1) * (Bm + 1); task += nw) {
        const int n = task / (Bm + 1), b = task % (Bm + 1);
        if (b > P) continue;  // warp-uniform
        typename O::S *E = out + (size_t)n * (A + 1) * SA + (size_t)b * Q;
        const float n2 = (float)(n * n);
        T R0[NH], R1[NH], Rm1[NH], Rm2[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const int c = cc[h];
            R0[h] = c <= P - b ? O::ld(E + c) : O::zero();                       // a = 0
            R1[h] = (A >= 1 && c <= P - b - 1) ? O::ld(E + SA + c) : O::zero();  // a = 1
            Rm1[h] = Rm2[h] = O::zero();
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const int c = cc[h];
            if (c <= P - b) O::st(E + c, O::mul(R0[h], fc[h]));
            if (A >= 1 && c <= P - b - 1) O::st(E + SA + c, O::mul(R1[h], fc[h]));
        }
        for (int a = 0; a + 2 <= A && a + 2 + b <= P; ++a) {
            const T den = O::ld(denA + a);
            T d0[NH], dm1[NH], dm2[NH];
            fill_down2<O, NH>(R0, d0, lane);
            fill_down2<O, NH>(Rm1, dm1, lane);
            fill_down2<O, NH>(Rm2, dm2, lane);
#pragma unroll
            for (int h = 0; h < NH; ++h) {
                T sv = O::add(O::mulf(O::mul(rd, R1[h]), (float)((a + 1) * (2 * a + 1))), O::mulf(R0[h], (float)(a * a) - n2));
                T t = O::mul(rs, d0[h]);
                if (a >= 1) t = O::add(t, O::mul(rx2, dm1[h]));
                if (a >= 2) t = O::add(t, dm2[h]);
                sv = O::add(sv, O::mulf(t, cc2[h]));
                const T R2 = O::neg(O::mul(sv, den));
                if (a + 2 + b + cc[h] <= P) O::st(E + (size_t)(a + 2) * SA + cc[h], O::mul(R2, fc[h]));
                Rm2[h] = Rm1[h];
                Rm1[h] = R0[h];
                R0[h] = R1[h];
                R1[h] = R2;
            }
        }
    }
}

// Legendre start values and sequence G^(n), n = 0..N, in double-double (one thread): the same
// AGM start values as pair.cuh (G^(0) = 1 / (2 AGM(rho_+, rho_-)), G^(1) from the
// half-difference sum) and the recursion of Eq. gfunc:recursion, forward where
// 2 max(N, 2) acosh(chi) <= 16 (error growth e^16 against 2^-104), otherwise Miller's backward
// recursion from L = N + ceil(30 / acosh chi) + 10 (start error e^-60), normalised by G^(0).
__device__ void dd_green_sequence(double r, double r1, double x, int N, ddv *G)
{
    const ddv dr = dd_two_sum(r, -r1), sr = dd_two_sum(r, r1), x2 = dd_two_prod(x, x);
    const ddv rm2 = dd_add(dd_mul(dr, dr), x2), rp2 = dd_add(dd_mul(sr, sr), x2);
    const ddv w2 = dd_mul_d(dd_two_prod(r, r1), 2.0);  // 2 r r1
    const ddv t = dd_div(rm2, w2);                     // chi - 1
    ddv a = dd_sqrt(rp2), b = dd_sqrt(rm2), csum = dd_make(0.0);
    double wgt = 1.0;
    for (int it = 0; it < 60; ++it) {
        const ddv c = dd_mul_d(dd_sub(a, b), 0.5);
        csum = dd_add(csum, dd_mul_d(dd_mul(c, c), wgt));
        wgt *= 2.0;
        const ddv an = dd_mul_d(dd_add(a, b), 0.5);
        b = dd_sqrt(dd_mul(a, b));
        a = an;
        if (fabs(c.hi) <= 1e-17 * a.hi) break;
    }
    const ddv G0 = dd_div(dd_make(0.5), a);
    const double td = t.hi;
    const double af = log1p(td + sqrt(td * (td + 2.0)));  // acosh(chi), decides the regime only
    const int Nr = N < 2 ? 2 : N;
    if (2.0 * Nr * af <= 16.0) {
        G[0] = G0;
        if (N >= 1) G[1] = dd_div(dd_mul(G0, csum), w2);
        for (int n = 2; n <= N; ++n) {
            const ddv up = dd_mul_d(dd_add(G[n - 1], dd_mul(t, G[n - 1])), 4.0 * (n - 1));
            G[n] = dd_mul(dd_sub(up, dd_mul_d(G[n - 2], 2.0 * n - 3.0)), dd_recip_int(2.0 * n - 1.0));
        }
        return;
    }
    const int L = N + (int)ceil(30.0 / af) + 10;
    ddv qh = dd_make(0.0), ql = dd_make(1.0);  // q_n, q_{n-1}
    if (L - 1 <= N) G[L - 1] = ql;
    for (int n = L; n >= 2; --n) {
        const ddv up = dd_mul_d(dd_add(ql, dd_mul(t, ql)), 4.0 * (n - 1));
        const ddv qn = dd_mul(dd_sub(up, dd_mul_d(qh, 2.0 * n - 1.0)), dd_recip_int(2.0 * n - 3.0));
        qh = ql;
        ql = qn;
        if (n - 2 <= N) G[n - 2] = qn;
        if (fabs(qn.hi) > 1e200) {
            qh = dd_mul_d(qh, 1e-200);
            ql = dd_mul_d(ql, 1e-200);
            const int top = L - 1 <= N ? L - 1 : N;
            for (int m = n - 2 < 0 ? 0 : n - 2; m <= top; ++m) G[m] = dd_mul_d(G[m], 1e-200);
        }
    }
    const ddv s = dd_div(G0, G[0]);
    for (int n = 0; n <= N; ++n) G[n] = dd_mul(G[n], s);
}

// sum of products a_i * b_i into (H, L): each product exact (FMA two-product), its high part
// added by two-sum, the low parts summed in FP64; renormalised by the caller
__device__ __forceinline__ void dd_acc2(double &H, double &L, ddv a, ddv b)
{
    const ddv p = dd_two_prod(a.hi, b.hi);
    const double cross = __fma_rn(a.hi, b.lo, __dmul_rn(a.lo, b.hi));
    const ddv s = dd_two_sum(H, p.hi);
    L = __dadd_rn(L, __dadd_rn(__dadd_rn(s.lo, p.lo), cross));
    H = s.hi;
}

// shared-memory layout of gbar_block (byte offsets, 16-byte aligned)
struct GbarSmem {
    size_t tv, tvt, b00, b01, g10, g11, G, rk, dtab, total;
};
__host__ __device__ inline size_t gb_al(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline GbarSmem gbar_layout(int N, int P, bool dd)
{
    const size_t nmw = (size_t)(N < 1 ? 1 : N) + 1, Q = (size_t)P + 1, es = dd ? 16 : 12;
    GbarSmem L;
    L.tv = 0;                                  // double-double Taylor vectors [12][Q]
    L.tvt = gb_al(L.tv + 12 * Q * 16);         // their products' factors in the base number type [8][Q]
    L.b00 = gb_al(L.tvt + 8 * Q * es);         // gbar_{0,0,k}: base number type [nmw][Q], then FP64
    L.b01 = gb_al(L.b00 + nmw * Q * es);       // gbar_{0,1,k}: the same
    L.g10 = gb_al(L.b01 + nmw * Q * es);       // gbar_{1,0,k}: FP64 [nmw][Q]
    L.g11 = gb_al(L.g10 + nmw * Q * 8);        // gbar_{1,1,k}: FP64 [nmw][Q]
    L.G = gb_al(L.g11 + nmw * Q * 8);          // G^(n), double-double [nmw]
    L.rk = gb_al(L.G + nmw * 16);              // 1 / (k + 1), double-double [Q]
    L.dtab = gb_al(L.rk + Q * 16);             // the fill's denominators [2 Q]
    L.total = gb_al(L.dtab + 2 * Q * 8);
    return L;
}

// base-type values to their nearest FP64 values in place (element i moves from byte 12 i or
// 16 i to byte 8 i): rounds of blockDim elements, each read completely before any write
template <class B>
__device__ void base_to_double_inplace(typename B::S *a, int count)
{
    double *d = reinterpret_cast<double *>(a);
    for (int base = 0; base < count; base += blockDim.x) {
        const int i = base + threadIdx.x;
        double v = 0.0;
        if (i < count) v = B::nearest(a[i]);
        __syncthreads();
        if (i < count) d[i] = v;
        __syncthreads();
    }
}

template <bool DDX>
__device__ void gbar_block(double r, double r1, double x, int N, int P, int A, int Bm, const RecTab &tab,
                           const PairParams &pp, double *sm, double *out, double scale, int fact,
                           float2 *dfout = nullptr, const ddv *Gpre = nullptr)
{
    using B = BaseNum<DDX>;
    using BS = typename B::S;
    (void)tab;
    (void)pp;
    const int Nw = N < 1 ? 1 : N;
    const int nmw = Nw + 1;
    const int Q = P + 1;
    // Reading of Appendix A (no precision given): the x-recursion and the closed first-derivative
    // forms couple G^(n) and G^(n-1) through their difference, which cancels as chi -> 1, and the
    // Laplace recursion (step 4) carries the errors of these base columns into the high mixed
    // coefficients: in FP64 the base columns of axially adjacent boxes on fine levels lose up to
    // ten digits at modes 0..32 and beyond.  Steps 1-3 therefore carry about 72 bits: start values
    // and Taylor vectors in double-double, the convolutions of steps 2-3 as triple-floats on the
    // FP32 pipe (DDX = false: about 72 bits, enough through modes 0..32) or in double-double
    // (DDX = true, for more modes at the FP64 parity bar).  The Laplace recursion, stable given
    // accurate base columns, stays in FP64 / FP32 pairs.
    const GbarSmem Ly = gbar_layout(N, P, DDX);
    uint8_t *base = reinterpret_cast<uint8_t *>(sm);
    ddv *tv = reinterpret_cast<ddv *>(base + Ly.tv);
    BS *tvt = reinterpret_cast<BS *>(base + Ly.tvt);
    BS *b00 = reinterpret_cast<BS *>(base + Ly.b00);
    BS *b01 = reinterpret_cast<BS *>(base + Ly.b01);
    double *g10 = reinterpret_cast<double *>(base + Ly.g10);
    double *g11 = reinterpret_cast<double *>(base + Ly.g11);
    ddv *G = reinterpret_cast<ddv *>(base + Ly.G);
    ddv *rk = reinterpret_cast<ddv *>(base + Ly.rk);
    // 1. G^(n), n = 0..Nw (precomputed per expansion, or here by one thread)
    if (Gpre) {
        for (int n = threadIdx.x; n <= Nw; n += blockDim.x) G[n] = Gpre[n];
    } else if (threadIdx.x == 0) {
        dd_green_sequence(r, r1, x, Nw, G);
    }
    for (int k = threadIdx.x; k < Q; k += blockDim.x) rk[k] = dd_recip_int((double)(k + 1));
    // 2. Taylor coefficients in x of 1/rho_pm^2 and the rational factors of Appendix A
    ddv *vp = tv, *vm = tv + Q, *fxp = tv + 2 * Q, *fxm = tv + 3 * Q, *hp = tv + 4 * Q, *hm = tv + 5 * Q;
    ddv *hp1 = tv + 6 * Q, *hm1 = tv + 7 * Q, *dhp = tv + 8 * Q, *dhm = tv + 9 * Q;
    ddv *wsp = tv + 10 * Q, *wsm = tv + 11 * Q;  // (c - x^2) v^2 for the r1 derivative of hp, hm
    const ddv xd = dd_make(x), r1d = dd_make(r1);
    const ddv cc = dd_mul(dd_two_sum(r, -r1), dd_two_sum(r, r1));  // r^2 - r1^2
    const ddv cmx = dd_sub(cc, dd_two_prod(x, x)), cpx = dd_neg(dd_add(cc, dd_two_prod(x, x)));
    if (threadIdx.x < 2) {
        const int sgn = threadIdx.x;
        const ddv aa = dd_two_sum(r, sgn == 0 ? r1 : -r1);
        ddv *v = sgn == 0 ? vp : vm;
        const ddv u0 = dd_add(dd_mul(aa, aa), dd_two_prod(x, x));
        const ddv iu0 = dd_div(dd_make(1.0), u0);
        v[0] = iu0;
        if (P >= 1) v[1] = dd_mul_d(dd_mul(xd, dd_mul(iu0, iu0)), -2.0);
        for (int q = 2; q <= P; ++q) v[q] = dd_neg(dd_mul(dd_add(dd_mul_d(dd_mul(xd, v[q - 1]), 2.0), v[q - 2]), iu0));
    }
    __syncthreads();
    // (c - x^2) w for a Taylor vector w: coefficient q
    auto cm = [&](const ddv *w, ddv c0, int q) {
        ddv s = dd_mul(c0, w[q]);
        if (q >= 1) s = dd_sub(s, dd_mul_d(dd_mul(xd, w[q - 1]), 2.0));
        if (q >= 2) s = dd_sub(s, w[q - 2]);
        return s;
    };
    for (int q = threadIdx.x; q <= P; q += blockDim.x) {
        fxp[q] = dd_add(dd_mul(xd, vp[q]), q >= 1 ? vp[q - 1] : dd_make(0.0));
        fxm[q] = dd_add(dd_mul(xd, vm[q]), q >= 1 ? vm[q - 1] : dd_make(0.0));
        hp[q] = cm(vp, cmx, q);
        hm[q] = cm(vm, cmx, q);
        hp1[q] = cm(vp, cpx, q);
        hm1[q] = cm(vm, cpx, q);
        ddv s0 = dd_make(0.0), s1 = dd_make(0.0);
        for (int t = 0; t <= q; ++t) {
            s0 = dd_fma(vp[t], vp[q - t], s0);
            s1 = dd_fma(vm[t], vm[q - t], s1);
        }
        wsp[q] = s0;
        wsm[q] = s1;
    }
    __syncthreads();
    // d/dr1 of (c - x^2)/((r + s r1)^2 + x^2) = -2 r1 v - 2 s (r + s r1) (c - x^2) v^2
    for (int q = threadIdx.x; q <= P; q += blockDim.x) {
        const ddv ap = dd_two_sum(r, r1), am = dd_two_sum(r, -r1);
        const ddv tp = cm(wsp, cmx, q), tm = cm(wsm, cmx, q);
        dhp[q] = dd_sub(dd_mul_d(dd_mul(r1d, vp[q]), -2.0), dd_mul_d(dd_mul(ap, tp), 2.0));
        dhm[q] = dd_add(dd_mul_d(dd_mul(r1d, vm[q]), -2.0), dd_mul_d(dd_mul(am, tm), 2.0));
    }
    __syncthreads();
    // the convolutions below use the factor pairs f+ + f- (mode n) and f+ - f- (mode n - 1):
    // sum_q (g^n + g^m) f+_q + (g^n - g^m) f-_q = sum_q g^n (f+ + f-)_q + g^m (f+ - f-)_q
    BS *tfxp = tvt, *tfxm = tvt + Q, *thp = tvt + 2 * Q, *thm = tvt + 3 * Q, *thp1 = tvt + 4 * Q, *thm1 = tvt + 5 * Q;
    BS *tdhp = tvt + 6 * Q, *tdhm = tvt + 7 * Q;
    for (int q = threadIdx.x; q <= P; q += blockDim.x) {
        tfxp[q] = B::from(dd_add(fxp[q], fxm[q]));
        tfxm[q] = B::from(dd_sub(fxp[q], fxm[q]));
        thp[q] = B::from(dd_add(hp[q], hm[q]));
        thm[q] = B::from(dd_sub(hp[q], hm[q]));
        thp1[q] = B::from(dd_add(hp1[q], hm1[q]));
        thm1[q] = B::from(dd_sub(hp1[q], hm1[q]));
        tdhp[q] = B::from(dd_add(dhp[q], dhm[q]));
        tdhm[q] = B::from(dd_sub(dhp[q], dhm[q]));
    }
    for (int n = threadIdx.x; n <= Nw; n += blockDim.x) b00[n * Q] = B::from(G[n]);
    __syncthreads();
    // 3a. x-recursion, coupled in n (G^(-1) = G^(1))
    for (int k = 0; k < P; ++k) {
        for (int n = threadIdx.x; n <= Nw; n += blockDim.x) {
            const int m = n == 0 ? 1 : n - 1;
            typename B::A S = B::zero();
            for (int q = 0; q <= k; ++q) {
                B::acc(S, b00[n * Q + k - q], tfxp[q]);
                B::acc(S, b00[m * Q + k - q], tfxm[q]);
            }
            b00[n * Q + k + 1] = B::from(dd_mul(dd_mul_d(B::fin(S), n - 0.5), rk[k]));
        }
        __syncthreads();
    }
    // 3b. first r and r1 derivatives, one task per (mode, order)
    const ddv i2r = dd_recip_int(2.0 * r), i2r1 = dd_recip_int(2.0 * r1);
    for (int task = threadIdx.x; task < nmw * P; task += blockDim.x) {
        const int n = task / P, k = task % P;
        const int m = n == 0 ? 1 : n - 1;
        typename B::A S1 = B::zero(), S2 = B::zero();
        for (int q = 0; q <= k; ++q) {
            const BS gn = b00[n * Q + k - q], gm = b00[m * Q + k - q];
            B::acc(S1, gn, thp[q]);
            B::acc(S1, gm, thm[q]);
            B::acc(S2, gn, thp1[q]);
            B::acc(S2, gm, thm1[q]);
        }
        const ddv g = B::to(b00[n * Q + k]);
        g10[n * Q + k] = dd_mul(dd_sub(dd_mul_d(B::fin(S1), n - 0.5), g), i2r).hi;
        b01[n * Q + k] = B::from(dd_mul(dd_sub(dd_mul_d(B::fin(S2), n - 0.5), g), i2r1));
    }
    __syncthreads();
    // 3c. mixed, one task per (mode, order)
    for (int task = threadIdx.x; task < nmw * (P - 1); task += blockDim.x) {
        const int n = task / (P - 1), k = task % (P - 1);
        const int m = n == 0 ? 1 : n - 1;
        typename B::A S = B::zero();
        for (int q = 0; q <= k; ++q) {
            B::acc(S, b00[n * Q + k - q], tdhp[q]);
            B::acc(S, b00[m * Q + k - q], tdhm[q]);
            B::acc(S, b01[n * Q + k - q], thp[q]);
            B::acc(S, b01[m * Q + k - q], thm[q]);
        }
        const ddv g = B::to(b01[n * Q + k]);
        g11[n * Q + k] = dd_mul(dd_sub(dd_mul_d(B::fin(S), n - 0.5), g), i2r).hi;
    }
    __syncthreads();
    // the base columns gbar_{0,0,k} and gbar_{0,1,k} as FP64 for the fill
    base_to_double_inplace<B>(b00, nmw * Q);
    base_to_double_inplace<B>(b01, nmw * Q);
    const double *g00 = reinterpret_cast<const double *>(b00);
    const double *g01 = reinterpret_cast<const double *>(b01);
    if (P <= 63) {  // warp-parallel fill (every order a plan accepts: 2M <= 32)
        double *dtab = reinterpret_cast<double *>(base + Ly.dtab);  // [2 Q]
        if (P <= 31) {
            if (dfout)
                gbar_fill_warp<NumDF, 1>(r, r1, N, P, A, Bm, Q, g00, g10, g01, g11, dfout, scale, fact,
                                         reinterpret_cast<float2 *>(dtab));
            else
                gbar_fill_warp<NumF64, 1>(r, r1, N, P, A, Bm, Q, g00, g10, g01, g11, out, scale, fact, dtab);
        } else {
            if (dfout)
                gbar_fill_warp<NumDF, 2>(r, r1, N, P, A, Bm, Q, g00, g10, g01, g11, dfout, scale, fact,
                                         reinterpret_cast<float2 *>(dtab));
            else
                gbar_fill_warp<NumF64, 2>(r, r1, N, P, A, Bm, Q, g00, g10, g01, g11, out, scale, fact, dtab);
        }
        return;
    }
    if (dfout) return;  // not reached: FP32-pair expansions come from plans (P = 2M <= 32)
    // 4. Laplace recursions, one mode per thread, into the output slab
    const int SA = (Bm + 1) * Q;  // stride of a
    for (int n = threadIdx.x; n <= N; n += blockDim.x) {
        double *E = out + (size_t)n * (A + 1) * SA;
        double n2 = (double)n * n;
#define EI(a_, b_, c_) E[(size_t)(a_) * SA + (b_) * Q + (c_)]
        for (int c = 0; c <= P; ++c) EI(0, 0, c) = g00[n * Q + c];
        if (A >= 1)
            for (int c = 0; c + 1 <= P; ++c) EI(1, 0, c) = g10[n * Q + c];
        if (Bm >= 1)
            for (int c = 0; c + 1 <= P; ++c) EI(0, 1, c) = g01[n * Q + c];
        if (A >= 1 && Bm >= 1)
            for (int c = 0; c + 2 <= P; ++c) EI(1, 1, c) = g11[n * Q + c];
        double r1s = r1 * r1, ir1s = 1.0 / r1s, rs = r * r, irs = 1.0 / rs;
        for (int a = 0; a <= 1 && a <= A; ++a)
            for (int b = 0; b + 2 <= Bm && a + b + 2 <= P; ++b) {
                double den = ir1s / ((b + 1.0) * (b + 2.0));
                for (int c = 0; a + b + 2 + c <= P; ++c) {
                    double s = (b + 1.0) * (2.0 * b + 1.0) * r1 * EI(a, b + 1, c) + (b * (double)b - n2) * EI(a, b, c);
                    double t = r1s * EI(a, b, c + 2);
                    if (b >= 1) t += 2.0 * r1 * EI(a, b - 1, c + 2);
                    if (b >= 2) t += EI(a, b - 2, c + 2);
                    s += (c + 1.0) * (c + 2.0) * t;
                    EI(a, b + 2, c) = -s * den;
                }
            }
        for (int a = 0; a + 2 <= A; ++a)
            for (int b = 0; b <= Bm && a + 2 + b <= P; ++b) {
                double den = irs / ((a + 1.0) * (a + 2.0));
                for (int c = 0; a + 2 + b + c <= P; ++c) {
                    double s = (a + 1.0) * (2.0 * a + 1.0) * r * EI(a + 1, b, c) + (a * (double)a - n2) * EI(a, b, c);
                    double t = rs * EI(a, b, c + 2);
                    if (a >= 1) t += 2.0 * r * EI(a - 1, b, c + 2);
                    if (a >= 2) t += EI(a - 2, b, c + 2);
                    s += (c + 1.0) * (c + 2.0) * t;
                    EI(a + 2, b, c) = -s * den;
                }
            }
        if (fact || scale != 1.0) {
            for (int a = 0; a <= A; ++a)
                for (int b = 0; b <= Bm && a + b <= P; ++b) {
                    double f = scale;
                    for (int c = 0; a + b + c <= P; ++c) {
                        if (fact && c > 0) f *= c;
                        EI(a, b, c) *= f;
                    }
                }
        }
#undef EI
    }
}

static size_t gbar_smem(int N, int P, bool dd) { return gbar_layout(N, P, dd).total; }

// double-double base columns beyond 33 modes, in every precision: there the cancellation of
// the base columns outruns the triple-float's ~72 bits (measured with triple-floats at modes
// 0..64, order 14: 1.3e-10 per mode on a depth-5 tree, FP64 path; 4.9e-5 at mode 64 on the
// depth-10 tree of 4e6 rings, MIXED path, whose other errors are ~1e-7)
static bool gexp_dd(afmm_plan p) { return p->N > 32; }

// unit entry point: one point per block, dense (P+1)^3 per mode
__global__ void k_gbar_points(int64_t np, const double *__restrict__ r, const double *__restrict__ r1,
                              const double *__restrict__ x, int nm, int P, const RecTab tab, PairParams pp, double *out)
{
    extern __shared__ double sm[];
    int64_t pidx = blockIdx.x;
    if (pidx >= np) return;
    size_t per = (size_t)nm * (P + 1) * (P + 1) * (P + 1);
    // evaluate in units of a power of two sigma near the pair's distance (exact scaling), so
    // that the triple-float words stay far inside the FP32 range, then undo it with the
    // homogeneity gbar_{i,j,k}(sigma y) = sigma^{-1-i-j-k} gbar_{i,j,k}(y) (Eq. gfunc:scaled)
    const double rr = r[pidx], rr1 = r1[pidx], xx = fabs(x[pidx]);
    const double dist = fmin(hypot(rr - rr1, xx), fmin(rr, rr1));
    const int e = dist > 0.0 ? ilogb(dist) : 0;
    gbar_block<true>(ldexp(rr, -e), ldexp(rr1, -e), ldexp(xx, -e), nm - 1, P, P, P, tab, pp, sm, out + pidx * per, 1.0,
                     0);
    __syncthreads();
    for (size_t i = threadIdx.x; i < per; i += blockDim.x) {
        const int Q = P + 1;
        const int c = (int)(i % Q), b = (int)((i / Q) % Q), a = (int)((i / ((size_t)Q * Q)) % Q);
        out[pidx * per + i] = ldexp(out[pidx * per + i], -e * (1 + a + b + c));
    }
    // odd x-derivatives change sign for x < 0 (G even in x)
    if (x[pidx] < 0.0) {
        __syncthreads();
        for (size_t i = threadIdx.x; i < per; i += blockDim.x)
            if ((i % (P + 1)) & 1) out[pidx * per + i] = -out[pidx * per + i];
    }
}

// Start values of the S2L expansions of one level: G^(n), n = 0..max(N, 1), at
// (R_s + a, R_s, b) in box units for every (station, slot a*4+b), one thread each (the serial
// double-double recursion would otherwise hold a whole block).  Out: [station][16][nmw].
__global__ void k_gexp_start(const int32_t *__restrict__ col_of_station, const int32_t *__restrict__ station_of_col,
                             int nstation, int level, double r0h, int Nw, ddv *__restrict__ gstart)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nstation * 16) return;
    const int st = t / 16, slot = t % 16, a = slot / 4, b = slot % 4;
    if (a <= 1 && b <= 1) return;
    const int col = col_of_station[st], nl = 1 << level;
    if (col + a >= nl || station_of_col[col + a] < 0) return;
    const double Rs = r0h + col + 0.5, Rb = Rs + a;
    dd_green_sequence(Rb, Rs, (double)b, Nw, gstart + (size_t)t * (Nw + 1));
}

// S2L expansions of one level: block = (station, slot a*4+b)
template <bool DDX>
__global__ void k_gexp_level(const int32_t *__restrict__ col_of_station, const int32_t *__restrict__ station_of_col,
                             int nstation, int level, double r0h, double h, int nm, int M, const RecTab tab,
                             PairParams pp, double *gexp, float2 *gexp_df, const ddv *__restrict__ gstart)
{
    extern __shared__ double sm[];
    int st = blockIdx.x / 16, slot = blockIdx.x % 16;
    int a = slot / 4, b = slot % 4;
    if (st >= nstation || (a <= 1 && b <= 1)) return;
    int col = col_of_station[st];
    int nl = 1 << level;
    if (col + a >= nl || station_of_col[col + a] < 0) return;
    double Rs = r0h + col + 0.5, Rb = Rs + a;
    size_t slab = (size_t)(M + 1) * (M + 1) * (2 * M + 1);
    double *out = gexp ? gexp + ((size_t)st * 16 + slot) * nm * slab : nullptr;
    float2 *dout = gexp_df ? gexp_df + ((size_t)st * 16 + slot) * nm * slab : nullptr;
    const int nmw = (nm - 1 < 1 ? 1 : nm - 1) + 1;
    gbar_block<DDX>(Rb, Rs, (double)b, nm - 1, 2 * M, M, M, tab, pp, sm, out, 1.0 / h, 1, dout,
                    gstart + ((size_t)st * 16 + slot) * nmw);
}

// the start values of a level, then its expansions
static afmm_status launch_gexp_level(afmm_plan p, int l, size_t gsm, double *gexp, float2 *gexp_df)
{
    const Level &v = p->lv[l];
    const double h = p->L / (double)(1 << l);
    const int Nw = p->N < 1 ? 1 : p->N;
    const int nt = v.nstation * 16;
    k_gexp_start<<<(unsigned)((nt + 63) / 64), 64, 0, p->stream>>>(v.col_of_station, v.station_of_col, v.nstation, l,
                                                                   p->r0 / h, Nw, reinterpret_cast<ddv *>(p->gstart));
    AFMM_LAUNCH_CHECK();
    if (gexp_dd(p))
        k_gexp_level<true><<<(unsigned)nt, 256, gsm, p->stream>>>(v.col_of_station, v.station_of_col, v.nstation, l,
                                                                  p->r0 / h, h, p->nmodes, p->M, *p->rec, p->pp, gexp,
                                                                  gexp_df, reinterpret_cast<const ddv *>(p->gstart));
    else
        k_gexp_level<false><<<(unsigned)nt, 256, gsm, p->stream>>>(v.col_of_station, v.station_of_col, v.nstation, l,
                                                                   p->r0 / h, h, p->nmodes, p->M, *p->rec, p->pp, gexp,
                                                                   gexp_df, reinterpret_cast<const ddv *>(p->gstart));
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

afmm_status launch_green_expansion(int64_t npts, const double *r, const double *r1, const double *x, int n_modes, int P,
                                   double *out, cudaStream_t st)
{
    RecTab tab;
    make_rec_tab(&tab);
    PairParams pp;
    pp.fwd_switch = default_fwd_switch(n_modes - 1);
    pp.miller_extra = 15.0;
    size_t per = (size_t)n_modes * (P + 1) * (P + 1) * (P + 1);
    AFMM_CUDA(cudaMemsetAsync(out, 0, per * npts * sizeof(double), st));
    size_t sm = gbar_smem(n_modes - 1, P, true);
    if (sm > 227 * 1024) return AFMM_EUNSUPPORTED;  // shared-memory working set of one point
    AFMM_CUDA(cudaFuncSetAttribute(k_gbar_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_gbar_points<<<(unsigned)npts, 128, sm, st>>>(npts, r, r1, x, n_modes, P, tab, pp, out);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}


template <typename R>
struct S2LArgs {
    const int32_t *unit_box, *unit_col, *s2l, *station_of_col;
    int64_t nunit;
    int level, nm, M, nc;
    const double *gexp;
    const R *mom_re, *mom_im;
    R *loc_re, *loc_im;
    const float2 *gexp_df, *mom_df_re, *mom_df_im;  // FP32-pair moments and expansions (FP64 path)
    float2 *locd_re, *locd_im;                      // FP32-pair locals (FP64 path)
};

template <typename R, int KPT>
__global__ void __launch_bounds__(128) k_s2l(const S2LArgs<R> a)
{
    extern __shared__ double sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int M = a.M, nc = a.nc, W = M + 1, C2 = 2 * M + 1;
    const int slab = W * W * C2;
    R *S = sm;                  // [W][W][C2] oriented expansion
    R *Ir = S + slab;           // [nc][32]
    R *Ii = Ir + (size_t)nc * 32;
    __shared__ int bx[32];
    __shared__ int src[32];
    __shared__ int any;
    const int64_t u = blockIdx.x;
    const int n = blockIdx.y;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    if (threadIdx.x < 32) bx[threadIdx.x] = a.unit_box[u * 32 + threadIdx.x];
    const int ucol = a.unit_col[u];
    const int col = ucol & 0xffff, pz = (ucol >> 30) & 1, pr = col & 1;
    const int nl = 1 << a.level;
    R accr[KPT], acci[KPT];
    int base[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        accr[q] = (R)0;
        acci[q] = (R)0;
        int kl = grp + 4 * q;
        int k = 0, rem = kl < nc ? kl : 0;
        while (rem >= M + 1 - k) { rem -= M + 1 - k; ++k; }
        base[q] = (k * W) * C2 + rem;  // + i*C2 + j
    }
    const size_t slabn = (size_t)slab;
    for (int slot = 0; slot < 27; ++slot) {
        int dr, dz;
        s2l_offset(pr, pz, slot, &dr, &dz);
        int scol = col + dr;
        if (scol < 0 || scol >= nl) continue;
        __syncthreads();
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        if (threadIdx.x < 32) {
            int b = bx[threadIdx.x];
            int s = b >= 0 ? a.s2l[(size_t)b * 27 + slot] : -1;
            src[threadIdx.x] = s;
            if (s >= 0) any = 1;
        }
        __syncthreads();
        if (!any) continue;
        int station = dr < 0 ? scol : col;  // the smaller radius
        int sidx = a.station_of_col[station];
        int ea = dr < 0 ? -dr : dr, eb = dz < 0 ? -dz : dz;
        bool inward = dr > 0, backward = dz > 0;
        const double *E = a.gexp + (((size_t)sidx * 16 + ea * 4 + eb) * a.nm + n) * slabn;
        for (int i = threadIdx.x; i < slab; i += blockDim.x) {
            int c = i % C2, ki = i / C2;
            int k = ki / W, ii = ki % W;
            if (k + ii + c > 2 * M) continue;
            R v = (R)(inward ? E[((size_t)ii * W + k) * C2 + c] : E[i]);
            S[i] = (backward && (c & 1)) ? -v : v;
        }
        for (int i = threadIdx.x; i < nc * 32; i += blockDim.x) {
            int c = i / 32, m = i % 32;
            int s = src[m];
            Ir[i] = s >= 0 ? a.mom_re[((size_t)s * a.nm + n) * nc + c] : (R)0;
            Ii[i] = s >= 0 ? a.mom_im[((size_t)s * a.nm + n) * nc + c] : (R)0;
        }
        __syncthreads();
        int ij = 0;
        for (int i = 0; i <= M; ++i) {
            for (int j = 0; i + j <= M; ++j, ++ij) {
                R xr = Ir[ij * 32 + lane], xi = Ii[ij * 32 + lane];
                int off = i * C2 + j;
#pragma unroll
                for (int q = 0; q < KPT; ++q) {
                    R e = S[base[q] + off];
                    accr[q] = fma(e, xr, accr[q]);
                    acci[q] = fma(e, xi, acci[q]);
                }
            }
        }
    }
    int b = bx[lane];
    if (b < 0) return;
    // F_kl += acc / l!
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        int kl = grp + 4 * q;
        if (kl < nc) {
            int k = 0, rem = kl;
            while (rem >= M + 1 - k) { rem -= M + 1 - k; ++k; }
            double f = 1.0;
            for (int t = 2; t <= rem; ++t) f *= t;
            R invf = (R)(1.0 / f);
            size_t o = ((size_t)b * a.nm + n) * nc + kl;
            a.loc_re[o] += accr[q] * invf;
            a.loc_im[o] += acci[q] * invf;
        }
    }
}

// ------------------------------------------------------------------------------------
// S2L in FP32-pair ("double-float") arithmetic for the FP64 path.  On GB300 an FP32 FMA
// issues 61x faster than an FP64 FMA, so each FP64 operand is held as hi + lo floats and
// each complex multiply-add is an exact FP32 two-product (hi*hi by FMA, plus the cross
// terms) folded into a (sum, error) pair by an exact two-sum: ~24 FP32 operations in
// place of two FP64 FMAs, relative accuracy ~1e-14.  Round-to-nearest intrinsics keep
// the compiler from contracting the error-free transformations.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float2 split_df(double v)
{
    float h = __double2float_rn(v);
    float l = __double2float_rn(v - (double)h);
    return make_float2(h, l);
}

// acc (S, E) += a * b, a = (ah, al), b = (bh, bl)
__device__ __forceinline__ void df_fma_acc(float &S, float &E, float2 a, float2 b)
{
    float p = __fmul_rn(a.x, b.x);
    float pe = __fmaf_rn(a.x, b.x, -p);
    pe = __fmaf_rn(a.x, b.y, pe);
    pe = __fmaf_rn(a.y, b.x, pe);
    float s = __fadd_rn(S, p);
    float v = __fsub_rn(s, S);
    float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, v)), __fsub_rn(p, v));
    E = __fadd_rn(E, __fadd_rn(err, pe));
    S = s;
}

// hi/lo split of an FP64 array into FP32 pairs (once per level, ahead of the S2L)
__global__ void k_split_df(const double *__restrict__ in, int64_t n, float2 *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = split_df(in[i]);
}

template <int KPT>
__global__ void __launch_bounds__(128) k_s2l_df(const S2LArgs<double> a)
{
    extern __shared__ double sm_raw[];
    float2 *sm = reinterpret_cast<float2 *>(sm_raw);
    const int M = a.M, nc = a.nc, W = M + 1, C2 = 2 * M + 1;
    const int slab = W * W * C2;
    float2 *S = sm;                 // [W][W][C2] oriented expansion, hi/lo
    float2 *Ir = S + slab;          // [nc][32]
    float2 *Ii = Ir + (size_t)nc * 32;
    __shared__ int bx[32];
    __shared__ int src[32];
    __shared__ int any;
    const int64_t u = blockIdx.x;
    const int n = blockIdx.y;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    if (threadIdx.x < 32) bx[threadIdx.x] = a.unit_box[u * 32 + threadIdx.x];
    const int ucol = a.unit_col[u];
    const int col = ucol & 0xffff, pz = (ucol >> 30) & 1, pr = col & 1;
    const int nl = 1 << a.level;
    float aSr[KPT], aEr[KPT], aSi[KPT], aEi[KPT];
    int base[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        aSr[q] = aEr[q] = aSi[q] = aEi[q] = 0.f;
        int kl = grp + 4 * q;
        int k = 0, rem = kl < nc ? kl : 0;
        while (rem >= M + 1 - k) { rem -= M + 1 - k; ++k; }
        base[q] = (k * W) * C2 + rem;
    }
    const size_t slabn = (size_t)slab;
    for (int slot = 0; slot < 27; ++slot) {
        int dr, dz;
        s2l_offset(pr, pz, slot, &dr, &dz);
        int scol = col + dr;
        if (scol < 0 || scol >= nl) continue;
        __syncthreads();
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        if (threadIdx.x < 32) {
            int b = bx[threadIdx.x];
            int s2 = b >= 0 ? a.s2l[(size_t)b * 27 + slot] : -1;
            src[threadIdx.x] = s2;
            if (s2 >= 0) any = 1;
        }
        __syncthreads();
        if (!any) continue;
        int station = dr < 0 ? scol : col;
        int sidx = a.station_of_col[station];
        int ea = dr < 0 ? -dr : dr, eb = dz < 0 ? -dz : dz;
        bool inward = dr > 0, backward = dz > 0;
        const float2 *E = a.gexp_df + (((size_t)sidx * 16 + ea * 4 + eb) * a.nm + n) * slabn;
        for (int i = threadIdx.x; i < slab; i += blockDim.x) {
            int c = i % C2, ki = i / C2;
            int k = ki / W, ii = ki % W;
            if (k + ii + c > 2 * M) continue;
            float2 v = inward ? E[((size_t)ii * W + k) * C2 + c] : E[i];
            S[i] = (backward && (c & 1)) ? make_float2(-v.x, -v.y) : v;
        }
        for (int i = threadIdx.x; i < nc * 32; i += blockDim.x) {
            int c = i / 32, m = i % 32;
            int s2 = src[m];
            Ir[i] = s2 >= 0 ? a.mom_df_re[((size_t)s2 * a.nm + n) * nc + c] : make_float2(0.f, 0.f);
            Ii[i] = s2 >= 0 ? a.mom_df_im[((size_t)s2 * a.nm + n) * nc + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        int ij = 0;
        for (int i = 0; i <= M; ++i) {
            for (int j = 0; i + j <= M; ++j, ++ij) {
                float2 xr = Ir[ij * 32 + lane], xi = Ii[ij * 32 + lane];
                int off = i * C2 + j;
#pragma unroll
                for (int q = 0; q < KPT; ++q) {
                    float2 e = S[base[q] + off];
                    df_fma_acc(aSr[q], aEr[q], e, xr);
                    df_fma_acc(aSi[q], aEi[q], e, xi);
                }
            }
        }
    }
    int b = bx[lane];
    if (b < 0) return;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        int kl = grp + 4 * q;
        if (kl < nc) {
            int k = 0, rem = kl;
            while (rem >= M + 1 - k) { rem -= M + 1 - k; ++k; }
            double f = 1.0;
            for (int t = 2; t <= rem; ++t) f *= t;
            const dfv rf = df_from_double(1.0 / f);
            size_t o = ((size_t)b * a.nm + n) * nc + kl;
            const dfv vr = df_add(df_make(a.locd_re[o].x, a.locd_re[o].y), df_mul(two_sum(aSr[q], aEr[q]), rf));
            const dfv vi = df_add(df_make(a.locd_im[o].x, a.locd_im[o].y), df_mul(two_sum(aSi[q], aEi[q]), rf));
            a.locd_re[o] = make_float2(vr.hi, vr.lo);
            a.locd_im[o] = make_float2(vi.hi, vi.lo);
        }
    }
}

static inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b > 0 ? (n + b - 1) / b : 1); }

template <int KPT>
static afmm_status launch_s2l_df_k(const S2LArgs<double> &a, cudaStream_t st, size_t sm)
{
    AFMM_CUDA(cudaFuncSetAttribute(k_s2l_df<KPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)a.nunit, (unsigned)a.nm);
    k_s2l_df<KPT><<<grid, 128, sm, st>>>(a);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

template <typename R, int KPT>
static afmm_status launch_s2l_k(const S2LArgs<R> &a, cudaStream_t st, size_t sm)
{
    AFMM_CUDA(cudaFuncSetAttribute(k_s2l<R, KPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dim3 grid((unsigned)a.nunit, (unsigned)a.nm);
    k_s2l<R, KPT><<<grid, 128, sm, st>>>(a);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

template <typename R>
static afmm_status launch_s2l(afmm_plan p, int l, const R *mre, const R *mim, R *lre, R *lim)
{
    Level &v = p->lv[l];
    if (v.nunit == 0) return AFMM_OK;
    S2LArgs<R> a;
    a.unit_box = v.unit_box;
    a.unit_col = v.unit_col;
    a.s2l = v.s2l;
    a.station_of_col = v.station_of_col;
    a.nunit = v.nunit;
    a.level = l;
    a.nm = p->nmodes;
    a.M = p->M;
    a.nc = p->ncoef;
    a.gexp = p->gexp;
    a.mom_re = mre;
    a.mom_im = mim;
    a.loc_re = lre;
    a.loc_im = lim;
    a.gexp_df = nullptr;
    a.mom_df_re = a.mom_df_im = nullptr;
    a.locd_re = a.locd_im = nullptr;
    int W = p->M + 1;
    size_t sm = sizeof(R) * ((size_t)W * W * (2 * p->M + 1) + 2 * (size_t)p->ncoef * 32);
    int kpt = (p->ncoef + 3) / 4;
    if (s2l_tc_enabled(p)) return launch_s2l_tc(p, l, mre, mim, lre, lim);
    if (kpt <= 4) return launch_s2l_k<R, 4>(a, p->stream, sm);
    if (kpt <= 8) return launch_s2l_k<R, 8>(a, p->stream, sm);
    if (kpt <= 12) return launch_s2l_k<R, 12>(a, p->stream, sm);
    if (kpt <= 16) return launch_s2l_k<R, 16>(a, p->stream, sm);
    if (kpt <= 24) return launch_s2l_k<R, 24>(a, p->stream, sm);
    if (kpt <= 32) return launch_s2l_k<R, 32>(a, p->stream, sm);
    if (kpt <= 40) return launch_s2l_k<R, 40>(a, p->stream, sm);
    return AFMM_EUNSUPPORTED;
}

static void tmark(afmm_plan p, int idx)
{
    if (p->timing && idx < 80) cudaEventRecord(p->ev[idx], p->stream);
}

// Far field for direction dir (0: sources -> field points, 1: transposed), in the real
// type R of the plan's precision.  Uses the strengths already permuted into p->qs_*;
// leaves the leaf-level locals in lv[d].loc_* (or loc32_* for the mixed precision).
template <typename R>
static afmm_status far_field_t(afmm_plan p, int dir)
{
    const bool mix = sizeof(R) == sizeof(float);
    const int d = p->d, M = p->M, nm = p->nmodes, nc = p->ncoef;
    cudaStream_t st = p->stream;
    const bool fw = dir == 0;
    const double *sr = fw ? p->s_r : p->t_r, *sz = fw ? p->s_z : p->t_z;
    int64_t nsrc = fw ? p->ns : p->nf;
    auto MR = [&](int l) { return mix ? (R *)p->lv[l].mom32_re : (R *)p->lv[l].mom_re; };
    auto MI = [&](int l) { return mix ? (R *)p->lv[l].mom32_im : (R *)p->lv[l].mom_im; };
    auto LR = [&](int l) { return mix ? (R *)p->lv[l].loc32_re : (R *)p->lv[l].loc_re; };
    auto LI = [&](int l) { return mix ? (R *)p->lv[l].loc32_im : (R *)p->lv[l].loc_im; };
    const R *q_re = mix ? (const R *)p->qs32 : (const R *)p->qs_re;
    const R *q_im = mix ? (const R *)p->qs32 + 2 : (const R *)p->qs_im;
    // P2M at the leaves (adaptive tree: the leaves of every level, deepest first, each level
    // before its M2M, which keeps the leaves' moments), then the upward pass
    const size_t psm = sizeof(R) * (32 * (size_t)nc + 2 * (size_t)nm * nc + M + 1);
    if (psm > 227 * 1024) return AFMM_EUNSUPPORTED;
    AFMM_CUDA(cudaFuncSetAttribute(k_p2m<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
    auto p2m = [&](int l, const int2 *rng) -> afmm_status {
        Level &v = p->lv[l];
        const double h = p->L / (double)(1 << l);
        k_p2m<R><<<(unsigned)v.nbox, 128, psm, st>>>(v.key, rng, v.nbox, sr, sz, q_re, q_im, nsrc, nm, M, p->r0, p->z0,
                                                     h, *p->rec, MR(l), MI(l));
        AFMM_LAUNCH_CHECK();
        return AFMM_OK;
    };
    if (!p->adaptive) AFMM_TRY(p2m(d, fw ? p->lv[d].srng : p->lv[d].trng));
    tmark(p, 2);
    for (int l = p->adaptive ? d : d - 1; l >= 2; --l) {
        Level &v = p->lv[l];
        if (p->adaptive) AFMM_TRY(p2m(l, fw ? v.srng_leaf : v.trng_leaf));
        if (l == d) continue;
        size_t sm = sizeof(R) * (2 * (size_t)nc + 4 * (size_t)(M + 1) * (M + 1));
        k_m2m<R><<<dim3((unsigned)v.nbox, (unsigned)nm), 128, sm, st>>>(v.child, p->lv[l + 1].key, v.nbox, nm, M, p->m2m_tab, MR(l + 1),
                                                    MI(l + 1), MR(l), MI(l));
        AFMM_LAUNCH_CHECK();
    }
    tmark(p, 3);
    // downward pass
    size_t gsm = gbar_smem(p->N, 2 * M, gexp_dd(p));
    if (gsm > 227 * 1024) return AFMM_EUNSUPPORTED;
    AFMM_CUDA(cudaFuncSetAttribute(k_gexp_level<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    AFMM_CUDA(cudaFuncSetAttribute(k_gexp_level<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    for (int l = 2; l <= d; ++l) {
        Level &v = p->lv[l];
        const int e = 16 + 4 * (l - 2);  // event slots: L2L, expansions, S2L, end
        size_t sm = sizeof(R) * (2 * (size_t)nc + 4 * (size_t)(M + 1) * (M + 1));
        tmark(p, e);
        k_l2l<R><<<dim3((unsigned)v.nbox, (unsigned)nm), 128, sm, st>>>(l >= 3 ? v.parent : nullptr, v.key, v.nbox, nm, M, p->l2l_tab,
                                                    l >= 3 ? LR(l - 1) : nullptr, l >= 3 ? LI(l - 1) : nullptr, LR(l),
                                                    LI(l));
        AFMM_LAUNCH_CHECK();
        tmark(p, e + 1);
        double h = p->L / (double)(1 << l);
        if (v.nstation > 0) {
            // the tensor-core S2L takes its expansions directly as FP32 pairs
            const bool dfx = s2l_tc_enabled(p);
            AFMM_TRY(launch_gexp_level(p, l, gsm, dfx ? nullptr : p->gexp, dfx ? p->gexp_df : nullptr));
        }
        tmark(p, e + 2);
        AFMM_TRY(launch_s2l<R>(p, l, MR(l), MI(l), LR(l), LI(l)));
        tmark(p, e + 3);
    }
    return AFMM_OK;
}

// Far field of the FP64 path: moments, locals and expansions as FP32 pairs throughout (the
// same steps as far_field_t); the leaf locals stay in lv[d].locd_* for the near kernel
static afmm_status far_field_df(afmm_plan p, int dir)
{
    const int d = p->d, M = p->M, nm = p->nmodes, nc = p->ncoef, W = M + 1;
    cudaStream_t st = p->stream;
    const bool fw = dir == 0;
    const double *sr = fw ? p->s_r : p->t_r, *sz = fw ? p->s_z : p->t_z;
    const int64_t nsrc = fw ? p->ns : p->nf;
    const float4 *qri = p->qsdf;
    // chunks of 32 sources, or 16 where the staging of 32 does not fit
    auto smem = [&](int ch) {
        return sizeof(float4) * (size_t)ch * nm + sizeof(float2) * ((size_t)ch * nc + 2 * (size_t)nm * nc + M + 1 + nm);
    };
    const int CH = smem(32) <= 227 * 1024 ? 32 : 16;
    const size_t psm = smem(CH);
    if (psm > 227 * 1024) return AFMM_EUNSUPPORTED;
    AFMM_CUDA(cudaFuncSetAttribute(k_p2m_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
    auto p2m = [&](int l, const int2 *rng) -> afmm_status {
        Level &v = p->lv[l];
        const double h = p->L / (double)(1 << l);
        k_p2m_df<<<(unsigned)v.nbox, 128, psm, st>>>(v.key, rng, v.nbox, sr, sz, qri, nsrc, nm, M, p->r0, p->z0, h,
                                                    *p->rec, v.momd_re, v.momd_im, CH);
        AFMM_LAUNCH_CHECK();
        return AFMM_OK;
    };
    // P2M at the leaves (adaptive tree: every level's leaves, each level before its M2M)
    if (!p->adaptive) AFMM_TRY(p2m(d, fw ? p->lv[d].srng : p->lv[d].trng));
    tmark(p, 2);
    const size_t ssm = sizeof(float2) * (2 * (size_t)nc + 4 * (size_t)W * W);
    for (int l = p->adaptive ? d : d - 1; l >= 2; --l) {
        Level &v = p->lv[l];
        if (p->adaptive) AFMM_TRY(p2m(l, fw ? v.srng_leaf : v.trng_leaf));
        if (l == d) continue;
        k_m2m_df<<<dim3((unsigned)v.nbox, (unsigned)((nm + SHIFT_MB - 1) / SHIFT_MB)), 128, ssm, st>>>(v.child, p->lv[l + 1].key, v.nbox, nm, M,
                                                                         p->m2m_tab_df, p->lv[l + 1].momd_re,
                                                                         p->lv[l + 1].momd_im, v.momd_re, v.momd_im);
        AFMM_LAUNCH_CHECK();
    }
    tmark(p, 3);
    const size_t gsm = gbar_smem(p->N, 2 * M, gexp_dd(p));
    if (gsm > 227 * 1024) return AFMM_EUNSUPPORTED;
    AFMM_CUDA(cudaFuncSetAttribute(k_gexp_level<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    AFMM_CUDA(cudaFuncSetAttribute(k_gexp_level<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    for (int l = 2; l <= d; ++l) {
        Level &v = p->lv[l];
        const int e = 16 + 4 * (l - 2);  // event slots: L2L, expansions, S2L, end
        tmark(p, e);
        k_l2l_df<<<dim3((unsigned)v.nbox, (unsigned)((nm + SHIFT_MB - 1) / SHIFT_MB)), 128, ssm, st>>>(
            l >= 3 ? v.parent : nullptr, v.key, v.nbox, nm, M, p->l2l_tab_df, l >= 3 ? p->lv[l - 1].locd_re : nullptr,
            l >= 3 ? p->lv[l - 1].locd_im : nullptr, v.locd_re, v.locd_im);
        AFMM_LAUNCH_CHECK();
        tmark(p, e + 1);
        if (v.nstation > 0) AFMM_TRY(launch_gexp_level(p, l, gsm, nullptr, p->gexp_df));
        tmark(p, e + 2);
        if (s2l_tc_enabled(p)) {
            AFMM_TRY(launch_s2l_tc(p, l, v.momd_re, v.momd_im, v.locd_re, v.locd_im));
        } else if (v.nunit > 0) {
            S2LArgs<double> a = {};
            a.unit_box = v.unit_box;
            a.unit_col = v.unit_col;
            a.s2l = v.s2l;
            a.station_of_col = v.station_of_col;
            a.nunit = v.nunit;
            a.level = l;
            a.nm = nm;
            a.M = M;
            a.nc = nc;
            a.gexp_df = p->gexp_df;
            a.mom_df_re = v.momd_re;
            a.mom_df_im = v.momd_im;
            a.locd_re = v.locd_re;
            a.locd_im = v.locd_im;
            const size_t sm = sizeof(float2) * ((size_t)W * W * (2 * M + 1) + 2 * (size_t)nc * 32);
            const int kpt = (nc + 3) / 4;
            afmm_status r = AFMM_EUNSUPPORTED;
            if (kpt <= 4) r = launch_s2l_df_k<4>(a, st, sm);
            else if (kpt <= 8) r = launch_s2l_df_k<8>(a, st, sm);
            else if (kpt <= 12) r = launch_s2l_df_k<12>(a, st, sm);
            else if (kpt <= 16) r = launch_s2l_df_k<16>(a, st, sm);
            else if (kpt <= 24) r = launch_s2l_df_k<24>(a, st, sm);
            else if (kpt <= 32) r = launch_s2l_df_k<32>(a, st, sm);
            else if (kpt <= 40) r = launch_s2l_df_k<40>(a, st, sm);
            AFMM_TRY(r);
        }
        tmark(p, e + 3);
    }
    return AFMM_OK;
}

afmm_status far_field(afmm_plan p, int dir)
{
    if (p->precision == AFMM_MIXED) return far_field_t<float>(p, dir);
    if (p->precision == AFMM_FP64) return far_field_df(p, dir);
    return far_field_t<double>(p, dir);  // AFMM_FP64_NATIVE
}

}  // namespace afmm
