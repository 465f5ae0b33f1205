// fourier.cu -- azimuthal Fourier analysis and synthesis of ring quantities (Sec. 2):
//   s(theta) = sum_{n=-N..N} S^(n) e^{i n theta}, S^(-n) = conj(S^(n))   (Eq. analysis:source)
//   phi(theta) = sum_n Phi^(n) e^{i n theta}                              (Eq. analysis:phi)
// Analysis from K equispaced samples theta_k = 2 pi k / K (exact for K >= 2N + 1):
//   S^(n) = (1/K) sum_k s(theta_k) e^{-i n theta_k};
// synthesis at the same angles: phi(theta_k) = Re Phi^(0) + 2 sum_{n>=1} Re(Phi^(n) e^{i n theta_k}).
// One thread per ring (point); the twiddles cos, sin(2 pi m / K) sit in shared memory as FP32
// pairs, the index m = n k mod K advances by n per step, and the sums are FP32-pair
// accumulations (FP64 in and out).
#include "common.cuh"
#include "df.cuh"

namespace afmm {

namespace {

constexpr int FT_THREADS = 128;
constexpr int FT_MAX_K = 4096;  // twiddle table: 16 B per angle in shared memory

__device__ void make_twiddles(int K, float4 *tw)
{
    for (int m = threadIdx.x; m < K; m += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)K, &sn, &cs);
        const dfv c = df_from_double(cs), s = df_from_double(sn);
        tw[m] = make_float4(c.hi, c.lo, s.hi, s.lo);
    }
    __syncthreads();
}

constexpr int FT_CHUNK = 8;  // modes (analysis) or angles (synthesis) per register block

// Each sample is split into an FP32 pair once per block of 8 modes (the split uses the FP64
// pipe); index m = n k mod K per (mode, angle).
__global__ void __launch_bounds__(FT_THREADS) k_fourier_analysis(int64_t npts, int K, const double *__restrict__ smp,
                                                                 int nm, double *__restrict__ S_re,
                                                                 double *__restrict__ S_im)
{
    extern __shared__ float4 tw[];
    make_twiddles(K, tw);
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const double iK = 1.0 / (double)K;
    for (int n0 = 0; n0 < nm; n0 += FT_CHUNK) {
        float ar[FT_CHUNK], er[FT_CHUNK], ai[FT_CHUNK], ei[FT_CHUNK];
        int m[FT_CHUNK], dn[FT_CHUNK];
#pragma unroll
        for (int j = 0; j < FT_CHUNK; ++j) {
            ar[j] = er[j] = ai[j] = ei[j] = 0.f;
            m[j] = 0;
            dn[j] = (n0 + j) % K;
        }
        for (int k = 0; k < K; ++k) {
            const dfv v = df_from_double(smp[(size_t)k * npts + p]);
#pragma unroll
            for (int j = 0; j < FT_CHUNK; ++j) {
                const float4 t = tw[m[j]];
                df_acc(ar[j], er[j], v, df_make(t.x, t.y));
                df_acc(ai[j], ei[j], v, df_make(-t.z, -t.w));
                m[j] += dn[j];
                if (m[j] >= K) m[j] -= K;
            }
        }
#pragma unroll
        for (int j = 0; j < FT_CHUNK; ++j)
            if (n0 + j < nm) {
                S_re[(size_t)(n0 + j) * npts + p] = ((double)ar[j] + (double)er[j]) * iK;
                S_im[(size_t)(n0 + j) * npts + p] = ((double)ai[j] + (double)ei[j]) * iK;
            }
    }
}

// Each coefficient is split once per block of 8 angles.
__global__ void __launch_bounds__(FT_THREADS) k_fourier_synthesis(int64_t npts, int nm, const double *__restrict__ P_re,
                                                                  const double *__restrict__ P_im, int K,
                                                                  double *__restrict__ phi)
{
    extern __shared__ float4 tw[];
    make_twiddles(K, tw);
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const dfv a0 = df_from_double(P_re[p]);
    for (int k0 = 0; k0 < K; k0 += FT_CHUNK) {
        float S[FT_CHUNK], E[FT_CHUNK];
        int m[FT_CHUNK], dk[FT_CHUNK];
#pragma unroll
        for (int j = 0; j < FT_CHUNK; ++j) {
            S[j] = a0.hi;
            E[j] = a0.lo;
            dk[j] = (k0 + j) % K;
            m[j] = dk[j];
        }
        for (int n = 1; n < nm; ++n) {
            // 2 (Re P cos - Im P sin): the factor 2 is exact
            const dfv pr = df_scale2(df_from_double(P_re[(size_t)n * npts + p]), 2.f);
            const dfv pi = df_scale2(df_from_double(P_im[(size_t)n * npts + p]), -2.f);
#pragma unroll
            for (int j = 0; j < FT_CHUNK; ++j) {
                const float4 t = tw[m[j]];
                df_acc(S[j], E[j], pr, df_make(t.x, t.y));
                df_acc(S[j], E[j], pi, df_make(t.z, t.w));
                m[j] += dk[j];
                if (m[j] >= K) m[j] -= K;
            }
        }
#pragma unroll
        for (int j = 0; j < FT_CHUNK; ++j)
            if (k0 + j < K) phi[(size_t)(k0 + j) * npts + p] = (double)S[j] + (double)E[j];
    }
}

}  // namespace

}  // namespace afmm

using namespace afmm;

extern "C" {

afmm_status afmm_fourier_analysis(int64_t npts, int K, const double *samples, int n_modes, double *S_re,
                                  double *S_im, void *stream)
{
    if (npts < 0 || K < 1 || K > FT_MAX_K || n_modes < 1 || !samples || !S_re || !S_im) return AFMM_EINVAL;
    if (npts == 0) return AFMM_OK;
    const unsigned grid = (unsigned)((npts + FT_THREADS - 1) / FT_THREADS);
    AFMM_CUDA(cudaFuncSetAttribute(k_fourier_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, K * (int)sizeof(float4)));
    k_fourier_analysis<<<grid, FT_THREADS, (size_t)K * sizeof(float4), (cudaStream_t)stream>>>(npts, K, samples,
                                                                                                n_modes, S_re, S_im);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

afmm_status afmm_fourier_synthesis(int64_t npts, int n_modes, const double *phi_re, const double *phi_im, int K,
                                   double *phi, void *stream)
{
    if (npts < 0 || K < 1 || K > FT_MAX_K || n_modes < 1 || !phi_re || !phi_im || !phi) return AFMM_EINVAL;
    if (npts == 0) return AFMM_OK;
    const unsigned grid = (unsigned)((npts + FT_THREADS - 1) / FT_THREADS);
    AFMM_CUDA(cudaFuncSetAttribute(k_fourier_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, K * (int)sizeof(float4)));
    k_fourier_synthesis<<<grid, FT_THREADS, (size_t)K * sizeof(float4), (cudaStream_t)stream>>>(npts, n_modes, phi_re,
                                                                                                 phi_im, K, phi);
    AFMM_LAUNCH_CHECK();
    return AFMM_OK;
}

}  // extern "C"
