// peaks.cu -- arithmetic-pipe peak probes for the benchmark's roofline (libafmm_peaks.so).
//
// Not part of the method: bench.py measures the FP32 and FP64 FMA throughput of the GPU it
// runs on with these kernels, so that the near-field and local-expansion kernels (FP32
// pipe) and the method's FP64 work can be quoted against measured peaks.
//
// Each thread runs CHAINS independent FMA chains x = x * a + b for `iters` iterations, with
// a and b chosen so that the values stay finite; the result is written so the work cannot
// be removed.  Operations per launch: blocks * threads * iters * CHAINS (x2 for the packed
// f32x2 form, one FMA counted as one operation).
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/afmm_peaks.h"

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_peak_ffma(float *__restrict__ sink, int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_ffma2(float *__restrict__ sink, int iters, float a, float b)
{
    float2 x[CHAINS];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k].x + x[k].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(float *__restrict__ sink, int iters, float a, float b)
{
    double x[CHAINS];
    const double ad = a, bd = b;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = __fma_rn(x[k], ad, bd);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace

extern "C" {

// Launch one probe: kind 0 = FP32 FMA, 1 = packed f32x2 FMA, 2 = FP64 FMA, with `blocks`
// blocks of 256 threads, on `stream`.  `sink` is a device buffer of at least blocks * 256
// floats.  *ops receives the FMA operations the launch performs.  Returns 0, or -1 for
// bad arguments, or the CUDA error code of the launch.
int afmm_peak_launch(int kind, int blocks, int iters, float *sink, double *ops, void *stream)
{
    if (blocks < 1 || iters < 1 || !sink || !ops || kind < 0 || kind > 2) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    const float a = 0.999999f, b = 1e-6f;
    if (kind == 0)
        k_peak_ffma<<<blocks, 256, 0, st>>>(sink, iters, a, b);
    else if (kind == 1)
        k_peak_ffma2<<<blocks, 256, 0, st>>>(sink, iters, a, b);
    else
        k_peak_dfma<<<blocks, 256, 0, st>>>(sink, iters, a, b);
    *ops = (double)blocks * 256.0 * (double)iters * CHAINS * (kind == 1 ? 2.0 : 1.0);
    return (int)cudaGetLastError();
}

}  // extern "C"
