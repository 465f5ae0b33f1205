/*
 * afmm_peaks.h -- C ABI of libafmm_peaks, the arithmetic-pipe probes the benchmark uses to
 * measure the FMA throughput of the GPU it runs on (the denominators of its FP32 and FP64
 * rooflines).  Not part of the method; the paper has no counterpart.
 */
#ifndef AFMM_PEAKS_H
#define AFMM_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Launch one probe kernel on `stream` (cudaStream_t, NULL = legacy default stream):
 * kind 0 = FP32 FMA, 1 = packed f32x2 FMA, 2 = FP64 FMA; `blocks` blocks of 256 threads,
 * each thread running 8 independent FMA chains for `iters` iterations.  `sink` is a
 * device buffer of at least blocks * 256 floats (caller-owned; receives one value per
 * thread so that the work is kept).  *ops (host) receives the FMA operations of the launch
 * (one FMA = one operation; a packed FMA = two).  Asynchronous: time it with events on the
 * same stream.  Returns 0, -1 for bad arguments (nothing launched), or the CUDA error code
 * of the launch. */
int afmm_peak_launch(int kind, int blocks, int iters, float *sink, double *ops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AFMM_PEAKS_H */
