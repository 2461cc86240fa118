/*
 * df_probe.h - measurement helpers shipped with the chemistry library.
 *
 * The paper has no counterpart: these calls only measure the GPU the library
 * runs on, so that throughput can be stated as a fraction of a measured peak.
 */
#ifndef DF_PROBE_H
#define DF_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif

/* Measured FP64 fused multiply-add throughput of the current device.
 * Runs a grid of 8 independent DFMA chains per thread (`iters` FMAs each) on
 * every SM, timed with CUDA events on a private stream; synchronous.
 * gflops: 2 * FMAs / time in GFLOP/s (host); ms: kernel time (host, may be NULL).
 * Returns 0 or a negative DF_E* code (DF_EINVAL for iters < 1). */
int df_probe_fp64_peak(int iters, double* gflops, double* ms);

/* y[i] = exp(x[i]) for i < n by the library's own table-driven exponential
 * (the one the rate kernels use), so that its accuracy can be checked against
 * CUDA's exp.  x, y: device memory; asynchronous on `stream` (a cudaStream_t). */
int df_probe_exp(const double* x, double* y, long long n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DF_PROBE_H */
