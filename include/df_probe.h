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

/* FP64 dependent-issue latency against throughput: one block of
 * warps_per_sm warps on every SM, each thread running `chains` independent
 * chains of `iters` dependent DFMAs (chains in {1, 2, 4, 8}, warps_per_sm in
 * [1, 32], iters >= 1), timed with CUDA events on a private stream after one
 * warm-up run; synchronous.
 * ns_per_step: kernel time / iters, i.e. the time of one dependent step of a
 * chain (host); gflops: 2 * FMAs / time (host, may be NULL).
 * Returns 0 or a negative DF_E* code (DF_EINVAL for arguments out of range). */
int df_probe_fp64_chains(int warps_per_sm, int chains, int iters, double* ns_per_step, double* gflops);

/* y[i] = exp(x[i]) for i < n by the library's own table-driven exponential
 * (the one the rate kernels use), so that its accuracy can be checked against
 * CUDA's exp.  table_bits: 6 (the 64-entry table of the library's kernels) or
 * 8 (the 256-entry table of the kernels generated for a loaded mechanism).
 * x, y: device memory; asynchronous on `stream` (a cudaStream_t).  Returns 0,
 * or DF_EINVAL for a negative n, a missing buffer or other table_bits. */
int df_probe_exp(const double* x, double* y, long long n, int table_bits, void* stream);

/* y[i] = ln(x[i]) by the library's own table-driven logarithm (the one the
 * rate kernels use for ln T and the Troe falloff), so that its accuracy can be
 * checked against CUDA's log.  x, y: device memory; asynchronous on `stream`.
 * DF_EINVAL for n < 0 or null arrays with n > 0. */
int df_probe_log(const double* x, double* y, long long n, void* stream);

/* y[i] = GELU(x[i]) (derivative = 0) or GELU'(x[i]) (derivative = 1) as the GEMM
 * epilogues compute them in FP32 (the network's activation, Sec. 2.3: GELU(z) =
 * z Phi(z) with Phi the normal CDF, through the library's own erfc), so that their
 * accuracy can be checked against the exact function.  x, y: device memory;
 * asynchronous on `stream`.  DF_EINVAL for n < 0 or null arrays with n > 0. */
int df_probe_gelu(const float* x, float* y, long long n, int derivative, void* stream);

/* C = A . B^T with the library's tcgen05 BF16 GEMM (the kernel under the DNN
 * integrator's layers), FP32 result without bias or activation, so that it can be
 * checked against a reference matmul.  A [M][K], B [N][K] bf16 (device, 16-byte
 * aligned, K a multiple of 8), C [M][N] f32 (device), N a multiple of 8; bn: output
 * tile width 64, 128 or 256 of the one-tile-per-CTA kernel, or -128, -160, -208,
 * -256 for the persistent kernel with a double-buffered accumulator (0 = choose).  err_flag (device int, may be NULL) is
 * set to 1 if a bounded pipeline wait ran out.  Asynchronous on `stream`. */
int df_probe_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, int bn, int* err_flag,
                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DF_PROBE_H */
