// FP64 throughput probe: eight independent fused multiply-add chains per
// thread on a grid that fills every SM.  The measured rate is the denominator
// of the integrator's FP64 roofline fraction.
#include "common.cuh"
#include "../../include/df_probe.h"
#include "fastexp.cuh"
#include "fastlog.cuh"

namespace df {

__global__ void __launch_bounds__(256) k_dfma_chains(double* out, int iters, double a, double b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x0 = 1.0 + tid * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
  double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[tid] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <int NC>
__global__ void k_fma_chains(double* out, int iters, double a, double b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) x[c] = 1.0 + tid * 1e-9 + c * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NC; ++c) s += x[c];
  out[tid] = s;
}

template <int B>
__global__ void k_exp_probe(const double* x, double* y, long long n) {
  __shared__ double2 tab[1 << B];
  const double2* src = B == 8 ? g_exp2_tab256 : g_exp2_tab;
  for (int i = threadIdx.x; i < (1 << B); i += blockDim.x) tab[i] = src[i];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_tang_b<B>(x[i], tab);
}

__global__ void k_log_probe(const double* x, double* y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = log_tab(x[i]);
}

}  // namespace df

using namespace df;

extern "C" int df_probe_log(const double* x, double* y, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(DF_EINVAL, "df_probe_log: bad arguments");
  if (n == 0) return DF_OK;
  k_log_probe<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cuda_check(cudaGetLastError(), "log probe kernel");
}

extern "C" int df_probe_exp(const double* x, double* y, long long n, int table_bits, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y)) || (table_bits != 6 && table_bits != 8))
    return set_error(DF_EINVAL, "df_probe_exp: bad arguments");
  if (n == 0) return DF_OK;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (table_bits == 8) k_exp_probe<8><<<blocks, threads, 0, (cudaStream_t)stream>>>(x, y, n);
  else k_exp_probe<6><<<blocks, threads, 0, (cudaStream_t)stream>>>(x, y, n);
  return cuda_check(cudaGetLastError(), "exp probe kernel");
}

extern "C" int df_probe_fp64_peak(int iters, double* gflops, double* ms) {
  if (iters < 1 || !gflops) return set_error(DF_EINVAL, "df_probe_fp64_peak: iters >= 1 and gflops required");
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  cudaDeviceProp prop;
  if ((rc = cuda_check(cudaGetDeviceProperties(&prop, dev), "properties"))) return rc;
  const int threads = 256;
  const int blocks = prop.multiProcessorCount * 8;
  double* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rc = cuda_check(cudaMalloc(&out, sizeof(double) * threads * blocks), "cudaMalloc");
  if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
  if (!rc) rc = cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = cuda_check(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  for (int rep = 0; rep < 4 && !rc; ++rep) {
    cudaEventRecord(e0, st);
    k_dfma_chains<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    rc = cuda_check(cudaEventSynchronize(e1), "probe kernel");
    float t = 0.f;
    if (!rc) rc = cuda_check(cudaEventElapsedTime(&t, e0, e1), "elapsed");
    if (!rc && rep > 0 && t < best) best = t;  // first run is warm-up
  }
  if (!rc) {
    const double flops = 2.0 * 8.0 * (double)iters * threads * blocks;
    *gflops = flops / (best * 1e-3) / 1e9;
    if (ms) *ms = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return rc;
}

extern "C" int df_probe_fp64_chains(int warps_per_sm, int chains, int iters, double* ns_per_step,
                                    double* gflops) {
  if (warps_per_sm < 1 || warps_per_sm > 32 || iters < 1 || !ns_per_step ||
      !(chains == 1 || chains == 2 || chains == 4 || chains == 8))
    return set_error(DF_EINVAL, "df_probe_fp64_chains: warps_per_sm in [1, 32], chains in {1, 2, 4, 8}, "
                                "iters >= 1, ns_per_step required");
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  int sms = 0;
  if ((rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return rc;
  const int threads = 32 * warps_per_sm;
  const int blocks = sms;
  double* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rc = cuda_check(cudaMalloc(&out, sizeof(double) * threads * blocks), "cudaMalloc");
  if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
  if (!rc) rc = cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = cuda_check(cudaEventCreate(&e1), "event");
  float t = 0.f;
  for (int rep = 0; rep < 2 && !rc; ++rep) {  // the first run is a warm-up
    cudaEventRecord(e0, st);
    switch (chains) {
      case 1: k_fma_chains<1><<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7); break;
      case 2: k_fma_chains<2><<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7); break;
      case 4: k_fma_chains<4><<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7); break;
      default: k_fma_chains<8><<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-7); break;
    }
    cudaEventRecord(e1, st);
    rc = cuda_check(cudaEventSynchronize(e1), "chain probe kernel");
    if (!rc) rc = cuda_check(cudaEventElapsedTime(&t, e0, e1), "elapsed");
  }
  if (!rc) {
    *ns_per_step = (double)t * 1e6 / iters;
    if (gflops) *gflops = 2.0 * chains * (double)iters * threads * blocks / (t * 1e-3) / 1e9;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  return rc;
}
