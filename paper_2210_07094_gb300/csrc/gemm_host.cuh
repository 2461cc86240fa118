// Launch of the tcgen05 GEMM (gemm_host.cu).
#pragma once
#include <cuda_runtime.h>

namespace df {
struct GemmParams;
// C = A . B^T with the epilogue of P.mode; A [M][K], B [N][K] bf16 device
// arrays (16-byte aligned, K a multiple of 8).  bn: output tile width
// (0 = choose).
int gemm_bf16(const void* A, const void* B, const GemmParams& P, cudaStream_t st, int bn = 0);
}  // namespace df
