// Host side of the tcgen05 GEMM: TMA tensor maps (cuTensorMapEncodeTiled reached
// through the runtime's driver entry point, so the library does not link the
// driver library) and the launch.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <string>

#include "common.cuh"
#include "gemm_host.cuh"
#include "tc_gemm.cuh"
#include "../../include/df_probe.h"

namespace df {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2D bf16 tensor [rows][K] (K contiguous), tiles of 64 (K) x box_rows, 128-byte swizzle
static int make_tmap(CUtensorMap* m, const void* ptr, int64_t rows, int64_t K, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error(DF_ECUDA, "cuTensorMapEncodeTiled unavailable");
  if (ld == 0) ld = K;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || (K % 8) != 0 || (ld % 8) != 0 || ld < K || rows < 1 ||
      K < 1)
    return set_error(DF_EINVAL, "GEMM operand must be 16-byte aligned with K and its row pitch multiples of 8");
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)GEMM_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DF_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return DF_OK;
}

// ring depth of the one-tile-per-CTA kernel: six stages (192 KB) for the
// 128-wide tile, whose main users are the weight gradients (K = the batch,
// 4096: a three-stage ring left the loads' latency exposed), three for the
// 64- and 256-wide tiles (the 64-wide output layer keeps three CTAs per SM)
template <int BN>
constexpr int gemm_stages() {
  return BN == 128 ? 6 : 3;
}

template <int BN>
static size_t gemm_smem() {
  return (size_t)gemm_stages<BN>() * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) + 1024 + 256;
}

// out0[r][c] = sum_z ws[z][r][c] (+ bias[c]), z in order
__global__ void k_splitk_reduce(const float* ws, int splits, int M, int N, const float* bias, float* out, int ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * N) return;
  const int r = (int)(i / N), c = (int)(i - (int64_t)r * N);
  float acc = 0.0f;
  for (int z = 0; z < splits; ++z) acc += ws[(int64_t)z * M * N + i];
  if (bias) acc += bias[c];
  out[(int64_t)r * ld + c] = acc;
}

template <int BN>
static int gemm_launch_bn(const void* A, const void* B, const GemmParams& P, cudaStream_t st) {
  CUtensorMap ta, tb;
  int rc = make_tmap(&ta, A, P.M, P.K, P.ldA, GEMM_BM);
  if (!rc) rc = make_tmap(&tb, B, P.N, P.K, P.ldB, BN);
  if (rc) return rc;
  auto kf = k_gemm_tc<BN, gemm_stages<BN>()>;
  const size_t sm = gemm_smem<BN>();
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    rc = cuda_check(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                    "set GEMM shared memory");
    if (rc) return rc;
    attr_set[dev] = true;
  }
  dim3 grid((P.N + BN - 1) / BN, (P.M + GEMM_BM - 1) / GEMM_BM);
  if (grid.y > 65535) return set_error(DF_EUNSUPPORTED, "GEMM M too large for one launch");
  // split-K when the output has few tiles but the reduction is long (weight
  // gradients: K = the batch): enough CTAs for the SMs, at least two k-blocks
  // each, within the caller's workspace
  GemmParams Q = P;
  Q.splits = 1;
  if (P.mode == EPI_F32 && P.ws && P.ws_elems > 0) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (int64_t)grid.x * grid.y;
    const int nk = (P.K + GEMM_BK - 1) / GEMM_BK;
    int64_t sp = std::min<int64_t>(nk / 2, (nsm + tiles - 1) / tiles);
    sp = std::min<int64_t>(sp, (int64_t)(P.ws_elems / ((size_t)P.M * P.N)));
    if (tiles * 2 <= nsm && sp >= 2) Q.splits = (int)sp;
  }
  grid.z = Q.splits;
  kf<<<grid, 128, sm, st>>>(ta, tb, Q);
  rc = cuda_check(cudaGetLastError(), "GEMM launch");
  if (!rc && Q.splits > 1) {
    const int64_t mn = (int64_t)P.M * P.N;
    k_splitk_reduce<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(P.ws, Q.splits, P.M, P.N, P.bias, P.out0, P.ld0);
    rc = cuda_check(cudaGetLastError(), "split-K reduction");
  }
  return rc;
}

constexpr int PERS_STAGES = 4;

// 2D bf16 output tensor [rows][cols] (row pitch ld) for TMA stores of 32-row x
// 16-column blocks, no swizzle
static int make_tmap_store(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int64_t ld) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return set_error(DF_ECUDA, "cuTensorMapEncodeTiled unavailable");
  if (ld == 0) ld = cols;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || (cols % 8) != 0 || (ld % 8) != 0 || ld < cols || rows < 1)
    return set_error(DF_EINVAL, "GEMM output must be 16-byte aligned with N and its row pitch multiples of 8");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {16, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DF_ECUDA, "cuTensorMapEncodeTiled (store) failed: " + std::to_string((int)r));
  return DF_OK;
}

template <int BN, int MODE, int EW>
static int gemm_launch_pers_mode(const CUtensorMap& ta, const CUtensorMap& tb, const GemmParams& P, cudaStream_t st) {
  int rc = DF_OK;
  CUtensorMap tc;
  memset(&tc, 0, sizeof(tc));
  if (MODE == EPI_GELU_BF16) {
    if (!P.out1) return set_error(DF_EINVAL, "GEMM: bf16 output missing");
    rc = make_tmap_store(&tc, P.out1, P.M, P.N, P.ld1);
    if (rc) return rc;
  }
  auto kf = k_gemm_tc_pers<BN, PERS_STAGES, MODE, EW>;
  const size_t sm = (size_t)PERS_STAGES * (GEMM_BM * GEMM_BK * 2 + BN * GEMM_BK * 2) +
                    pers_epi_bytes(MODE, EW) + 1024 + 256;
  static int nsm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return set_error(DF_EUNSUPPORTED, "device index out of range");
  if (!nsm[dev]) {
    rc = cuda_check(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                    "set GEMM shared memory");
    if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (rc) {
      nsm[dev] = 0;
      return rc;
    }
  }
  const int64_t tiles = (int64_t)((P.M + GEMM_BM - 1) / GEMM_BM) * ((P.N + BN - 1) / BN);
  const int grid = (int)std::min<int64_t>(tiles, nsm[dev]);
  kf<<<grid, pers_threads(EW), sm, st>>>(ta, tb, tc, P);
  return cuda_check(cudaGetLastError(), "persistent GEMM launch");
}

template <int BN>
static int gemm_launch_pers(const void* A, const void* B, const GemmParams& P, cudaStream_t st) {
  CUtensorMap ta, tb;
  int rc = make_tmap(&ta, A, P.M, P.K, P.ldA, GEMM_BM);
  if (!rc) rc = make_tmap(&tb, B, P.N, P.K, P.ldB, BN);
  if (rc) return rc;
  // sixteen epilogue warps for the inference GELU layers (four per TMEM lane
  // quarter: on the 11-1600-800-400-9 network's 262144-row chunk the forward
  // pass took 1.16 ms against 1.45 ms with eight), twelve for the training
  // epilogues (their registers allow three warps per quarter: on 4096-row
  // batches the epilogue's latency, not the MMAs, sets the time), eight for
  // plain FP32 output
  switch (P.mode) {
    case EPI_F32:
      return gemm_launch_pers_mode<BN, EPI_F32, 8>(ta, tb, P, st);
    case EPI_GELU_BF16:
      return gemm_launch_pers_mode<BN, EPI_GELU_BF16, 16>(ta, tb, P, st);
    case EPI_TRAIN_FWD:
      return gemm_launch_pers_mode<BN, EPI_TRAIN_FWD, 12>(ta, tb, P, st);
    case EPI_BWD_DZ:
      return gemm_launch_pers_mode<BN, EPI_BWD_DZ, 12>(ta, tb, P, st);
    default:
      return set_error(DF_EINVAL, "GEMM epilogue mode");
  }
}

// tile width for the persistent kernel: each N-tile re-streams its 128-row A
// tile, so a tile costs about (BN + 128) column-units; minimise
// ceil(N / BN) * (BN + 128) (measured on 262144 x 800 x 1600: 128 / 160 / 208 /
// 256 wide took 0.714 / 0.573 / 0.534 / 0.617 ms, which this cost ranks
// alike), ties to the wider tile.  With fewer than 128 row tiles (M < 16384: the training batches) the
// last wave's balance matters as much: the cost is then the number of waves
// of tiles over the SMs times (BN + 128) (4096 x 1600: 208 wide, two waves, in
// place of 256 wide, two waves of which the second is half empty; 4096 x 400:
// 128 wide, one wave of 128 tiles, in place of 64 tiles 208 wide)
static int pick_bn(int N, int M, int nsm) {
  const int cand[4] = {256, 208, 160, 128};
  const int64_t nM = (M + GEMM_BM - 1) / GEMM_BM;
  const bool few = nM < 128 && nsm > 0;
  int best = 128;
  int64_t best_cost = INT64_MAX;
  for (int c : cand) {
    const int64_t nN = (N + c - 1) / c;
    const int64_t cost = (few ? (nM * nN + nsm - 1) / nsm : nN) * (c + 128);
    if (cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

int gemm_bf16(const void* A, const void* B, const GemmParams& P, cudaStream_t st, int bn) {
  if (P.M < 1 || P.N < 1 || P.K < 1 || (P.N % 8) != 0)
    return set_error(DF_EINVAL, "GEMM sizes: M, N, K >= 1 and N a multiple of 8");
  if (bn == 0) {
    static int nsm[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !nsm[dev] &&
        cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm[dev] = 0;
    const int sms = (dev >= 0 && dev < 64) ? nsm[dev] : 0;
    bn = P.N <= 64 ? 64 : (P.M >= 1024 ? -pick_bn(P.N, P.M, sms) : 128);
  }
  switch (bn) {
    case -128:
      return gemm_launch_pers<128>(A, B, P, st);
    case -160:
      return gemm_launch_pers<160>(A, B, P, st);
    case -208:
      return gemm_launch_pers<208>(A, B, P, st);
    case -256:
      return gemm_launch_pers<256>(A, B, P, st);
    case 64:
      return gemm_launch_bn<64>(A, B, P, st);
    case 128:
      return gemm_launch_bn<128>(A, B, P, st);
    case 256:
      return gemm_launch_bn<256>(A, B, P, st);
    default:
      return set_error(DF_EINVAL, "GEMM tile width must be 64, 128, 256 or (persistent) -128, -160, -208, -256");
  }
}

}  // namespace df

namespace df {
// GELU probe: the epilogues' pair function on (x[2i], x[2i+1]) (an odd last
// element paired with 0), or the derivative
__global__ void k_gelu_probe(const float* x, float* y, long long n, int derivative) {
  const long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  if (derivative) {
    y[i] = gelu_grad_f(x[i]);
    if (i + 1 < n) y[i + 1] = gelu_grad_f(x[i + 1]);
    return;
  }
  float g0, g1;
  gelu2_f(x[i], i + 1 < n ? x[i + 1] : 0.0f, g0, g1);
  y[i] = g0;
  if (i + 1 < n) y[i + 1] = g1;
}
}  // namespace df

using namespace df;

extern "C" int df_probe_gelu(const float* x, float* y, long long n, int derivative, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return set_error(DF_EINVAL, "df_probe_gelu: bad arguments");
  if (n == 0) return DF_OK;
  const long long pairs = (n + 1) / 2;
  k_gelu_probe<<<(unsigned)((pairs + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n, derivative);
  return cuda_check(cudaGetLastError(), "GELU probe kernel");
}

extern "C" int df_probe_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, int bn,
                                  int* err_flag, void* stream) {
  if (!A || !B || !C) return set_error(DF_EINVAL, "df_probe_gemm_bf16: null pointer");
  GemmParams P;
  memset(&P, 0, sizeof(P));
  P.M = M;
  P.N = N;
  P.K = K;
  P.mode = EPI_F32;
  P.out0 = C;
  P.ld0 = N;
  P.err = err_flag;
  return gemm_bf16(A, B, P, (cudaStream_t)stream, bn);
}
