// DNN chemistry integrator (Sec. 2.3; Sec. 3.2 DNNInferencer): Box-Cox
// features, a fully connected network with three GELU hidden layers on the
// tcgen05 GEMM (gemm_host.cu), the inverse transform, T from the conserved
// enthalpy (Sec. 3.2 correctThermo) and the FP64 integrator as the fallback for
// cells outside the training range.  Training: MSE on the normalised change of
// F(Y), backward through the same GEMM, Adam on FP32 master weights.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "chem_thread.cuh"
#include "common.cuh"
#include "gemm_host.cuh"
#include "tc_gemm.cuh"

namespace df {

constexpr int DNN_IN = 16;   // padded feature count (2 + N <= 16)
constexpr int DNN_OUT = 16;  // padded output count (N <= 14: two inputs are T and p)

struct DnnLayout {
  int w[3];
  int64_t off[8];  // W1 b1 W2 b2 W3 b3 W4 b4
  int64_t total;
  __host__ __device__ int out(int l) const { return l < 3 ? w[l] : DNN_OUT; }
  __host__ __device__ int in(int l) const { return l == 0 ? DNN_IN : w[l - 1]; }
};

static DnnLayout make_layout(const df_dnn_opts& o) {
  DnnLayout L;
  for (int i = 0; i < 3; ++i) L.w[i] = o.width[i];
  int64_t p = 0;
  for (int l = 0; l < 4; ++l) {
    L.off[2 * l] = p;
    p += (int64_t)L.out(l) * L.in(l);
    L.off[2 * l + 1] = p;
    p += L.out(l);
  }
  L.total = p;
  return L;
}

}  // namespace df

struct df_dnn {
  df_dnn_opts o;
  df::DnnLayout L;
  int device = 0;
  int64_t step = 0;
  // FP32 master parameters, Adam moments, gradients (same layout)
  float* params = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grads = nullptr;
  // bf16 weights [out][in] and transposes [in][out]
  __nv_bfloat16* wb[4] = {nullptr, nullptr, nullptr, nullptr};
  __nv_bfloat16* wtb[4] = {nullptr, nullptr, nullptr, nullptr};
  // normalisation: mean_in, std_in, in_min, in_max (DNN_IN each), mean_out, std_out (DNN_OUT)
  float* norm = nullptr;
  float norm_host[4 * df::DNN_IN + 2 * df::DNN_OUT];
  // training scratch (batch rows B)
  int64_t B = 0;
  __nv_bfloat16 *X = nullptr, *XT = nullptr;
  float* Z[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16* H[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16* HT[3] = {nullptr, nullptr, nullptr};
  float *U = nullptr, *tgt = nullptr;
  __nv_bfloat16 *dU = nullptr, *dUT = nullptr;
  __nv_bfloat16* dZ[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16* dZT[3] = {nullptr, nullptr, nullptr};
  double* loss_part = nullptr;  // per-block partial sums
  // training step replayed from a CUDA graph: the batch is copied into these
  // buffers and the step's scalars (lr, bias corrections) read from train_sc
  double *bT = nullptr, *bp = nullptr, *bY = nullptr, *bYn = nullptr;
  float* train_sc = nullptr;
  float* splitk_ws = nullptr;  // split-K partial sums of the small-output GEMMs (weight gradients)
  size_t splitk_elems = 0;
  cudaGraphExec_t train_exec = nullptr;
  int64_t train_n = -1;
  cudaStream_t cap_stream = nullptr;  // private stream the step is captured on
  bool no_graph = false;              // capture unavailable here: enqueue the kernels directly
  // inference scratch (chunk rows)
  int64_t chunk = 0;
  __nv_bfloat16 *iX = nullptr, *iH[3] = {nullptr, nullptr, nullptr};
  float* iU = nullptr;
  int32_t* imask = nullptr;
  float* iYl = nullptr;   // [16][chunk] Y^lambda of the chunk, FP32 (features -> post)
  double* rawb = nullptr;  // raw-variable range bounds: lo[16], hi[16] (T, p, Y_k)
  // fallback list, per-cell flags and status scratch (grown on demand)
  int64_t list_cap = 0;
  int32_t* list = nullptr;
  int32_t* fb_status = nullptr;
  uint8_t* fb_flag = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_ranged = nullptr, ev_fallback = nullptr;
  unsigned long long* counter = nullptr;
  int* err = nullptr;
};

namespace df {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  // SplitMix64 finaliser (Steele, Lea & Flood 2014)
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Glorot-uniform weights for the real (unpadded) fan-in / fan-out, zero bias
__global__ void k_dnn_init(float* P, DnnLayout L, int n_in, int n_out, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.total) return;
  for (int l = 0; l < 4; ++l) {
    const int64_t w0 = L.off[2 * l], b0 = L.off[2 * l + 1];
    const int in = L.in(l), out = L.out(l);
    if (i >= w0 && i < b0) {
      const int64_t e = i - w0;
      const int r = (int)(e / in), c = (int)(e % in);
      const int rin = l == 0 ? n_in : in, rout = l == 3 ? n_out : out;
      if (r >= rout || c >= rin) {
        P[i] = 0.0f;
        return;
      }
      const double a = sqrt(6.0 / (rin + rout));
      const double u = (mix64(seed ^ mix64((uint64_t)i)) >> 11) * (1.0 / 9007199254740992.0);
      P[i] = (float)((2.0 * u - 1.0) * a);
      return;
    }
    if (i >= b0 && i < b0 + out) {
      P[i] = 0.0f;
      return;
    }
  }
}

// bf16 copies of W [out][in]: wb in the same layout and wtb = W^T [in][out],
// through a 32 x 32 shared-memory tile so both writes coalesce
__global__ void k_dnn_cast(const float* W, int out, int in, __nv_bfloat16* wb, __nv_bfloat16* wtb) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j, c = c0 + tx;
    if (r < out && c < in) {
      const __nv_bfloat16 b = __float2bfloat16_rn(W[(int64_t)r * in + c]);
      wb[(int64_t)r * in + c] = b;
      tile[j][tx] = b;
    }
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int c = c0 + j, r = r0 + tx;
    if (r < out && c < in) wtb[(int64_t)c * out + r] = tile[tx][j];
  }
}

// Box-Cox transform in FP64: F(Y) = (max(Y, 0)^lambda - 1) / lambda
__device__ __forceinline__ double ylam(double Y, double lam, const double2* tab) {
  return Y > 0.0 ? exp_tang(lam * log(Y), tab) : 0.0;
}

struct FeatArgs {
  int64_t ncells;  // stride of the SoA arrays
  int64_t c0, n;   // cells [c0, c0 + n)
  int N;
  double lam;
  const double *T, *p, *Y, *Ynext;
  const float* norm;  // mean_in, std_in, in_min, in_max, mean_out, std_out
  float margin;
  __nv_bfloat16* X;   // [n][16]
  __nv_bfloat16* XT;  // [16][ldT] or null
  int64_t ldT;
  float* tgt;         // [n][16] or null (normalised change of F(Y))
  int32_t* mask;      // [n] in-range flag or null
};

__global__ void k_dnn_features(FeatArgs a) {
  __shared__ double2 tab[64];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = g_exp2_tab[i];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t c = a.c0 + i;
  const float* mean_in = a.norm;
  const float* std_in = a.norm + DNN_IN;
  const float* lo = a.norm + 2 * DNN_IN;
  const float* hi = a.norm + 3 * DNN_IN;
  const float* mean_out = a.norm + 4 * DNN_IN;
  const float* std_out = a.norm + 4 * DNN_IN + DNN_OUT;
  float f[DNN_IN];
#pragma unroll
  for (int k = 0; k < DNN_IN; ++k) f[k] = 0.0f;
  f[0] = (float)a.T[c];
  f[1] = (float)a.p[c];
  double yl[16];
  for (int k = 0; k < a.N; ++k) {
    yl[k] = ylam(a.Y[(int64_t)k * a.ncells + c], a.lam, tab);
    f[2 + k] = (float)((yl[k] - 1.0) / a.lam);
  }
  bool in_range = true;
  __nv_bfloat16 xb[DNN_IN];
#pragma unroll
  for (int k = 0; k < DNN_IN; ++k) {
    const bool real = k < 2 + a.N;
    if (real) {
      const float w = hi[k] - lo[k];
      in_range = in_range && f[k] >= lo[k] - a.margin * w && f[k] <= hi[k] + a.margin * w;
    }
    xb[k] = __float2bfloat16_rn(real ? (f[k] - mean_in[k]) / std_in[k] : 0.0f);
  }
  uint4* xo = reinterpret_cast<uint4*>(a.X + i * DNN_IN);
  xo[0] = *reinterpret_cast<const uint4*>(xb);
  xo[1] = *reinterpret_cast<const uint4*>(xb + 8);
  if (a.XT) {
#pragma unroll
    for (int k = 0; k < DNN_IN; ++k) a.XT[(int64_t)k * a.ldT + i] = xb[k];
  }
  if (a.mask) a.mask[i] = in_range ? 1 : 0;
  if (a.tgt) {
    float* t = a.tgt + i * DNN_OUT;
#pragma unroll
    for (int k = 0; k < DNN_OUT; ++k) t[k] = 0.0f;
    for (int k = 0; k < a.N; ++k) {
      const double yn = ylam(a.Ynext[(int64_t)k * a.ncells + c], a.lam, tab);
      const double du = (yn - yl[k]) / a.lam;
      t[k] = (float)((du - mean_out[k]) / std_out[k]);
    }
  }
}

// Training features, one thread per (row, species): the same values as
// k_dnn_features (F(Y) in FP64, rounded to FP32, z-scored in FP32, rounded to
// BF16; the target's change of F(Y) in FP64), with the FP64 transforms of a
// row spread over N threads so that a 4096-row batch occupies the SMs and no
// lane of the narrow FP64 pipe idles (a thread per row left the log and
// exponential chains of all species exposed).  The thread of species s also
// writes the row's columns s, s + N, ... of the 16 - N inputs that are not
// species (T, p, zero padding) and of the 16 - N zero target columns.
// Writes X [n][16], XT [16][ldT] and tgt [n][16].
__global__ void k_dnn_features_train(FeatArgs a) {
  __shared__ double2 tab[64];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = g_exp2_tab[i];
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / a.N;
  const int sp = (int)(t - i * a.N);
  if (i >= a.n) return;
  const int64_t c = a.c0 + i;
  const float* mean_in = a.norm;
  const float* std_in = a.norm + DNN_IN;
  const float* mean_out = a.norm + 4 * DNN_IN;
  const float* std_out = a.norm + 4 * DNN_IN + DNN_OUT;
  const double yl = ylam(a.Y[(int64_t)sp * a.ncells + c], a.lam, tab);
  const float f = (float)((yl - 1.0) / a.lam);
  const __nv_bfloat16 xs = __float2bfloat16_rn((f - mean_in[2 + sp]) / std_in[2 + sp]);
  a.X[i * DNN_IN + 2 + sp] = xs;
  a.XT[(int64_t)(2 + sp) * a.ldT + i] = xs;
  const double yn = ylam(a.Ynext[(int64_t)sp * a.ncells + c], a.lam, tab);
  const double du = (yn - yl) / a.lam;
  float* trow = a.tgt + i * DNN_OUT;
  trow[sp] = (float)((du - mean_out[sp]) / std_out[sp]);
  // inputs other than species: 0 -> T, 1 -> p, then the padding 2 + N .. 15
  for (int e = sp; e < DNN_IN - a.N; e += a.N) {
    const int k = e < 2 ? e : e + a.N;
    float xk = 0.0f;
    if (k == 0) xk = ((float)a.T[c] - mean_in[0]) / std_in[0];
    if (k == 1) xk = ((float)a.p[c] - mean_in[1]) / std_in[1];
    const __nv_bfloat16 xb = __float2bfloat16_rn(xk);
    a.X[i * DNN_IN + k] = xb;
    a.XT[(int64_t)k * a.ldT + i] = xb;
  }
  for (int e = a.N + sp; e < DNN_OUT; e += a.N) trow[e] = 0.0f;
}

// Training-range test on the raw variables: the Box-Cox transform is monotonic,
// so [min, max] of F(Y_k) maps to bounds on Y_k; cells outside any bound are
// flagged and appended to the fallback list (one atomic per cell outside).
__device__ __forceinline__ double ipow(double a, int e) {
  double r = 1.0;
  while (e > 0) {
    if (e & 1) r *= a;
    a *= a;
    e >>= 1;
  }
  return r;
}

// Y^lambda in FP64 without a logarithm, for lambda = 1/m with m an integer.
// Y = f 2^(m q) exactly (integer operations on the exponent field: f keeps
// Y's mantissa with exponent r = e mod m, so f lies in [1, 2^m)), hence
// Y^lambda = f^(1/m) 2^q.  f^(1/m) is seeded in FP32 (relative error ~2e-7)
// and refined by one Newton step on x^m = f, x <- x - x (1 - f / x^m) / m,
// which squares the relative error (to about (m-1)/2 * 4e-14); 1 / x^m is an
// FP32 reciprocal refined by one Newton step.  Nine FP64 operations where a
// logarithm and an exponential take several times that on the narrow FP64
// pipe.  f^(1/m) lies in [1, 2), so 2^q goes straight into the exponent
// field (the result is never subnormal for lambda <= 1).
__device__ __forceinline__ double ylam_newton(double Y, int m, float lamf, double inv_m) {
  if (!(Y > 0.0)) return 0.0;
  int eadj = 0;
  if (Y < 2.2250738585072014e-308) {  // subnormal: scale by 2^54 first
    Y *= 18014398509481984.0;
    eadj = -54;
  }
  const long long bits = __double_as_longlong(Y);
  const int e = (int)((bits >> 52) & 0x7FF) - 1023 + eadj;
  int q = e / m, r = e - q * m;
  if (r < 0) {
    r += m;
    --q;
  }
  const double f = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | ((long long)(r + 1023) << 52));
  const float x0f = powf((float)f, lamf);
  const double x0 = (double)x0f;
  double xm;
  if (m == 10) {
    const double x2 = x0 * x0, x4 = x2 * x2;
    xm = x4 * x4 * x2;
  } else {
    xm = ipow(x0, m);
  }
  const double r0 = (double)__frcp_rn((float)xm);
  const double r1 = r0 * fma(-xm, r0, 2.0);
  const double d = fma(-f, r1, 1.0);
  const double x1 = fma(x0, -inv_m * d, x0);
  return __longlong_as_double(__double_as_longlong(x1) + ((long long)q << 52));
}

// Inference features (stage 1): the encoding of k_dnn_features (F(Y) in FP64,
// rounded to FP32, z-scored in FP32, rounded to BF16) with Y^lambda from
// ylam_newton.  Y^lambda is kept, in FP32, for the post stage, which uses it
// only in ratios or next to a change of its own size (see k_dnn_post).
struct FeatInferArgs {
  int64_t ncells, c0, n;
  int N;
  int inv_lam;  // 1 / lambda (integer)
  float lam;
  const double *T, *p, *Y;
  const float* norm;
  __nv_bfloat16* X;  // [n][16]
  float* Yl;         // [N][ldYl]
  int64_t ldYl;
};

__global__ void k_dnn_features_infer(FeatInferArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t c = a.c0 + i;
  const float* mean_in = a.norm;
  const float* std_in = a.norm + DNN_IN;
  __nv_bfloat16 xb[DNN_IN];
#pragma unroll
  for (int k = 0; k < DNN_IN; ++k) xb[k] = __float2bfloat16_rn(0.0f);
  xb[0] = __float2bfloat16_rn(((float)a.T[c] - mean_in[0]) / std_in[0]);
  xb[1] = __float2bfloat16_rn(((float)a.p[c] - mean_in[1]) / std_in[1]);
  const double inv_m = 1.0 / a.inv_lam, mm = (double)a.inv_lam;
#pragma unroll
  for (int k = 0; k < DNN_IN - 2; ++k) {
    if (k < a.N) {
      const double yl = ylam_newton(a.Y[(int64_t)k * a.ncells + c], a.inv_lam, a.lam, inv_m);
      a.Yl[(int64_t)k * a.ldYl + i] = (float)yl;
      const float fk = (float)fma(yl, mm, -mm);  // (Y^lambda - 1) / lambda
      xb[2 + k] = __float2bfloat16_rn((fk - mean_in[2 + k]) / std_in[2 + k]);
    }
  }
  uint4* xo = reinterpret_cast<uint4*>(a.X + i * DNN_IN);
  xo[0] = *reinterpret_cast<const uint4*>(xb);
  xo[1] = *reinterpret_cast<const uint4*>(xb + 8);
}

__global__ void k_dnn_range(int64_t ncells, int N, const double* T, const double* p, const double* Y,
                            const double* rawb, uint8_t* flag, int32_t* list, unsigned long long* counter) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const double* lo = rawb;
  const double* hi = rawb + DNN_IN;
  bool in = T[c] >= lo[0] && T[c] <= hi[0] && p[c] >= lo[1] && p[c] <= hi[1];
  for (int k = 0; k < N; ++k) {
    const double y = fmax(Y[(int64_t)k * ncells + c], 0.0);
    in = in && y >= lo[2 + k] && y <= hi[2 + k];
  }
  flag[c] = in ? 0 : 1;
  if (!in) list[atomicAdd(counter, 1ull)] = (int32_t)c;
}

// zero the rows [n, nrows) of a padded batch (features and their transpose)
__global__ void k_dnn_zero_rows(__nv_bfloat16* X, __nv_bfloat16* XT, int64_t ldT, int64_t n, int64_t nrows) {
  const int64_t i = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int k = 0; k < DNN_IN; ++k) {
    X[i * DNN_IN + k] = __float2bfloat16_rn(0.0f);
    XT[(int64_t)k * ldT + i] = __float2bfloat16_rn(0.0f);
  }
}

// loss = sum over rows < n and outputs < N of (U - tgt)^2 / (n_norm N) (the
// mean when n_norm = n; a shard's share of the mean over n_norm rows
// otherwise); dU = dloss/dU as bf16 [rows][16] and its transpose [16][ldT];
// per-block partial sums of the squared errors
// rows per block of the loss kernel (a 4096-row batch spreads over 64 SMs)
constexpr int LOSS_ROWS = 64;

__global__ void k_dnn_loss(const float* U, const float* tgt, int64_t n, int64_t n_norm, int64_t nrows, int N,
                           __nv_bfloat16* dU, __nv_bfloat16* dUT, int64_t ldT, double* part) {
  __shared__ double red[LOSS_ROWS];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < nrows) {
    const double scale = 2.0 / ((double)n_norm * N);
#pragma unroll
    for (int k = 0; k < DNN_OUT; ++k) {
      float g = 0.0f;
      if (i < n && k < N) {
        const double d = (double)U[i * DNN_OUT + k] - (double)tgt[i * DNN_OUT + k];
        acc += d * d;
        g = (float)(scale * d);
      }
      const __nv_bfloat16 gb = __float2bfloat16_rn(g);
      dU[i * DNN_OUT + k] = gb;
      dUT[(int64_t)k * ldT + i] = gb;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out = sum of the n partials in a fixed order (lane-strided sums, then a
// fixed shuffle tree; one warp)
__global__ void k_sum_partials(const double* part, int n, double* out) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[0] = s;
}

// bias gradient: db[r] = sum over the first ncol columns of the bf16 row r, in
// a fixed order (each thread a strided partial, then a tree): FP32 sums, whose
// error (~(ncol / blockDim + log2 blockDim) ulp of the sum of |terms|) sits far
// below the BF16 rounding of the terms; FP64 on the narrow pipe cost more than
// the GEMMs of the step
__global__ void k_dnn_rowsum(const __nv_bfloat16* A, int64_t ld, int rows, int64_t ncol, float* db) {
  const int r = blockIdx.x;
  if (r >= rows) return;
  __shared__ float red[256];
  float acc = 0.0f;
  for (int64_t c = threadIdx.x; c < ncol; c += blockDim.x) acc += __bfloat162float(A[(int64_t)r * ld + c]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[r] = red[0];
}

// sc = {lr, 1 - beta1^t, 1 - beta2^t} of this step (device memory, so a
// captured step can be replayed with new values)
__global__ void k_set_train_scalars(float* sc, float lr, float c1, float c2) {
  sc[0] = lr;
  sc[1] = c1;
  sc[2] = c2;
}

// Adam (Kingma & Ba 2015, Algorithm 1) in FP32 on the master weights; the
// coefficients beta and 1 - beta are rounded to FP32 from their FP64 values
// (1 - (float)0.999 would be 5e-5 off 0.001)
__global__ void k_adam(float* P, float* m1, float* m2, const float* g, int64_t n, const float* sc, float b1,
                       float omb1, float b2, float omb2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float lr = sc[0], c1 = sc[1], c2 = sc[2];
  const float gi = g[i];
  const float a = b1 * m1[i] + omb1 * gi;
  const float b = b2 * m2[i] + omb2 * (gi * gi);
  m1[i] = a;
  m2[i] = b;
  P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

struct PostArgs {
  int64_t ncells, c0, n;
  int N;
  double lam;
  int inv_lam;  // 1 / lambda (integer)
  const double* blob;
  MechDims d;
  double* T;
  const double* p;
  double* Y;
  const float* U;  // [n][16] normalised network output
  const float* norm;
  const uint8_t* flag;  // [ncells] 1: advanced by the fallback
  const float* Yl;      // [N][ldYl] Y^lambda of the chunk (FP32)
  int64_t ldYl;
  int32_t* used_fallback;
  int32_t* status;
  int32_t* list;
  unsigned long long* counter;
  uint32_t inert;  // bit k: species k has a zero net stoichiometric coefficient in every reaction
};

// Stage 3 of the inference: Y' = F^{-1}(F(Y) + u), renormalised, and T' from
// h(T', Y') = h(T, Y) at fixed p.  Species that no reaction changes (bits of
// a.inert) keep their input mass fraction exactly, as the kinetics has it; the
// others are scaled so that the mass fractions sum to one.
//
// Y' is formed as Y + dY.  With z = Y^lambda and r = lambda u / z, Y' = Y (1 + r)^m
// (m = 1/lambda) exactly, so for |r| <= 1/2 dY = Y expm1(m log1p(r)) carries the
// relative precision of r however small the change; z enters only through the
// ratio, so its FP32 value suffices.  For larger changes (and Y = 0), Y' = (z +
// lambda u)^m directly.
//
// T' = T + tau with the enthalpy balance written in differences, so it needs no
// FP64: with h_k(T) = sum_j c_kj T^j the NASA-7 enthalpy over R per unit mass,
//   sum_k Y'_k [h_k(T + tau) - h_k(T)] = sum_k (Y_k - Y'_k) h_k(T) = R,
// and the left side is tau (t1 + tau (t2 + ... tau t5)), t_i the Taylor
// coefficients at T of the mixture polynomial sum_k Y'_k h_k (t1 = cp/R).  Every
// term keeps its relative precision in FP32 (no large h is ever subtracted), and
// Newton on tau converges in a few steps; only Y' - Y, the renormalisation and
// T + tau are FP64.
__global__ void k_dnn_post(PostArgs a) {
  __shared__ float hc[DNN_OUT][6];
  const double* sp = a.blob + a.d.off_sp;
  for (int t = threadIdx.x; t < a.N * 6; t += blockDim.x) {
    const int k = t / 6, j = t % 6;
    const double iw = sp[SP_REC * k + 1];
    const double* c7 = sp + SP_REC * k + 2;
    hc[k][j] = (float)(iw * (j == 0 ? c7[5] : c7[j - 1] / (double)j));
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t c = a.c0 + i;
  if (a.flag[c]) {
    if (a.used_fallback) a.used_fallback[c] = 1;
    return;
  }
  const float* mean_out = a.norm + 4 * DNN_IN;
  const float* std_out = a.norm + 4 * DNN_IN + DNN_OUT;
  const float lamf = (float)a.lam;
  const float m = (float)a.inv_lam;
  double Yo[DNN_OUT], Yn[DNN_OUT];
  double s = 0.0, s_inert = 0.0;
#pragma unroll
  for (int k = 0; k < DNN_OUT; ++k) {
    if (k < a.N) {
      const double y = a.Y[(int64_t)k * a.ncells + c];
      Yo[k] = y;
      if ((a.inert >> k) & 1u) {
        Yn[k] = y;
        s_inert += y;
        continue;
      }
      const float lu = lamf * fmaf(a.U[i * DNN_OUT + k], std_out[k], mean_out[k]);
      const float z = a.Yl[(int64_t)k * a.ldYl + i];
      double yn;
      if (z > 0.0f && fabsf(lu) <= 0.5f * z) {
        yn = fma(y, (double)expm1f(m * log1pf(lu / z)), y);
      } else {
        const double zz = (double)z + (double)lu;
        yn = zz > 0.0 ? ipow(zz, a.inv_lam) : 0.0;
      }
      Yn[k] = yn;
      s += yn;
    }
  }
  // (1 - s_inert) / s: FP32 reciprocal of s and one Newton step (s is within
  // rounding of 1 - s_inert, far from zero when the reacting species carry mass)
  double is = 0.0;
  if (s > 0.0) {
    const double r0 = (double)__frcp_rn((float)s);
    is = (1.0 - s_inert) * (r0 * fma(-s, r0, 2.0));
  }
  const double T0 = a.T[c];
  const float Tf = (float)T0;
  float D[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float R = 0.0f;
#pragma unroll
  for (int k = 0; k < DNN_OUT; ++k) {
    if (k < a.N) {
      if (!((a.inert >> k) & 1u)) Yn[k] *= is;
      const float yf = (float)Yn[k];
      const float dy = (float)(Yo[k] - Yn[k]);
      float hk = hc[k][5];
#pragma unroll
      for (int j = 4; j >= 0; --j) hk = fmaf(hk, Tf, hc[k][j]);
      R = fmaf(dy, hk, R);
#pragma unroll
      for (int j = 0; j < 6; ++j) D[j] = fmaf(yf, hc[k][j], D[j]);
    }
  }
  // Taylor coefficients at T of sum_j D_j x^j: t_i = sum_{j >= i} C(j, i) D_j T^(j-i)
  const float T1 = Tf, T2 = T1 * T1, T3 = T2 * T1, T4 = T3 * T1;
  const float t1 = D[1] + 2.f * D[2] * T1 + 3.f * D[3] * T2 + 4.f * D[4] * T3 + 5.f * D[5] * T4;
  const float t2 = D[2] + 3.f * D[3] * T1 + 6.f * D[4] * T2 + 10.f * D[5] * T3;
  const float t3 = D[3] + 4.f * D[4] * T1 + 10.f * D[5] * T2;
  const float t4 = D[4] + 5.f * D[5] * T1;
  const float t5 = D[5];
  float tau = R / t1;
#pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    const float g = tau * (t1 + tau * (t2 + tau * (t3 + tau * (t4 + tau * t5)))) - R;
    const float dg = t1 + tau * (2.f * t2 + tau * (3.f * t3 + tau * (4.f * t4 + tau * 5.f * t5)));
    const float step = g / dg;
    tau -= step;
    if (fabsf(step) <= 1e-7f * fabsf(tau)) break;
  }
  a.T[c] = T0 + (double)tau;
#pragma unroll
  for (int k = 0; k < DNN_OUT; ++k)
    if (k < a.N) a.Y[(int64_t)k * a.ncells + c] = Yn[k];
  if (a.used_fallback) a.used_fallback[c] = 0;
  if (a.status) a.status[c] = DF_CELL_OK;
}

__global__ void k_copy_status(const int32_t* list, const unsigned long long* count, const int32_t* src,
                              int32_t* dst) {
  const int64_t n = (int64_t)*count;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[list[i]] = src[list[i]];
}

// ---------------------------------------------------------------------------
// norm statistics: per-block FP64 partials (sum, sum of squares, min, max) of
// the 2 + N input features and the N output changes; fixed-order final sum
// ---------------------------------------------------------------------------
constexpr int NSTAT = DNN_IN + DNN_OUT;

__global__ void k_dnn_stats(int64_t n, int N, double lam, const double* T, const double* p, const double* Y,
                            const double* Yn, double* part) {
  __shared__ double2 tab[64];
  __shared__ double s1[256], s2[256], smin[256], smax[256];
  for (int i = threadIdx.x; i < 64; i += blockDim.x) tab[i] = g_exp2_tab[i];
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int f = 0; f < NSTAT; ++f) {
    double v = 0.0;
    bool valid = c < n;
    if (valid) {
      if (f == 0) v = T[c];
      else if (f == 1) v = p[c];
      else if (f < 2 + N) v = (ylam(Y[(int64_t)(f - 2) * n + c], lam, tab) - 1.0) / lam;
      else if (f >= DNN_IN && f < DNN_IN + N) {
        const int k = f - DNN_IN;
        v = (ylam(Yn[(int64_t)k * n + c], lam, tab) - ylam(Y[(int64_t)k * n + c], lam, tab)) / lam;
      } else valid = false;
    }
    s1[threadIdx.x] = valid ? v : 0.0;
    s2[threadIdx.x] = valid ? v * v : 0.0;
    smin[threadIdx.x] = valid ? v : INFINITY;
    smax[threadIdx.x] = valid ? v : -INFINITY;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        s1[threadIdx.x] += s1[threadIdx.x + s];
        s2[threadIdx.x] += s2[threadIdx.x + s];
        smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
        smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double* o = part + ((int64_t)blockIdx.x * NSTAT + f) * 4;
      o[0] = s1[0];
      o[1] = s2[0];
      o[2] = smin[0];
      o[3] = smax[0];
    }
    __syncthreads();
  }
}

__global__ void k_dnn_stats_final(const double* part, int64_t nblocks, int64_t n, int N, float* norm) {
  const int f = threadIdx.x;
  if (f >= NSTAT) return;
  double s1 = 0.0, s2 = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int64_t b = 0; b < nblocks; ++b) {
    const double* o = part + (b * NSTAT + f) * 4;
    s1 += o[0];
    s2 += o[1];
    mn = fmin(mn, o[2]);
    mx = fmax(mx, o[3]);
  }
  const double mean = s1 / n;
  double var = s2 / n - mean * mean;
  double sd = var > 0.0 ? sqrt(var) : 0.0;
  // a constant feature (an inert species' change) keeps a tiny scale, so the
  // network's residual output on it maps back to (almost) no change
  if (!(sd > 1e-30)) sd = 1e-30;
  if (f < DNN_IN) {
    const bool real = f < 2 + N;
    norm[f] = real ? (float)mean : 0.0f;
    norm[DNN_IN + f] = real ? (float)sd : 1.0f;
    norm[2 * DNN_IN + f] = real ? (float)mn : 0.0f;
    norm[3 * DNN_IN + f] = real ? (float)mx : 0.0f;
  } else {
    const int k = f - DNN_IN;
    const bool real = k < N;
    norm[4 * DNN_IN + k] = real ? (float)mean : 0.0f;
    norm[4 * DNN_IN + DNN_OUT + k] = real ? (float)sd : 1.0f;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int dev_alloc(void** p, size_t bytes) {
  return cuda_check(cudaMalloc(p, std::max<size_t>(bytes, 16)), "cudaMalloc (DNN)");
}

static int dnn_cast_all(df_dnn* d, cudaStream_t st) {
  for (int l = 0; l < 4; ++l) {
    const int out = d->L.out(l), in = d->L.in(l);
    const dim3 grid((unsigned)((in + 31) / 32), (unsigned)((out + 31) / 32));
    k_dnn_cast<<<grid, dim3(32, 8), 0, st>>>(d->params + d->L.off[2 * l], out, in, d->wb[l], d->wtb[l]);
  }
  return cuda_check(cudaGetLastError(), "weight cast");
}

static int dnn_alloc(df_dnn* d) {
  const DnnLayout& L = d->L;
  int rc = 0;
  rc = rc ? rc : dev_alloc((void**)&d->params, L.total * 4);
  rc = rc ? rc : dev_alloc((void**)&d->m1, L.total * 4);
  rc = rc ? rc : dev_alloc((void**)&d->m2, L.total * 4);
  rc = rc ? rc : dev_alloc((void**)&d->grads, L.total * 4);
  for (int l = 0; l < 4 && !rc; ++l) {
    const size_t n = (size_t)L.out(l) * L.in(l);
    rc = dev_alloc((void**)&d->wb[l], n * 2);
    if (!rc) rc = dev_alloc((void**)&d->wtb[l], n * 2);
  }
  rc = rc ? rc : dev_alloc((void**)&d->norm, sizeof(d->norm_host));
  rc = rc ? rc : dev_alloc((void**)&d->rawb, 2 * DNN_IN * sizeof(double));
  rc = rc ? rc : dev_alloc((void**)&d->counter, 16);
  rc = rc ? rc : dev_alloc((void**)&d->err, 16);
  if (rc) return rc;
  cudaMemset(d->m1, 0, L.total * 4);
  cudaMemset(d->m2, 0, L.total * 4);
  cudaMemset(d->grads, 0, L.total * 4);
  cudaMemset(d->err, 0, 16);
  return cuda_check(cudaGetLastError(), "DNN buffers");
}

static int dnn_train_buffers(df_dnn* d) {
  if (d->X) return DF_OK;
  const int64_t B = ((int64_t)d->o.batch + 7) / 8 * 8;
  d->B = B;
  int rc = 0;
  rc = rc ? rc : dev_alloc((void**)&d->X, B * DNN_IN * 2);
  rc = rc ? rc : dev_alloc((void**)&d->XT, B * DNN_IN * 2);
  for (int l = 0; l < 3 && !rc; ++l) {
    const int w = d->L.w[l];
    rc = dev_alloc((void**)&d->Z[l], B * w * 4);
    if (!rc) rc = dev_alloc((void**)&d->H[l], B * w * 2);
    if (!rc) rc = dev_alloc((void**)&d->HT[l], B * w * 2);
    if (!rc) rc = dev_alloc((void**)&d->dZ[l], B * w * 2);
    if (!rc) rc = dev_alloc((void**)&d->dZT[l], B * w * 2);
  }
  rc = rc ? rc : dev_alloc((void**)&d->U, B * DNN_OUT * 4);
  rc = rc ? rc : dev_alloc((void**)&d->tgt, B * DNN_OUT * 4);
  rc = rc ? rc : dev_alloc((void**)&d->dU, B * DNN_OUT * 2);
  rc = rc ? rc : dev_alloc((void**)&d->dUT, B * DNN_OUT * 2);
  rc = rc ? rc : dev_alloc((void**)&d->loss_part, ((B + LOSS_ROWS - 1) / LOSS_ROWS + 1) * 8);
  rc = rc ? rc : dev_alloc((void**)&d->bT, B * 8);
  rc = rc ? rc : dev_alloc((void**)&d->bp, B * 8);
  rc = rc ? rc : dev_alloc((void**)&d->bY, B * d->o.n_species * 8);
  rc = rc ? rc : dev_alloc((void**)&d->bYn, B * d->o.n_species * 8);
  rc = rc ? rc : dev_alloc((void**)&d->train_sc, 4 * 4);
  d->splitk_elems = (size_t)2 << 20;
  rc = rc ? rc : dev_alloc((void**)&d->splitk_ws, d->splitk_elems * 4);
  return rc;
}

static int dnn_infer_buffers(df_dnn* d) {
  if (d->iX) return DF_OK;
  const int64_t C = d->o.infer_chunk;
  d->chunk = C;
  int rc = dev_alloc((void**)&d->iX, C * DNN_IN * 2);
  for (int l = 0; l < 3 && !rc; ++l) rc = dev_alloc((void**)&d->iH[l], C * d->L.w[l] * 2);
  rc = rc ? rc : dev_alloc((void**)&d->iU, C * DNN_OUT * 4);
  rc = rc ? rc : dev_alloc((void**)&d->iYl, C * DNN_OUT * 4);
  if (!rc && !d->side)
    rc = cuda_check(cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking), "fallback stream");
  if (!rc && !d->ev_ranged) rc = cuda_check(cudaEventCreateWithFlags(&d->ev_ranged, cudaEventDisableTiming), "event");
  if (!rc && !d->ev_fallback)
    rc = cuda_check(cudaEventCreateWithFlags(&d->ev_fallback, cudaEventDisableTiming), "event");
  return rc;
}

// Bounds of the raw variables equivalent to the feature range [in_min, in_max]
// widened by range_margin: T and p directly, Y_k through the inverse Box-Cox
// transform F^{-1}(z) = max(1 + lambda z, 0)^{1/lambda} (monotonic).
static int update_raw_bounds(df_dnn* d) {
  double b[2 * DNN_IN];
  const float* lo = d->norm_host + 2 * DNN_IN;
  const float* hi = d->norm_host + 3 * DNN_IN;
  const double lam = d->o.lambda, mg = d->o.range_margin;
  for (int k = 0; k < DNN_IN; ++k) {
    // the bounds are stored in FP32: widen each by one FP32 ulp so a training
    // value that the rounding moved past its bound still counts as inside
    double l = std::nextafter(lo[k], -INFINITY), h = std::nextafter(hi[k], INFINITY);
    if (std::isfinite(l) && std::isfinite(h)) {
      const double w = h - l;
      l -= mg * w;
      h += mg * w;
    }
    if (k >= 2) {
      auto inv = [&](double z) -> double {
        if (z == INFINITY) return INFINITY;
        const double a = 1.0 + lam * z;
        return a > 0.0 ? std::pow(a, 1.0 / lam) : 0.0;
      };
      const double yl = inv(l), yh = inv(h);
      // a lower bound at F(0) = -1/lambda admits Y = 0 exactly
      l = (1.0 + lam * l <= 0.0) ? -INFINITY : yl;
      h = yh;
    }
    b[k] = l;
    b[DNN_IN + k] = h;
  }
  return cuda_check(cudaMemcpy(d->rawb, b, sizeof(b), cudaMemcpyHostToDevice), "range bounds");
}

static int gemm(df_dnn* d, const void* A, int ldA, const void* B, int ldB, int M, int N, int K, int mode,
                const float* bias, float* out0, int ld0, __nv_bfloat16* out1, int ld1, __nv_bfloat16* out2,
                int ld2, const float* aux, int lda, cudaStream_t st) {
  GemmParams P;
  memset(&P, 0, sizeof(P));
  P.M = M;
  P.N = N;
  P.K = K;
  P.ldA = ldA;
  P.ldB = ldB;
  P.mode = mode;
  P.bias = bias;
  P.aux = aux;
  P.lda = lda;
  P.out0 = out0;
  P.ld0 = ld0;
  P.out1 = out1;
  P.ld1 = ld1;
  P.out2 = out2;
  P.ld2 = ld2;
  P.err = d->err;
  if (mode == EPI_F32) {
    P.ws = d->splitk_ws;
    P.ws_elems = d->splitk_ws ? d->splitk_elems : 0;
  }
  return gemm_bf16(A, B, P, st, 0);
}

// inference layers: X [M][16] bf16 -> U [M][16] f32
static int dnn_forward_infer(df_dnn* d, const __nv_bfloat16* X, int64_t M, float* U, cudaStream_t st) {
  const DnnLayout& L = d->L;
  const float* P = d->params;
  int rc = gemm(d, X, 0, d->wb[0], 0, (int)M, L.w[0], DNN_IN, EPI_GELU_BF16, P + L.off[1], nullptr, 0, d->iH[0],
                L.w[0], nullptr, 0, nullptr, 0, st);
  if (!rc)
    rc = gemm(d, d->iH[0], 0, d->wb[1], 0, (int)M, L.w[1], L.w[0], EPI_GELU_BF16, P + L.off[3], nullptr, 0,
              d->iH[1], L.w[1], nullptr, 0, nullptr, 0, st);
  if (!rc)
    rc = gemm(d, d->iH[1], 0, d->wb[2], 0, (int)M, L.w[2], L.w[1], EPI_GELU_BF16, P + L.off[5], nullptr, 0,
              d->iH[2], L.w[2], nullptr, 0, nullptr, 0, st);
  if (!rc)
    rc = gemm(d, d->iH[2], 0, d->wb[3], 0, (int)M, DNN_OUT, L.w[2], EPI_F32, P + L.off[7], U, DNN_OUT, nullptr, 0,
              nullptr, 0, nullptr, 0, st);
  return rc;
}

static int check_err_flag(df_dnn* d, cudaStream_t st) {
  int h = 0;
  int rc = cuda_check(cudaMemcpyAsync(&h, d->err, 4, cudaMemcpyDeviceToHost, st), "read DNN error flag");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "synchronise");
  if (!rc && h) {
    cudaMemsetAsync(d->err, 0, 4, st);
    return set_error(DF_ETIMEOUT, "a tensor-core pipeline wait ran out");
  }
  return rc;
}

}  // namespace df

using namespace df;

extern "C" {

void df_dnn_opts_default(df_dnn_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->n_species = 9;
  o->width[0] = 1600;
  o->width[1] = 800;
  o->width[2] = 400;
  o->lambda = 0.1;
  o->batch = 4096;
  o->infer_chunk = 262144;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->adam_eps = 1e-8;
  o->range_margin = 0.0;
}

static int check_opts(const df_dnn_opts& o) {
  if (o.n_species < 1 || o.n_species + 2 > DNN_IN || o.n_species > DNN_OUT)
    return set_error(DF_EINVAL, "df_dnn: n_species must be in [1, 14]");
  for (int i = 0; i < 3; ++i)
    if (o.width[i] < 8 || o.width[i] % 8 != 0 || o.width[i] > 16384)
      return set_error(DF_EINVAL, "df_dnn: hidden widths must be multiples of 8 in [8, 16384]");
  const double inv = 1.0 / o.lambda;
  if (!(o.lambda > 0.0) || std::fabs(inv - std::round(inv)) > 1e-9 || inv > 64)
    return set_error(DF_EINVAL, "df_dnn: 1/lambda must be an integer <= 64");
  if (o.batch < 8 || o.infer_chunk < 128 || o.infer_chunk > (1 << 23))
    return set_error(DF_EINVAL, "df_dnn: batch >= 8, infer_chunk in [128, 2^23]");
  return DF_OK;
}

int df_dnn_create(const df_dnn_opts* opts, uint64_t seed, df_dnn** out) {
  if (!out) return set_error(DF_EINVAL, "df_dnn_create: null output");
  *out = nullptr;
  df_dnn_opts o;
  if (opts) o = *opts;
  else df_dnn_opts_default(&o);
  int rc = check_opts(o);
  if (rc) return rc;
  df_dnn* d = new (std::nothrow) df_dnn();
  if (!d) return set_error(DF_ENOMEM, "df_dnn_create");
  d->o = o;
  d->L = make_layout(o);
  cudaGetDevice(&d->device);
  rc = dnn_alloc(d);
  if (rc) {
    df_dnn_free(d);
    return rc;
  }
  k_dnn_init<<<(unsigned)((d->L.total + 255) / 256), 256>>>(d->params, d->L, o.n_species + 2, o.n_species, seed);
  rc = cuda_check(cudaGetLastError(), "DNN init");
  if (!rc) rc = dnn_cast_all(d, 0);
  // identity normalisation, infinite range
  for (int k = 0; k < DNN_IN; ++k) {
    d->norm_host[k] = 0.0f;
    d->norm_host[DNN_IN + k] = 1.0f;
    d->norm_host[2 * DNN_IN + k] = -INFINITY;
    d->norm_host[3 * DNN_IN + k] = INFINITY;
  }
  for (int k = 0; k < DNN_OUT; ++k) {
    d->norm_host[4 * DNN_IN + k] = 0.0f;
    d->norm_host[4 * DNN_IN + DNN_OUT + k] = 1.0f;
  }
  if (!rc)
    rc = cuda_check(cudaMemcpy(d->norm, d->norm_host, sizeof(d->norm_host), cudaMemcpyHostToDevice), "norm");
  if (!rc) rc = update_raw_bounds(d);
  if (!rc) rc = cuda_check(cudaDeviceSynchronize(), "DNN create");
  if (rc) {
    df_dnn_free(d);
    return rc;
  }
  *out = d;
  return DF_OK;
}

void df_dnn_free(df_dnn* d) {
  if (!d) return;
  void* ptrs[] = {d->params, d->m1, d->m2, d->grads, d->norm, d->X, d->XT, d->U, d->tgt, d->dU, d->dUT,
                  d->loss_part, d->iX, d->iU, d->imask, d->list, d->fb_status, d->counter, d->err, d->iYl,
                  d->rawb, d->fb_flag, d->bT, d->bp, d->bY, d->bYn, d->train_sc, d->splitk_ws};
  if (d->train_exec) cudaGraphExecDestroy(d->train_exec);
  if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
  if (d->side) cudaStreamDestroy(d->side);
  if (d->ev_ranged) cudaEventDestroy(d->ev_ranged);
  if (d->ev_fallback) cudaEventDestroy(d->ev_fallback);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int l = 0; l < 4; ++l) {
    if (d->wb[l]) cudaFree(d->wb[l]);
    if (d->wtb[l]) cudaFree(d->wtb[l]);
  }
  for (int l = 0; l < 3; ++l) {
    void* q[] = {d->Z[l], d->H[l], d->HT[l], d->dZ[l], d->dZT[l], d->iH[l]};
    for (void* p : q)
      if (p) cudaFree(p);
  }
  delete d;
}

int df_dnn_set_norm(df_dnn* d, const float* mean_in, const float* std_in, const float* mean_out,
                    const float* std_out, const float* in_min, const float* in_max) {
  if (!d) return set_error(DF_EINVAL, "df_dnn_set_norm: null handle");
  const int nin = d->o.n_species + 2, nout = d->o.n_species;
  const float* src[6] = {mean_in, std_in, in_min, in_max, mean_out, std_out};
  const int off[6] = {0, DNN_IN, 2 * DNN_IN, 3 * DNN_IN, 4 * DNN_IN, 4 * DNN_IN + DNN_OUT};
  for (int a = 0; a < 6; ++a) {
    if (!src[a]) continue;
    const int cnt = a < 4 ? nin : nout;
    for (int k = 0; k < cnt; ++k) {
      if ((a == 1 || a == 5) && !(src[a][k] > 0.0f)) return set_error(DF_EINVAL, "df_dnn_set_norm: std <= 0");
      d->norm_host[off[a] + k] = src[a][k];
    }
  }
  int rc = cuda_check(cudaMemcpy(d->norm, d->norm_host, sizeof(d->norm_host), cudaMemcpyHostToDevice), "norm");
  if (!rc) rc = update_raw_bounds(d);
  return rc;
}

int df_dnn_get_norm(const df_dnn* d, float* mean_in, float* std_in, float* mean_out, float* std_out,
                    float* in_min, float* in_max) {
  if (!d) return set_error(DF_EINVAL, "df_dnn_get_norm: null handle");
  const int nin = d->o.n_species + 2, nout = d->o.n_species;
  float* dst[6] = {mean_in, std_in, in_min, in_max, mean_out, std_out};
  const int off[6] = {0, DNN_IN, 2 * DNN_IN, 3 * DNN_IN, 4 * DNN_IN, 4 * DNN_IN + DNN_OUT};
  for (int a = 0; a < 6; ++a)
    if (dst[a]) memcpy(dst[a], d->norm_host + off[a], sizeof(float) * (a < 4 ? nin : nout));
  return DF_OK;
}

int df_dnn_fit_norm(df_dnn* d, int64_t n, const double* T, const double* p, const double* Y, const double* Yn,
                    df_stream_t stream) {
  if (!d || n < 1 || !T || !p || !Y || !Yn) return set_error(DF_EINVAL, "df_dnn_fit_norm: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nb = (n + 255) / 256;
  double* part = nullptr;
  int rc = cuda_check(cudaMallocAsync(&part, (size_t)nb * NSTAT * 4 * 8, st), "stats scratch");
  if (rc) return rc;
  k_dnn_stats<<<(unsigned)nb, 256, 0, st>>>(n, d->o.n_species, d->o.lambda, T, p, Y, Yn, part);
  k_dnn_stats_final<<<1, 64, 0, st>>>(part, nb, n, d->o.n_species, d->norm);
  rc = cuda_check(cudaGetLastError(), "stats kernels");
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(d->norm_host, d->norm, sizeof(d->norm_host), cudaMemcpyDeviceToHost, st),
                    "read norm");
  cudaFreeAsync(part, st);
  if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "synchronise");
  if (!rc) rc = update_raw_bounds(d);
  return rc;
}

// The kernels of one forward and backward pass on the staged batch (bT, bp,
// bY, bYn): the loss partials and the gradients (d->grads), no update.
static int dnn_grad_enqueue(df_dnn* d, int64_t n, int64_t n_norm, cudaStream_t st) {
  const DnnLayout& L = d->L;
  const int64_t B = d->B;
  const int64_t M = (n + 7) / 8 * 8;  // rows used by the GEMMs (K of the weight gradients)
  const int N = d->o.n_species;
  int rc = DF_OK;
  FeatArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.ncells = n;
  fa.c0 = 0;
  fa.n = n;
  fa.N = N;
  fa.lam = d->o.lambda;
  fa.T = d->bT;
  fa.p = d->bp;
  fa.Y = d->bY;
  fa.Ynext = d->bYn;
  fa.norm = d->norm;
  fa.margin = 0.0f;
  fa.X = d->X;
  fa.XT = d->XT;
  fa.ldT = B;
  fa.tgt = d->tgt;
  k_dnn_features_train<<<(unsigned)(((int64_t)N * n + 255) / 256), 256, 0, st>>>(fa);
  if (M > n) k_dnn_zero_rows<<<1, 8, 0, st>>>(d->X, d->XT, B, n, M);
  float* P = d->params;
  float* G = d->grads;
  // forward (keep Z, H, H^T)
  const __nv_bfloat16* in = d->X;
  for (int l = 0; l < 3 && !rc; ++l) {
    rc = gemm(d, in, 0, d->wb[l], 0, (int)M, L.w[l], L.in(l), EPI_TRAIN_FWD, P + L.off[2 * l + 1], d->Z[l], L.w[l],
              d->H[l], L.w[l], d->HT[l], (int)B, nullptr, 0, st);
    in = d->H[l];
  }
  if (!rc)
    rc = gemm(d, d->H[2], 0, d->wb[3], 0, (int)M, DNN_OUT, L.w[2], EPI_F32, P + L.off[7], d->U, DNN_OUT, nullptr, 0,
              nullptr, 0, nullptr, 0, st);
  if (rc) return rc;
  const int nbl = (int)((M + LOSS_ROWS - 1) / LOSS_ROWS);
  k_dnn_loss<<<nbl, LOSS_ROWS, 0, st>>>(d->U, d->tgt, n, n_norm, M, N, d->dU, d->dUT, B, d->loss_part);
  k_sum_partials<<<1, 32, 0, st>>>(d->loss_part, nbl, d->loss_part + nbl);
  // backward: layer 4
  rc = gemm(d, d->dUT, (int)B, d->HT[2], (int)B, DNN_OUT, L.w[2], (int)M, EPI_F32, nullptr, G + L.off[6], L.w[2],
            nullptr, 0, nullptr, 0, nullptr, 0, st);
  k_dnn_rowsum<<<DNN_OUT, 256, 0, st>>>(d->dUT, B, DNN_OUT, M, G + L.off[7]);
  // dZ3 = (dU W4) * gelu'(Z3)
  if (!rc)
    rc = gemm(d, d->dU, 0, d->wtb[3], 0, (int)M, L.w[2], DNN_OUT, EPI_BWD_DZ, nullptr, nullptr, 0, d->dZ[2], L.w[2],
              d->dZT[2], (int)B, d->Z[2], L.w[2], st);
  for (int l = 2; l >= 0 && !rc; --l) {
    // weight gradient of layer l: dZ_l^T . H_{l-1}  (H_{-1} = X)
    const __nv_bfloat16* hinT = l > 0 ? d->HT[l - 1] : d->XT;
    const int in_w = L.in(l);
    rc = gemm(d, d->dZT[l], (int)B, hinT, (int)B, L.w[l], in_w, (int)M, EPI_F32, nullptr, G + L.off[2 * l], in_w,
              nullptr, 0, nullptr, 0, nullptr, 0, st);
    k_dnn_rowsum<<<L.w[l], 256, 0, st>>>(d->dZT[l], B, L.w[l], M, G + L.off[2 * l + 1]);
    if (!rc && l > 0)
      rc = gemm(d, d->dZ[l], 0, d->wtb[l], 0, (int)M, L.w[l - 1], L.w[l], EPI_BWD_DZ, nullptr, nullptr, 0,
                d->dZ[l - 1], L.w[l - 1], d->dZT[l - 1], (int)B, d->Z[l - 1], L.w[l - 1], st);
  }
  return cuda_check(cudaGetLastError(), "gradient kernels");
}

// Adam (bias-corrected, scalars of this step in train_sc) on the master
// weights with the gradients in d->grads, then the bf16 copies.
static int dnn_adam_enqueue(df_dnn* d, cudaStream_t st) {
  const DnnLayout& L = d->L;
  const float b1 = (float)d->o.beta1, b2 = (float)d->o.beta2;
  const float omb1 = (float)(1.0 - d->o.beta1), omb2 = (float)(1.0 - d->o.beta2);
  k_adam<<<(unsigned)((L.total + 255) / 256), 256, 0, st>>>(d->params, d->m1, d->m2, d->grads, L.total,
                                                             d->train_sc, b1, omb1, b2, omb2, (float)d->o.adam_eps);
  int rc = cuda_check(cudaGetLastError(), "Adam kernel");
  if (!rc) rc = dnn_cast_all(d, st);
  return rc;
}

// The kernels of one training step on the staged batch.
static int dnn_train_enqueue(df_dnn* d, int64_t n, cudaStream_t st) {
  int rc = dnn_grad_enqueue(d, n, n, st);
  if (!rc) rc = dnn_adam_enqueue(d, st);
  return rc;
}

// Copy a batch into the library's staging buffers (the captured training step
// reads it from there).
static int dnn_stage_batch(df_dnn* d, int64_t n, const double* T, const double* p, const double* Y,
                           const double* Yn, cudaStream_t st) {
  const int N = d->o.n_species;
  int rc = cuda_check(cudaMemcpyAsync(d->bT, T, n * 8, cudaMemcpyDeviceToDevice, st), "stage T");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(d->bp, p, n * 8, cudaMemcpyDeviceToDevice, st), "stage p");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(d->bY, Y, n * N * 8, cudaMemcpyDeviceToDevice, st), "stage Y");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(d->bYn, Yn, n * N * 8, cudaMemcpyDeviceToDevice, st), "stage Y_next");
  return rc;
}

// this step's Adam scalars: lr and the bias corrections 1 - beta^t (t = d->step)
static int dnn_set_step_scalars(df_dnn* d, float lr, cudaStream_t st) {
  const float c1 = (float)(1.0 - std::pow(d->o.beta1, (double)d->step));
  const float c2 = (float)(1.0 - std::pow(d->o.beta2, (double)d->step));
  k_set_train_scalars<<<1, 1, 0, st>>>(d->train_sc, lr, c1, c2);
  return cuda_check(cudaGetLastError(), "train scalars");
}

// the loss of the step (squared errors over n_norm * N), when asked for
// (synchronises the stream)
static int train_step_loss(df_dnn* d, int64_t n, int64_t n_norm, int rc, float* loss_out, cudaStream_t st) {
  if (!rc && loss_out) {
    const int64_t M = (n + 7) / 8 * 8;
    const int nbl = (int)((M + LOSS_ROWS - 1) / LOSS_ROWS);
    double l = 0.0;
    rc = cuda_check(cudaMemcpyAsync(&l, d->loss_part + nbl, 8, cudaMemcpyDeviceToHost, st), "read loss");
    if (!rc) rc = check_err_flag(d, st);
    *loss_out = (float)(l / ((double)n_norm * d->o.n_species));
  }
  return rc;
}

int df_dnn_train_step(df_dnn* d, int64_t n, const double* T, const double* p, const double* Y, const double* Yn,
                      float lr, float* loss_out, df_stream_t stream) {
  if (!d || n < 1 || n > d->o.batch || !T || !p || !Y || !Yn)
    return set_error(DF_EINVAL, "df_dnn_train_step: bad arguments (1 <= n <= batch)");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = dnn_train_buffers(d);
  if (!rc) rc = dnn_stage_batch(d, n, T, p, Y, Yn, st);
  if (rc) return rc;
  d->step += 1;
  rc = dnn_set_step_scalars(d, lr, st);
  if (rc) return rc;
  // The step's ~25 launches are captured once per batch size, on a private
  // stream (the caller's may be the legacy stream, which cannot be captured),
  // after a first eager step has done the one-time set-up, and replayed on the
  // caller's stream.  Inside a caller's own stream capture they are simply
  // enqueued.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  rc = cuda_check(cudaStreamIsCapturing(st, &cs), "capture status");
  if (rc) return rc;
  if (cs != cudaStreamCaptureStatusNone || d->step == 1 || d->no_graph)
    return train_step_loss(d, n, n, dnn_train_enqueue(d, n, st), loss_out, st);
  if (!d->train_exec || d->train_n != n) {
    if (d->train_exec) cudaGraphExecDestroy(d->train_exec);
    d->train_exec = nullptr;
    d->train_n = -1;
    if (!d->cap_stream)
      rc = cuda_check(cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (rc) return rc;
    if (cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      d->no_graph = true;  // capture unavailable: run the kernels as they are from now on
      return train_step_loss(d, n, n, dnn_train_enqueue(d, n, st), loss_out, st);
    }
    const int erc = dnn_train_enqueue(d, n, d->cap_stream);
    cudaGraph_t g = nullptr;
    rc = cuda_check(cudaStreamEndCapture(d->cap_stream, &g), "end capture");
    if (erc) {
      if (g) cudaGraphDestroy(g);
      return erc;
    }
    if (!rc) rc = cuda_check(cudaGraphInstantiate(&d->train_exec, g, 0), "instantiate training graph");
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    d->train_n = n;
  }
  rc = cuda_check(cudaGraphLaunch(d->train_exec, st), "launch training graph");
  return train_step_loss(d, n, n, rc, loss_out, st);
}

int df_dnn_grad(df_dnn* d, int64_t n, int64_t n_total, const double* T, const double* p, const double* Y,
                const double* Yn, float* loss_out, df_stream_t stream) {
  if (!d || n < 1 || n > d->o.batch || n_total < n || !T || !p || !Y || !Yn)
    return set_error(DF_EINVAL, "df_dnn_grad: bad arguments (1 <= n <= batch, n_total >= n)");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = dnn_train_buffers(d);
  if (!rc) rc = dnn_stage_batch(d, n, T, p, Y, Yn, st);
  if (!rc) rc = dnn_grad_enqueue(d, n, n_total, st);
  return train_step_loss(d, n, n_total, rc, loss_out, st);
}

int df_dnn_grad_buffer(df_dnn* d, float** grads, int64_t* count) {
  if (!d || !grads) return set_error(DF_EINVAL, "df_dnn_grad_buffer: bad arguments");
  *grads = d->grads;
  if (count) *count = d->L.total;
  return DF_OK;
}

int df_dnn_adam_step(df_dnn* d, float lr, df_stream_t stream) {
  if (!d) return set_error(DF_EINVAL, "df_dnn_adam_step: null handle");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = dnn_train_buffers(d);
  if (rc) return rc;
  d->step += 1;
  rc = dnn_set_step_scalars(d, lr, st);
  if (!rc) rc = dnn_adam_enqueue(d, st);
  return rc;
}

int df_dnn_get_adam_state(const df_dnn* d, float* m1, float* m2, int64_t* step) {
  if (!d) return set_error(DF_EINVAL, "df_dnn_get_adam_state: null handle");
  int rc = DF_OK;
  if (m1) rc = cuda_check(cudaMemcpy(m1, d->m1, d->L.total * 4, cudaMemcpyDeviceToHost), "read first moments");
  if (!rc && m2) rc = cuda_check(cudaMemcpy(m2, d->m2, d->L.total * 4, cudaMemcpyDeviceToHost), "read second moments");
  if (step) *step = d->step;
  return rc;
}

int df_dnn_forward_raw(df_dnn* d, int64_t n, const void* X, float* U, df_stream_t stream) {
  if (!d || n < 1 || !X || !U) return set_error(DF_EINVAL, "df_dnn_forward_raw: bad arguments");
  int rc = dnn_infer_buffers(d);
  if (rc) return rc;
  if (n > d->chunk) return set_error(DF_EINVAL, "df_dnn_forward_raw: n exceeds the inference chunk");
  cudaStream_t st = (cudaStream_t)stream;
  rc = dnn_forward_infer(d, static_cast<const __nv_bfloat16*>(X), n, U, st);
  if (!rc) rc = check_err_flag(d, st);
  return rc;
}

int df_dnn_infer(df_dnn* d, const df_mech* mc, int64_t ncells, double* T, const double* p, double* Y, double dt,
                 const df_integ_opts* fopts, int32_t* used_fallback, int64_t* n_fallback, int32_t* status,
                 df_stream_t stream) {
  if (!d || !mc || ncells < 0 || (ncells > 0 && (!T || !p || !Y)))
    return set_error(DF_EINVAL, "df_dnn_infer: bad arguments");
  if (mc->dims.N != d->o.n_species) return set_error(DF_EINVAL, "df_dnn_infer: mechanism and network disagree on N");
  if (n_fallback) *n_fallback = 0;
  if (ncells == 0) return DF_OK;
  df_mech* m = const_cast<df_mech*>(mc);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = dnn_infer_buffers(d);
  if (rc) return rc;
  if (d->list_cap < ncells) {
    if (d->list) cudaFree(d->list);
    if (d->fb_status) cudaFree(d->fb_status);
    if (d->fb_flag) cudaFree(d->fb_flag);
    d->list = nullptr;
    d->fb_status = nullptr;
    d->fb_flag = nullptr;
    rc = dev_alloc((void**)&d->list, ncells * 4);
    if (!rc) rc = dev_alloc((void**)&d->fb_status, ncells * 4);
    if (!rc) rc = dev_alloc((void**)&d->fb_flag, ncells);
    if (rc) return rc;
    d->list_cap = ncells;
  }
  // 1. training-range test over all cells -> fallback list (device count)
  rc = cuda_check(cudaMemsetAsync(d->counter, 0, 8, st), "reset fallback counter");
  if (rc) return rc;
  k_dnn_range<<<(unsigned)((ncells + 255) / 256), 256, 0, st>>>(ncells, d->o.n_species, T, p, Y, d->rawb,
                                                                d->fb_flag, d->list, d->counter);
  rc = cuda_check(cudaGetLastError(), "range kernel");
  // 2. the FP64 integrator advances the fallback cells on a side stream (its
  //    work count stays on the device); the network runs on the caller's stream
  df_integ_opts o;
  if (fopts) o = *fopts;
  else df_integ_opts_default(&o);
  if (o.reactor != 0) return set_error(DF_EUNSUPPORTED, "df_dnn_infer: the network is a constant-pressure model");
  if (!rc) rc = cuda_check(cudaEventRecord(d->ev_ranged, st), "event");
  if (!rc) rc = cuda_check(cudaStreamWaitEvent(d->side, d->ev_ranged, 0), "event wait");
  if (!rc)
    rc = launch_integrate_list(m, ncells, T, p, Y, dt, o, d->fb_status, nullptr, d->list, ncells, d->side,
                               d->counter);
  if (!rc && status) {
    k_copy_status<<<256, 256, 0, d->side>>>(d->list, d->counter, d->fb_status, status);
    rc = cuda_check(cudaGetLastError(), "fallback status copy");
  }
  if (!rc) rc = cuda_check(cudaEventRecord(d->ev_fallback, d->side), "event");
  // 3. the network on the other cells, chunk by chunk
  const int inv = (int)std::lround(1.0 / d->o.lambda);
  uint32_t inert = 0;  // species with an empty (reaction, net nu) list
  for (int k = 0; k < m->dims.N && k < 32; ++k)
    if (m->csr_host[k + 1] == m->csr_host[k]) inert |= 1u << k;
  for (int64_t c0 = 0; c0 < ncells && !rc; c0 += d->chunk) {
    const int64_t nc = std::min<int64_t>(d->chunk, ncells - c0);
    FeatInferArgs fa;
    fa.ncells = ncells;
    fa.c0 = c0;
    fa.n = nc;
    fa.N = d->o.n_species;
    fa.lam = (float)d->o.lambda;
    fa.inv_lam = inv;
    fa.T = T;
    fa.p = p;
    fa.Y = Y;
    fa.norm = d->norm;
    fa.X = d->iX;
    fa.Yl = d->iYl;
    fa.ldYl = d->chunk;
    k_dnn_features_infer<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(fa);
    rc = dnn_forward_infer(d, d->iX, nc, d->iU, st);
    if (rc) break;
    PostArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.ncells = ncells;
    pa.c0 = c0;
    pa.n = nc;
    pa.N = d->o.n_species;
    pa.lam = d->o.lambda;
    pa.inv_lam = inv;
    pa.blob = m->blob_dev;
    pa.d = m->dims;
    pa.T = T;
    pa.p = p;
    pa.Y = Y;
    pa.U = d->iU;
    pa.norm = d->norm;
    pa.flag = d->fb_flag;
    pa.Yl = d->iYl;
    pa.ldYl = d->chunk;
    pa.used_fallback = used_fallback;
    pa.status = status;
    pa.inert = inert;
    k_dnn_post<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(pa);
    rc = cuda_check(cudaGetLastError(), "DNN pre/post kernels");
  }
  // 4. join the fallback, report the count
  if (!rc) rc = cuda_check(cudaStreamWaitEvent(st, d->ev_fallback, 0), "event wait");
  unsigned long long nfb = 0;
  if (!rc) rc = cuda_check(cudaMemcpyAsync(&nfb, d->counter, 8, cudaMemcpyDeviceToHost, st), "read fallback count");
  if (!rc) rc = check_err_flag(d, st);
  if (rc) return rc;
  if (n_fallback) *n_fallback = (int64_t)nfb;
  return DF_OK;
}

int64_t df_dnn_param_count(const df_dnn* d) { return d ? d->L.total : 0; }

int df_dnn_get_params(const df_dnn* d, float* host) {
  if (!d || !host) return set_error(DF_EINVAL, "df_dnn_get_params: bad arguments");
  return cuda_check(cudaMemcpy(host, d->params, d->L.total * 4, cudaMemcpyDeviceToHost), "read params");
}

int df_dnn_get_grads(const df_dnn* d, float* host) {
  if (!d || !host) return set_error(DF_EINVAL, "df_dnn_get_grads: bad arguments");
  return cuda_check(cudaMemcpy(host, d->grads, d->L.total * 4, cudaMemcpyDeviceToHost), "read grads");
}

int df_dnn_set_params(df_dnn* d, const float* host) {
  if (!d || !host) return set_error(DF_EINVAL, "df_dnn_set_params: bad arguments");
  int rc = cuda_check(cudaMemcpy(d->params, host, d->L.total * 4, cudaMemcpyHostToDevice), "write params");
  if (!rc) rc = dnn_cast_all(d, 0);
  if (!rc) rc = cuda_check(cudaDeviceSynchronize(), "cast");
  return rc;
}

static const char DNN_MAGIC[8] = {'D', 'F', 'D', 'N', 'N', '0', '0', '1'};

int df_dnn_save(const df_dnn* d, const char* path) {
  if (!d || !path) return set_error(DF_EINVAL, "df_dnn_save: bad arguments");
  std::vector<float> h(d->L.total);
  int rc = df_dnn_get_params(d, h.data());
  if (rc) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(DF_EINVAL, std::string("df_dnn_save: cannot open ") + path);
  bool ok = fwrite(DNN_MAGIC, 1, 8, f) == 8 && fwrite(&d->o, sizeof(d->o), 1, f) == 1 &&
            fwrite(d->norm_host, sizeof(d->norm_host), 1, f) == 1 &&
            fwrite(h.data(), 4, h.size(), f) == h.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? DF_OK : set_error(DF_EINVAL, "df_dnn_save: write failed");
}

int df_dnn_load(const char* path, df_dnn** out) {
  if (!path || !out) return set_error(DF_EINVAL, "df_dnn_load: bad arguments");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(DF_EINVAL, std::string("df_dnn_load: cannot open ") + path);
  char magic[8];
  df_dnn_opts o;
  float norm[4 * DNN_IN + 2 * DNN_OUT];
  bool ok = fread(magic, 1, 8, f) == 8 && !memcmp(magic, DNN_MAGIC, 8) && fread(&o, sizeof(o), 1, f) == 1 &&
            fread(norm, sizeof(norm), 1, f) == 1;
  int rc = ok ? check_opts(o) : set_error(DF_EINVAL, "df_dnn_load: not a network file");
  df_dnn* d = nullptr;
  if (!rc) rc = df_dnn_create(&o, 0, &d);
  if (!rc) {
    std::vector<float> h(d->L.total);
    if (fread(h.data(), 4, h.size(), f) != h.size()) rc = set_error(DF_EINVAL, "df_dnn_load: truncated file");
    if (!rc) rc = df_dnn_set_params(d, h.data());
    if (!rc) {
      memcpy(d->norm_host, norm, sizeof(norm));
      rc = cuda_check(cudaMemcpy(d->norm, d->norm_host, sizeof(norm), cudaMemcpyHostToDevice), "norm");
      if (!rc) rc = update_raw_bounds(d);
    }
  }
  fclose(f);
  if (rc) {
    df_dnn_free(d);
    return rc;
  }
  *out = d;
  return DF_OK;
}

}  // extern "C"
