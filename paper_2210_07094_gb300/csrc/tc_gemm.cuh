// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05) with
// TMA loads and the accumulator in tensor memory, for the MLP of the DNN
// chemistry integrator (Sec. 2.3: a fully connected network with three hidden
// layers).
//
//   C[m, n] = sum_k A[m, k] B[n, k]     A: [M][K], B: [N][K], both K-contiguous
//
// One 128 x BN output tile per CTA (4 warps).  Warp 0 lane 0 issues the TMA
// loads of 128x64 (A) and BNx64 (B) bf16 tiles (128-byte swizzle) into a
// STAGES-deep ring guarded by mbarriers; warp 1 lane 0 issues tcgen05.mma
// (M = 128, N = BN, K = 16 per instruction) into a TMEM accumulator of BN fp32
// columns and releases each ring slot with tcgen05.commit; then all four warps
// read their 32 TMEM lanes (tcgen05.ld) and run the epilogue.  Every mbarrier
// wait is bounded: on timeout the kernel records an error code and still frees
// its tensor memory before it returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace df {

enum EpiMode : int {
  EPI_F32 = 0,        // out0 f32 [M][ld0] = acc (+ bias)
  EPI_GELU_BF16 = 1,  // out1 bf16 [M][ld1] = gelu(acc + bias)
  EPI_TRAIN_FWD = 2,  // out0 f32 Z = acc + bias; out1 bf16 gelu(Z); out2 bf16 gelu(Z)^T [N][ld2]
  EPI_BWD_DZ = 3,     // dZ = acc * gelu'(aux [M][lda]); out1 bf16 dZ; out2 bf16 dZ^T [N][ld2]
};

struct GemmParams {
  int M, N, K;
  int ldA, ldB;  // leading dimensions (elements) of the A and B operands (0: K)
  int mode;
  const float* bias;  // [N] or null
  const float* aux;   // EPI_BWD_DZ: pre-activation of the layer input
  int lda;
  float* out0;
  __nv_bfloat16* out1;
  __nv_bfloat16* out2;
  int ld0, ld1, ld2;
  int* err;           // device error flag (0 = ok)
  // EPI_F32 split-K (one-tile-per-CTA kernel): with splits > 1, CTA z sums
  // its share of the k-blocks into ws[z][M][N]; a second kernel adds the
  // slices in a fixed order into out0 (+ bias)
  int splits;
  float* ws;
  size_t ws_elems;
};

constexpr int GEMM_BM = 128;
constexpr int GEMM_BK = 64;
constexpr long long GEMM_WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait for the phase of the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > GEMM_WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row groups
// 1024 bytes apart (tile base 1024-byte aligned)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Phi(-|z|) = erfc(|z| / sqrt 2) / 2 by the Chebyshev-fitted form of Press,
// Teukolsky, Vetterling and Flannery (Numerical Recipes, Sec. 6.2):
// erfc(a) = t exp(-a^2 + P(t)), t = 1 / (1 + a/2), fractional error below
// 1.2e-7 for every a >= 0, so the deep tails of the GELU keep their relative
// accuracy.  Folded for the hardware exp2: with b = a sqrt(log2 e),
// erfc(a) / 2 = t 2^(-b^2 + log2(e) P(t) - 1); the coefficients below are
// log2(e) times the published ones (the constant term also carries the -1).
// One reciprocal, eleven FMA/MUL and one exp2 (hardware approximations,
// relative error ~2^-22).
__device__ __forceinline__ float half_erfc_scaled(float az) {
  constexpr double L2E = 1.4426950408889634;
  constexpr float kb = (float)(0.70710678118654752 * 1.2011224087864498);  // 1/sqrt2 * sqrt(log2 e)
  constexpr float kt = (float)(0.5 / 1.2011224087864498);
  const float b = az * kb;
  float t;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(kt, b, 1.0f)));
  float p = (float)(0.17087277 * L2E);
  p = fmaf(p, t, (float)(-0.82215223 * L2E));
  p = fmaf(p, t, (float)(1.48851587 * L2E));
  p = fmaf(p, t, (float)(-1.13520398 * L2E));
  p = fmaf(p, t, (float)(0.27886807 * L2E));
  p = fmaf(p, t, (float)(-0.18628806 * L2E));
  p = fmaf(p, t, (float)(0.09678418 * L2E));
  p = fmaf(p, t, (float)(0.37409196 * L2E));
  p = fmaf(p, t, (float)(1.00002368 * L2E));
  p = fmaf(p, t, (float)(-1.26551223 * L2E - 1.0));
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fmaf(-b, b, p)));
  return t * e;
}

// GELU(z) = z Phi(z), Phi the standard normal CDF (any z; the reference form)
__device__ __forceinline__ float gelu_tail_f(float z) {
  const float h = half_erfc_scaled(fabsf(z));
  return z * (z >= 0.0f ? 1.0f - h : h);
}

// Packed FP32 pairs: Blackwell's f32x2 instructions do two FP32 operations in
// one issue slot.  A pair lives in one 64-bit register (low half first).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
  f32x2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ constexpr f32x2 f2_splat_bits(uint32_t bits) {
  return ((f32x2)bits << 32) | (f32x2)bits;
}
__device__ __forceinline__ f32x2 f2_splat(float v) { return f2_splat_bits(__float_as_uint(v)); }

// GELU of a pair, z Phi(z).  With a = |z| <= GELU_FIT_A, Phi(-a) =
// 2^(-a^2 log2(e)/2 + Q(a)), where Q(a) = log2(Phi(-a) e^(a^2/2)) is smooth and
// slowly varying (-1 at a = 0, about -3.3 at a = 4) and is evaluated by a
// degree-8 polynomial in x = a/2 - 1, interpolated at the Chebyshev points of
// [0, 4] (csrc/gen_gelu_fit.py): relative error of Phi(-a) below 1.7e-6 in FP32
// Horner, one hardware exp2 (relative error ~2^-22) per value.  Then GELU(z)
// = z Phi(-a) for z < 0 and z - z Phi(-a) for z >= 0, so the negative tail
// keeps its relative accuracy.  Pairs with |z| > 4 (rare for pre-activations)
// take the erfc form of gelu_tail_f.
constexpr float GELU_FIT_A = 4.0f;
// the fitted form, valid for |z0|, |z1| <= GELU_FIT_A
__device__ __forceinline__ void gelu2_fit(float z0, float z1, float& g0, float& g1) {
  const f32x2 z = f2_pack(z0, z1);
  const f32x2 a = z & f2_splat_bits(0x7FFFFFFFu);
  const f32x2 x = f2_fma(a, f2_splat(0.5f), f2_splat(-1.0f));
  f32x2 q = f2_splat(-0.00023163699370343238f);
  q = f2_fma(q, x, f2_splat(-4.95363783556968e-05f));
  q = f2_fma(q, x, f2_splat(0.0027473631780594587f));
  q = f2_fma(q, x, f2_splat(-0.011412550695240498f));
  q = f2_fma(q, x, f2_splat(0.037877749651670456f));
  q = f2_fma(q, x, f2_splat(-0.11411471664905548f));
  q = f2_fma(q, x, f2_splat(0.3297445476055145f));
  q = f2_fma(q, x, f2_splat(-1.0768771171569824f));
  q = f2_fma(q, x, f2_splat(-2.5725913047790527f));
  const f32x2 e = f2_fma(f2_mul(a, a), f2_splat((float)(-0.5 * 1.4426950408889634)), q);
  float e0, e1, h0, h1;
  f2_unpack(e, e0, e1);
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(h0) : "f"(e0));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(h1) : "f"(e1));
  const f32x2 t = f2_mul(z, f2_pack(h0, h1));       // z Phi(-|z|)
  const f32x2 d = f2_fma(t, f2_splat(-1.0f), z);   // z - z Phi(-|z|)
  float t0, t1, d0, d1;
  f2_unpack(t, t0, t1);
  f2_unpack(d, d0, d1);
  g0 = z0 < 0.0f ? t0 : d0;
  g1 = z1 < 0.0f ? t1 : d1;
}

__device__ __forceinline__ void gelu2_f(float z0, float z1, float& g0, float& g1) {
  if (fmaxf(fabsf(z0), fabsf(z1)) > GELU_FIT_A) {
    g0 = gelu_tail_f(z0);
    g1 = gelu_tail_f(z1);
    return;
  }
  gelu2_fit(z0, z1, g0, g1);
}

// GELU of 2P values in place.  One range test for the whole group, so the
// common case (every |z| <= 4) is straight-line code in which the compiler
// interleaves the P independent pairs; a group with a larger value takes the
// per-pair test.
template <int P>
__device__ __forceinline__ void gelu_group(float (&v)[2 * P]) {
  float amax = 0.0f;
#pragma unroll
  for (int j = 0; j < 2 * P; ++j) amax = fmaxf(amax, fabsf(v[j]));
  if (amax <= GELU_FIT_A) {
#pragma unroll
    for (int j = 0; j < P; ++j) gelu2_fit(v[2 * j], v[2 * j + 1], v[2 * j], v[2 * j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < P; ++j) gelu2_f(v[2 * j], v[2 * j + 1], v[2 * j], v[2 * j + 1]);
  }
}

__device__ __forceinline__ float gelu_f(float z) {
  float g, g1;
  gelu2_f(z, 0.0f, g, g1);
  return g;
}
// GELU'(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float h = half_erfc_scaled(fabsf(z));
  const float Phi = z >= 0.0f ? 1.0f - h : h;
  return Phi + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmParams P) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int A_BYTES = GEMM_BM * GEMM_BK * 2;
  constexpr int B_BYTES = BN * GEMM_BK * 2;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);  // full[S], empty[S], done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tslot;
  const int m0 = blockIdx.y * GEMM_BM, n0 = blockIdx.x * BN;
  const int nk_all = (P.K + GEMM_BK - 1) / GEMM_BK;
  const int nsplit = P.splits > 1 ? P.splits : 1;
  // k-blocks [kb0, kb0 + nk) of this split (the host keeps nsplit <= nk_all)
  const int kb0 = (int)((int64_t)blockIdx.z * nk_all / nsplit);
  const int nk = (int)((int64_t)(blockIdx.z + 1) * nk_all / nsplit) - kb0;
  bool timed_out = false;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1)) {
        timed_out = true;
        break;
      }
      mbar_expect_tx(full0 + 8 * s, A_BYTES + B_BYTES);
      tma_load_2d(smem_u32(sA + s * A_BYTES), &tmA, (kb0 + kb) * GEMM_BK, m0, full0 + 8 * s);
      tma_load_2d(smem_u32(sB + s * B_BYTES), &tmB, (kb0 + kb) * GEMM_BK, n0, full0 + 8 * s);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(GEMM_BM, BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(full0 + 8 * s, ph)) {
        timed_out = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
      for (int kk = 0; kk < GEMM_BK / 16; ++kk) {
        const uint64_t ad = sdesc_sw128(a0 + kk * 32), bd = sdesc_sw128(b0 + kk * 32);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       empty0 + 8 * s)
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                 : "memory");
  }
  __syncwarp();
  // epilogue: warp w owns accumulator rows (TMEM lanes) 32w .. 32w + 31
  const bool ok_done = mbar_wait(done, 0);
  if (!ok_done) timed_out = true;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0 + warp * 32 + lane;
  if (ok_done) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      const uint32_t ta = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
          "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int nb = n0 + c0;
      if (nb >= P.N) continue;
      const bool rok = row < P.M;
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
      if (nsplit > 1) {  // partial sum of this split (bias added by the reduction)
        if (rok) {
          float* o = P.ws + ((size_t)blockIdx.z * P.M + row) * P.N + nb;
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (nb + j < P.N) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        continue;
      }
      if (P.bias) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += (nb + j < P.N) ? P.bias[nb + j] : 0.0f;
      }
      if (P.mode == EPI_F32) {
        if (rok) {
          float* o = P.out0 + (size_t)row * P.ld0 + nb;
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (nb + j < P.N) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
      } else {
        if (P.mode == EPI_TRAIN_FWD && rok) {
          float* o = P.out0 + (size_t)row * P.ld0 + nb;
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (nb + j < P.N) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        if (P.mode == EPI_BWD_DZ) {
          const float* az = P.aux + (size_t)(rok ? row : 0) * P.lda + nb;
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = (rok && nb + j < P.N) ? v[j] * gelu_grad_f(az[j]) : 0.0f;
        } else {
          gelu_group<16>(v);
        }
        __nv_bfloat16 hb[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) hb[j] = __float2bfloat16_rn(v[j]);
        if (P.out1 && rok) {
          __nv_bfloat16* o = P.out1 + (size_t)row * P.ld1 + nb;
#pragma unroll
          for (int j = 0; j < 32; j += 8)
            if (nb + j < P.N) *reinterpret_cast<uint4*>(o + j) = *reinterpret_cast<const uint4*>(hb + j);
        }
        if (P.out2 && rok) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (nb + j < P.N) P.out2[(size_t)(nb + j) * P.ld2 + row] = hb[j];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(BN) : "memory");
  }
  if (timed_out && P.err) atomicExch(P.err, 1);
}

}  // namespace df

namespace df {

// ---------------------------------------------------------------------------
// Persistent variant: one CTA per SM walks the output tiles (tile t = blockIdx.x
// + j * gridDim.x, row-block major so consecutive tiles share their A rows in
// L2).  Ten warps: warp 0 lane 0 issues TMA loads into a STAGES-deep ring,
// warp 1 lane 0 issues tcgen05.mma into one of TWO TMEM accumulators (tile j
// uses buffer j & 1), warps 2..9 drain the other accumulator through the
// epilogue, so the epilogue of tile j overlaps the MMAs of tile j + 1.  A warp
// may only read the TMEM lane quarter (warp % 4), so two epilogue warps share
// each quarter and take alternate 16-column chunks: two warps per SM
// sub-partition hide the latency of the epilogue's loads and transcendentals.
// BN is any multiple of 16 up to 256 (the epilogue reads TMEM 16 columns at
// a time).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// bf16 output staging of the persistent kernel's EPI_GELU_BF16 epilogue: per
// epilogue warp two blocks of 32 rows x 16 columns (1 KB each), stored to
// global memory by TMA (box 16 x 32, no swizzle)
constexpr int PERS_STAGE_C_WARP = 32 * 16 * 2;
__host__ __device__ constexpr int pers_stage_c_bytes(int epi_warps) { return epi_warps * 2 * PERS_STAGE_C_WARP; }
// staging of the training epilogues (EPI_TRAIN_FWD, EPI_BWD_DZ): per epilogue
// warp one block of 32 rows x 16 FP32 columns at a row stride of 20 floats
// (80 bytes: the 16-byte accesses of eight consecutive lanes, one row each or
// two to four lanes per row, fall on distinct bank groups)
constexpr int PERS_STAGE_T_LD = 20;
constexpr int PERS_STAGE_T_WARP = 32 * PERS_STAGE_T_LD * 4;
__host__ __device__ constexpr int pers_epi_bytes(int mode, int epi_warps) {
  return mode == EPI_GELU_BF16 ? pers_stage_c_bytes(epi_warps)
         : (mode == EPI_TRAIN_FWD || mode == EPI_BWD_DZ) ? epi_warps * PERS_STAGE_T_WARP
                                                         : 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// TMA store of a shared-memory block to the 2D tensor at (x = column, y = row);
// elements outside the tensor are not written
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}

// bias + GELU of one 16-column chunk, packed to bf16 pairs (EPI_GELU_BF16)
__device__ __forceinline__ void gemm_gelu_chunk(const GemmParams& P, const uint32_t (&r)[16], int nb,
                                                uint32_t (&hb)[8]) {
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
  if (P.bias) {
    if (nb + 16 <= P.N && (reinterpret_cast<uintptr_t>(P.bias + nb) & 15) == 0) {
      const float4* b4 = reinterpret_cast<const float4*>(P.bias + nb);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 b = __ldg(b4 + q);
        v[4 * q] += b.x;
        v[4 * q + 1] += b.y;
        v[4 * q + 2] += b.z;
        v[4 * q + 3] += b.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += (nb + j < P.N) ? __ldg(P.bias + nb + j) : 0.0f;
    }
  }
  gelu_group<8>(v);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    hb[j] = *reinterpret_cast<const uint32_t*>(&h);
  }
}

// Epilogue of one 16-column chunk of one accumulator row, the mode fixed at
// compile time.  Bias loads are four 16-byte loads (the same address across the
// warp); the per-column bounds tests run only on the ragged last chunk.
template <int MODE>
__device__ __forceinline__ void gemm_epilogue_16(const GemmParams& P, const uint32_t (&r)[16], int row, int nb) {
  if (nb >= P.N) return;
  const bool rok = row < P.M;
  const bool full = nb + 16 <= P.N;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
  if (P.bias) {
    if (full && (reinterpret_cast<uintptr_t>(P.bias + nb) & 15) == 0) {
      const float4* b4 = reinterpret_cast<const float4*>(P.bias + nb);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 b = __ldg(b4 + q);
        v[4 * q] += b.x;
        v[4 * q + 1] += b.y;
        v[4 * q + 2] += b.z;
        v[4 * q + 3] += b.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += (nb + j < P.N) ? __ldg(P.bias + nb + j) : 0.0f;
    }
  }
  if (MODE == EPI_F32 || MODE == EPI_TRAIN_FWD) {
    if (rok) {
      float* o = P.out0 + (size_t)row * P.ld0 + nb;
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        if (full || nb + j < P.N) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
    if (MODE == EPI_F32) return;
  }
  if (MODE == EPI_BWD_DZ) {
    const float* az = P.aux + (size_t)(rok ? row : 0) * P.lda + nb;
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = (rok && (full || nb + j < P.N)) ? v[j] * gelu_grad_f(az[j]) : 0.0f;
  } else {
    gelu_group<8>(v);
  }
  __nv_bfloat162 hb[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) hb[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
  if (P.out1 && rok) {
    __nv_bfloat16* o = P.out1 + (size_t)row * P.ld1 + nb;
    if (full || nb + 8 <= P.N) *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(hb);
    if (full) *reinterpret_cast<uint4*>(o + 8) = *reinterpret_cast<const uint4*>(hb + 4);
  }
  if (MODE != EPI_GELU_BF16 && P.out2 && rok) {
    const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(hb);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (full || nb + j < P.N) P.out2[(size_t)(nb + j) * P.ld2 + row] = h[j];
  }
}

// The training epilogues of the persistent kernel for one 16-column chunk of
// the warp's 32 rows (rows row0 .. row0 + 31, lane l owning row row0 + l in
// TMEM).  Row-major global data moves through the warp's staging block, so a
// warp instruction reads or writes 64-byte (FP32) or 32-byte (BF16) row
// segments of eight or sixteen rows instead of one 16-byte piece of each of 32
// rows: the pre-activation read of EPI_BWD_DZ, the FP32 Z and the BF16 H / dZ
// writes.  The transposed BF16 output is written per lane as before (lanes on
// consecutive rows: each store instruction covers 64 contiguous bytes).  Same
// values and rounding as gemm_epilogue_16.
// EPI_BWD_DZ: the lane's share of a chunk's pre-activation block (rows
// row0 + 8 it + lane / 4, columns nb + 4 (lane % 4) .. + 3; zero outside the
// matrix), loaded one chunk ahead so the global-load latency overlaps the
// previous chunk's arithmetic (the first chunk of a tile: before the wait for
// the tile's accumulator)
__device__ __forceinline__ void bwd_load_aux(const GemmParams& P, int row0, int lane, int nb, float4 (&z)[4]) {
  const int r4 = lane >> 2, c4 = 4 * (lane & 3);
  const bool full = nb + 16 <= P.N;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int gr = row0 + 8 * it + r4;
    z[it] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (gr < P.M && nb < P.N) {
      const float* src = P.aux + (size_t)gr * P.lda + nb + c4;
      if (full && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        z[it] = __ldg(reinterpret_cast<const float4*>(src));
      } else {
        float t[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) t[e] = (nb + c4 + e < P.N) ? __ldg(src + e) : 0.0f;
        z[it] = make_float4(t[0], t[1], t[2], t[3]);
      }
    }
  }
}

template <int MODE>
__device__ __forceinline__ void gemm_epilogue_16_staged(const GemmParams& P, const uint32_t (&r)[16], int row0,
                                                        int lane, int nb, float* stg, const float4 (&za)[4]) {
  static_assert(MODE == EPI_TRAIN_FWD || MODE == EPI_BWD_DZ, "training epilogues only");
  if (nb >= P.N) return;
  const int row = row0 + lane;
  const bool rok = row < P.M;
  const bool full = nb + 16 <= P.N;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
  if (P.bias) {
    if (full && (reinterpret_cast<uintptr_t>(P.bias + nb) & 15) == 0) {
      const float4* b4 = reinterpret_cast<const float4*>(P.bias + nb);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 b = __ldg(b4 + q);
        v[4 * q] += b.x;
        v[4 * q + 1] += b.y;
        v[4 * q + 2] += b.z;
        v[4 * q + 3] += b.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += (nb + j < P.N) ? __ldg(P.bias + nb + j) : 0.0f;
    }
  }
  float* mine = stg + lane * PERS_STAGE_T_LD;
  // lane's place in a row-segment pass: FP32 rows take four lanes (eight rows
  // per pass), BF16 rows two (sixteen rows per pass)
  const int r4 = lane >> 2, c4 = 4 * (lane & 3);
  const int r2 = lane >> 1, h2 = lane & 1;
  __syncwarp();  // the previous chunk's reads of the block are done
  if (MODE == EPI_BWD_DZ) {
#pragma unroll
    for (int it = 0; it < 4; ++it) *reinterpret_cast<float4*>(stg + (8 * it + r4) * PERS_STAGE_T_LD + c4) = za[it];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 z = *reinterpret_cast<const float4*>(mine + 4 * q);
      const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 4 * q + e;
        v[j] = (rok && (full || nb + j < P.N)) ? v[j] * gelu_grad_f(zz[e]) : 0.0f;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(mine + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    __syncwarp();
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int rr = 8 * it + r4, gr = row0 + rr;
      if (gr < P.M) {
        const float4 z = *reinterpret_cast<const float4*>(stg + rr * PERS_STAGE_T_LD + c4);
        float* dst = P.out0 + (size_t)gr * P.ld0 + nb + c4;
        if (full) {
          *reinterpret_cast<float4*>(dst) = z;
        } else {
          const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (nb + c4 + e < P.N) dst[e] = zz[e];
        }
      }
    }
    gelu_group<8>(v);
  }
  __nv_bfloat162 hb[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) hb[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
  if (P.out1) {
    __syncwarp();  // the FP32 reads of the block are done
    uint4* m4 = reinterpret_cast<uint4*>(mine);
    m4[0] = *reinterpret_cast<const uint4*>(hb);
    m4[1] = *reinterpret_cast<const uint4*>(hb + 4);
    __syncwarp();
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int rr = 16 * it + r2, gr = row0 + rr;
      if (gr < P.M) {
        const uint4 val = reinterpret_cast<const uint4*>(stg + rr * PERS_STAGE_T_LD)[h2];
        __nv_bfloat16* dst = P.out1 + (size_t)gr * P.ld1 + nb + 8 * h2;
        if (full) {
          *reinterpret_cast<uint4*>(dst) = val;
        } else {
          const __nv_bfloat16* e8 = reinterpret_cast<const __nv_bfloat16*>(&val);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (nb + 8 * h2 + e < P.N) dst[e] = e8[e];
        }
      }
    }
  }
  if (P.out2 && rok) {
    const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(hb);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (full || nb + j < P.N) P.out2[(size_t)(nb + j) * P.ld2 + row] = h[j];
  }
}

template <int BN>
__host__ __device__ constexpr int tmem_cols_for() {
  return (2 * BN <= 32) ? 32 : (2 * BN <= 64) ? 64 : (2 * BN <= 128) ? 128 : (2 * BN <= 256) ? 256 : 512;
}

// threads of the persistent kernel: TMA warp, MMA warp, EW epilogue warps
__host__ __device__ constexpr int pers_threads(int epi_warps) { return 64 + 32 * epi_warps; }

template <int BN, int STAGES, int MODE, int EW = 8>
__global__ void __launch_bounds__(pers_threads(EW), 1)
    k_gemm_tc_pers(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, GemmParams P) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tile width");
  static_assert(EW % 4 == 0 && EW >= 4 && EW <= 16, "epilogue warps: whole TMEM lane quarters");
  constexpr int EPI_THREADS = 32 * EW;
  constexpr int GROUPS = EW / 4;  // epilogue warps per TMEM lane quarter
  extern __shared__ uint8_t smem_raw[];
  constexpr int A_BYTES = GEMM_BM * GEMM_BK * 2;
  constexpr int B_BYTES = BN * GEMM_BK * 2;
  static_assert(B_BYTES % 1024 == 0, "B tile must keep 1024-byte alignment");
  constexpr int TCOLS = tmem_cols_for<BN>();
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  // EPI_GELU_BF16 output staging: two 32-row x 16-column bf16 blocks per epilogue warp
  uint8_t* sC = sB + STAGES * B_BYTES;
  constexpr int C_BYTES = pers_epi_bytes(MODE, EW);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sC + C_BYTES);  // full[S] empty[S] accf[2] acce[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, EPI_THREADS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    if (MODE == EPI_GELU_BF16)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tslot;
  const int nM = (P.M + GEMM_BM - 1) / GEMM_BM, nN = (P.N + BN - 1) / BN;
  const int ntiles = nM * nN;
  const int nk = (P.K + GEMM_BK - 1) / GEMM_BK;
  bool timed_out = false;

  if (warp == 0) {
    if (lane == 0) {
      int kc = 0;
      for (int t = blockIdx.x; t < ntiles && !timed_out; t += gridDim.x) {
        const int m0 = (t / nN) * GEMM_BM, n0 = (t % nN) * BN;
        for (int kb = 0; kb < nk; ++kb, ++kc) {
          const int s = kc % STAGES;
          const uint32_t ph = (kc / STAGES) & 1;
          if (kc >= STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1)) {
            timed_out = true;
            break;
          }
          mbar_expect_tx(full0 + 8 * s, A_BYTES + B_BYTES);
          tma_load_2d(smem_u32(sA + s * A_BYTES), &tmA, kb * GEMM_BK, m0, full0 + 8 * s);
          tma_load_2d(smem_u32(sB + s * B_BYTES), &tmB, kb * GEMM_BK, n0, full0 + 8 * s);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(GEMM_BM, BN);
      int kc = 0, i = 0;
      for (int t = blockIdx.x; t < ntiles && !timed_out; t += gridDim.x, ++i) {
        const int b = i & 1, u = i >> 1;
        if (u >= 1 && !mbar_wait(acce0 + 8 * b, (u - 1) & 1)) {
          timed_out = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tacc = taddr + (uint32_t)(b * BN);
        for (int kb = 0; kb < nk; ++kb, ++kc) {
          const int s = kc % STAGES;
          const uint32_t ph = (kc / STAGES) & 1;
          if (!mbar_wait(full0 + 8 * s, ph)) {
            timed_out = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
          for (int kk = 0; kk < GEMM_BK / 16; ++kk) {
            const uint64_t ad = sdesc_sw128(a0 + kk * 32), bd = sdesc_sw128(b0 + kk * 32);
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tacc),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           empty0 + 8 * s)
                       : "memory");
        }
        if (timed_out) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         accf0 + 8 * b)
                     : "memory");
      }
    }
  } else {
    // epilogue warps 2 .. EW + 1: TMEM lane quarter warp % 4; the GROUPS warps
    // of a quarter take every GROUPS-th 16-column chunk, from (warp - 2) / 4.
    // The TMEM load of the next chunk is issued before the current chunk is
    // processed, so its latency overlaps the arithmetic.
    const int q = warp & 3;
    const int grp = (warp - 2) >> 2;
    const uint32_t stg0 = smem_u32(sC) + (uint32_t)((warp - 2) * 2 * PERS_STAGE_C_WARP);
    int sbuf = 0;
    int i = 0;
    float4 za[4];  // EPI_BWD_DZ: the next chunk's pre-activation block
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1, u = i >> 1;
      const int m0 = (t / nN) * GEMM_BM, n0 = (t % nN) * BN;
      if (MODE == EPI_BWD_DZ && 16 * grp < BN) bwd_load_aux(P, m0 + q * 32, lane, n0 + 16 * grp, za);
      if (!mbar_wait(accf0 + 8 * b, u & 1)) {
        timed_out = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = m0 + q * 32 + lane;
      const uint32_t tbase = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN);
      uint32_t r[16], rn[16];
      constexpr int CS = 16 * GROUPS;  // column stride of one warp's chunks
      int c0 = 16 * grp;
      if (c0 < BN) {
        tmem_ld16(tbase + (uint32_t)c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      }
#pragma unroll 1
      for (; c0 < BN; c0 += CS) {
        const bool more = c0 + CS < BN;
        if (more) tmem_ld16(tbase + (uint32_t)(c0 + CS), rn);
        if (MODE == EPI_GELU_BF16) {
          if (n0 + c0 < P.N) {
            uint32_t hb[8];
            gemm_gelu_chunk(P, r, n0 + c0, hb);
            const uint32_t dst = stg0 + (uint32_t)(sbuf * PERS_STAGE_C_WARP);
            // the staging block written two chunks ago must have been read out
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            __syncwarp();
            st_shared_v4(dst + lane * 32, hb[0], hb[1], hb[2], hb[3]);
            st_shared_v4(dst + lane * 32 + 16, hb[4], hb[5], hb[6], hb[7]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              tma_store_2d(&tmC, dst, n0 + c0, m0 + q * 32);
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
            sbuf ^= 1;
          }
        } else if (MODE == EPI_TRAIN_FWD || MODE == EPI_BWD_DZ) {
          float* stg = reinterpret_cast<float*>(sC + (warp - 2) * PERS_STAGE_T_WARP);
          float4 zc[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) zc[e] = za[e];
          if (MODE == EPI_BWD_DZ && more) bwd_load_aux(P, m0 + q * 32, lane, n0 + c0 + CS, za);
          gemm_epilogue_16_staged<(MODE == EPI_BWD_DZ) ? EPI_BWD_DZ : EPI_TRAIN_FWD>(P, r, m0 + q * 32, lane,
                                                                                   n0 + c0, stg, zc);
        } else {
          gemm_epilogue_16<MODE>(P, r, row, n0 + c0);
        }
        if (more) {
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) r[j] = rn[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acce0 + 8 * b);
    }
    // the staging blocks must stay valid until the last stores have read them
    if (MODE == EPI_GELU_BF16 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS) : "memory");
  }
  if (timed_out && P.err) atomicExch(P.err, 1);
}

}  // namespace df
