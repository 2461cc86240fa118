// exp(x) in FP64 by the table-driven method of P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989:
//   x = (64 m + j) ln2/64 + r,  |r| <= ln2/128,
//   exp(x) = 2^m * 2^(j/64) * exp(r),  exp(r) - 1 = r + r^2/2 + ... + r^5/120.
// The 64 entries 2^(j/64) are stored as a double-double (hi + lo), each part
// rounded to nearest from a 60-digit decimal evaluation; the evaluation uses
// the leading part (about 1 ulp in all instead of about half of one, one FP64
// operation fewer); the reduction uses ln2/64 split into two doubles with
// fused multiply-adds.  The truncated Taylor tail r^6/720 <= 3.5e-17 stays
// below one ulp.  |x| >= 700, inf and NaN go to
// the library exp().  The kernels stage the table into shared memory (lanes
// index it with different j).  A variant with 256 entries 2^(j/256) (|r| <=
// ln2/512, so exp(r) - 1 needs terms only up to r^4/24, the tail r^5/120 <=
// 3.8e-17) saves one FP64 operation per exponential for 4 KB of shared memory
// per block instead of 1 KB; a translation unit picks it by defining
// DF_EXP_TABLE_BITS as 8 (the kernels generated for a loaded mechanism).
#pragma once

#ifndef DF_EXP_TABLE_BITS
#define DF_EXP_TABLE_BITS 6
#endif

namespace df {

constexpr int EXP_TAB_BITS = DF_EXP_TABLE_BITS;
static_assert(EXP_TAB_BITS == 6 || EXP_TAB_BITS == 8, "exp table: 64 or 256 entries");
constexpr int EXP_TAB_SIZE = 1 << EXP_TAB_BITS;

static __device__ const double2 g_exp2_tab[64] = {
    {0x1.0000000000000p+0, 0x0.0p+0},
    {0x1.02c9a3e778061p+0, -0x1.19083535b085dp-56},
    {0x1.059b0d3158574p+0, 0x1.d73e2a475b465p-55},
    {0x1.0874518759bc8p+0, 0x1.186be4bb284ffp-57},
    {0x1.0b5586cf9890fp+0, 0x1.8a62e4adc610bp-54},
    {0x1.0e3ec32d3d1a2p+0, 0x1.03a1727c57b53p-59},
    {0x1.11301d0125b51p+0, -0x1.6c51039449b3ap-54},
    {0x1.1429aaea92de0p+0, -0x1.32fbf9af1369ep-54},
    {0x1.172b83c7d517bp+0, -0x1.19041b9d78a76p-55},
    {0x1.1a35beb6fcb75p+0, 0x1.e5b4c7b4968e4p-55},
    {0x1.1d4873168b9aap+0, 0x1.e016e00a2643cp-54},
    {0x1.2063b88628cd6p+0, 0x1.dc775814a8495p-55},
    {0x1.2387a6e756238p+0, 0x1.9b07eb6c70573p-54},
    {0x1.26b4565e27cddp+0, 0x1.2bd339940e9d9p-55},
    {0x1.29e9df51fdee1p+0, 0x1.612e8afad1255p-55},
    {0x1.2d285a6e4030bp+0, 0x1.0024754db41d5p-54},
    {0x1.306fe0a31b715p+0, 0x1.6f46ad23182e4p-55},
    {0x1.33c08b26416ffp+0, 0x1.32721843659a6p-54},
    {0x1.371a7373aa9cbp+0, -0x1.63aeabf42eae2p-54},
    {0x1.3a7db34e59ff7p+0, -0x1.5e436d661f5e3p-56},
    {0x1.3dea64c123422p+0, 0x1.ada0911f09ebcp-55},
    {0x1.4160a21f72e2ap+0, -0x1.ef3691c309278p-58},
    {0x1.44e086061892dp+0, 0x1.89b7a04ef80d0p-59},
    {0x1.486a2b5c13cd0p+0, 0x1.3c1a3b69062f0p-56},
    {0x1.4bfdad5362a27p+0, 0x1.d4397afec42e2p-56},
    {0x1.4f9b2769d2ca7p+0, -0x1.4b309d25957e3p-54},
    {0x1.5342b569d4f82p+0, -0x1.07abe1db13cadp-55},
    {0x1.56f4736b527dap+0, 0x1.9bb2c011d93adp-54},
    {0x1.5ab07dd485429p+0, 0x1.6324c054647adp-54},
    {0x1.5e76f15ad2148p+0, 0x1.ba6f93080e65ep-54},
    {0x1.6247eb03a5585p+0, -0x1.383c17e40b497p-54},
    {0x1.6623882552225p+0, -0x1.bb60987591c34p-54},
    {0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54},
    {0x1.6dfb23c651a2fp+0, -0x1.bbe3a683c88abp-57},
    {0x1.71f75e8ec5f74p+0, -0x1.16e4786887a99p-55},
    {0x1.75feb564267c9p+0, -0x1.0245957316dd3p-54},
    {0x1.7a11473eb0187p+0, -0x1.41577ee04992fp-55},
    {0x1.7e2f336cf4e62p+0, 0x1.05d02ba15797ep-56},
    {0x1.82589994cce13p+0, -0x1.d4c1dd41532d8p-54},
    {0x1.868d99b4492edp+0, -0x1.fc6f89bd4f6bap-54},
    {0x1.8ace5422aa0dbp+0, 0x1.6e9f156864b27p-54},
    {0x1.8f1ae99157736p+0, 0x1.5cc13a2e3976cp-55},
    {0x1.93737b0cdc5e5p+0, -0x1.75fc781b57ebcp-57},
    {0x1.97d829fde4e50p+0, -0x1.d185b7c1b85d1p-54},
    {0x1.9c49182a3f090p+0, 0x1.c7c46b071f2bep-56},
    {0x1.a0c667b5de565p+0, -0x1.359495d1cd533p-54},
    {0x1.a5503b23e255dp+0, -0x1.d2f6edb8d41e1p-54},
    {0x1.a9e6b5579fdbfp+0, 0x1.0fac90ef7fd31p-54},
    {0x1.ae89f995ad3adp+0, 0x1.7a1cd345dcc81p-54},
    {0x1.b33a2b84f15fbp+0, -0x1.2805e3084d708p-57},
    {0x1.b7f76f2fb5e47p+0, -0x1.5584f7e54ac3bp-56},
    {0x1.bcc1e904bc1d2p+0, 0x1.23dd07a2d9e84p-55},
    {0x1.c199bdd85529cp+0, 0x1.11065895048ddp-55},
    {0x1.c67f12e57d14bp+0, 0x1.2884dff483cadp-54},
    {0x1.cb720dcef9069p+0, 0x1.503cbd1e949dbp-56},
    {0x1.d072d4a07897cp+0, -0x1.cbc3743797a9cp-54},
    {0x1.d5818dcfba487p+0, 0x1.2ed02d75b3707p-55},
    {0x1.da9e603db3285p+0, 0x1.c2300696db532p-54},
    {0x1.dfc97337b9b5fp+0, -0x1.1a5cd4f184b5cp-54},
    {0x1.e502ee78b3ff6p+0, 0x1.39e8980a9cc8fp-55},
    {0x1.ea4afa2a490dap+0, -0x1.e9c23179c2893p-54},
    {0x1.efa1bee615a27p+0, 0x1.dc7f486a4b6b0p-54},
    {0x1.f50765b6e4540p+0, 0x1.9d3e12dd8a18bp-54},
    {0x1.fa7c1819e90d8p+0, 0x1.74853f3a5931ep-55},
};

// (double)v for |v| < 2^20, assembled from the integer's sign, leading one and
// the bits below it with integer operations, so that the conversion takes no
// slot of the narrow FP64 pipe (exact: every such integer is a double)
__device__ __forceinline__ double small_int_to_double(int v) {
  const unsigned a = (unsigned)(v < 0 ? -v : v);
  const int lz = __clz(a | 1u);                  // the leading one of a > 0 at bit 31 - lz
  const unsigned mant = ((a << lz) << 1) >> 12;  // the (at most 19) bits below it, left-aligned
  const unsigned hi = ((unsigned)(v < 0) << 31) | ((unsigned)(1023 + 31 - lz) << 20) | mant;
  return __hiloint2double(a != 0u ? (int)hi : 0, 0);
}

// 2^(j/256) as double-doubles (gen_exptab.py, 60-digit evaluation)
static __device__ const double2 g_exp2_tab256[256] = {
#include "fastexp_table256.inc"
};

// the table the kernels of this translation unit stage into shared memory
__device__ __forceinline__ const double2* exp_table_src() { return EXP_TAB_BITS == 8 ? g_exp2_tab256 : g_exp2_tab; }

// the reduction and polynomial of exp_tang for |x| < 700 (no range guard), with
// a table of 2^B entries
template <int B>
__device__ __forceinline__ double exp_tang_core_b(double x, const double2* tab) {
  static_assert(B == 6 || B == 8, "exp table: 64 or 256 entries");
  const double SHIFT = 0x1.8p52;                 // 1.5 * 2^52: round-to-integer shifter
  // 2^B / ln 2, and ln 2 / 2^B in a leading and a trailing part
  const double INV_L = B == 8 ? 0x1.71547652b82fep+8 : 0x1.71547652b82fep+6;
  const double L1 = B == 8 ? 0x1.62e42fefa39efp-9 : 0x1.62e42fefa39efp-7;
  const double L2 = B == 8 ? 0x1.abc9e3b39803fp-64 : 0x1.abc9e3b39803fp-62;
  const double t = fma(x, INV_L, SHIFT);
  const int k = __double2loint(t);               // t = SHIFT + k exactly; |k| < 2^18
  const double kd = small_int_to_double(k);      // = t - SHIFT, without an FP64 subtraction
  double r = fma(-kd, L1, x);
  r = fma(-kd, L2, r);
  const int j = k & ((1 << B) - 1);
  const int m = k >> B;
  const double r2 = r * r;
  double q;
  if (B == 8) {
    q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  } else {
    q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
  }
  q = fma(q, r, 0.5);
  const double p = fma(q, r2, r);                // exp(r) - 1
  // 2^(j/2^B) exp(r) = t + t p with t the table's leading double alone: one
  // rounding more than with its trailing part (about 1 ulp in all, within the
  // 2 ulp the tests allow) for one FP64 operation less
  const double tj = tab[j].x;
  const double s = fma(tj, p, tj);
  return __hiloint2double(__double2hiint(s) + (int)((unsigned)m << 20), __double2loint(s));
}

__device__ __forceinline__ double exp_tang_core(double x, const double2* tab) {
  return exp_tang_core_b<EXP_TAB_BITS>(x, tab);
}

// exp of two arguments at once: both reductions and polynomials in one
// straight-line block (two independent dependency chains for the scheduler),
// the rare |x| >= 700 / inf / NaN cases fixed up afterwards
__device__ __forceinline__ void exp_tang2(double x1, double x2, const double2* tab, double& e1, double& e2) {
  const bool big1 = (__double2hiint(x1) & 0x7fffffff) >= 0x4085E000;
  const bool big2 = (__double2hiint(x2) & 0x7fffffff) >= 0x4085E000;
  e1 = exp_tang_core(big1 ? 0.0 : x1, tab);
  e2 = exp_tang_core(big2 ? 0.0 : x2, tab);
  if (big1 | big2) {
    if (big1) e1 = exp(x1);
    if (big2) e2 = exp(x2);
  }
}

template <int B>
__device__ __forceinline__ double exp_tang_b(double x, const double2* tab) {
  // |x| >= 700, inf and NaN, tested on the high word with integer operations
  // (0x4085E000 is the high word of 700.0; the low word of 700.0 is zero), so
  // the narrow FP64 pipe is not spent on the guard
  if ((__double2hiint(x) & 0x7fffffff) >= 0x4085E000) return exp(x);
  return exp_tang_core_b<B>(x, tab);
}

__device__ __forceinline__ double exp_tang(double x, const double2* tab) { return exp_tang_b<EXP_TAB_BITS>(x, tab); }

}  // namespace df
