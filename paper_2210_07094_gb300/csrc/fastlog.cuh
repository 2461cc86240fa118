// ln(x) in FP64 by a table of 128 reciprocals (the table-driven scheme of
// J.-M. Muller, "Elementary Functions: Algorithms and Implementation",
// table-based reduction):
//   x = 2^m y, y in [1, 2);  j = the top 7 bits of y's fraction;
//   t = y r_j - 1 with r_j ~ 1 / (1 + (j + 1/2)/128), so |t| <= 2^-8;
//   ln x = m ln2 + (-ln r_j) + log1p(t),  log1p(t) = t - t^2/2 + ... + t^7/7
// (the truncated t^8/8 <= 2^-67).  t comes from one fused multiply-add, so it
// carries the relative precision of the product; -ln r_j is a double-double
// evaluated to 60 digits from the stored r_j (gen_logtab.py), ln 2 is split so
// that m * LN2_HI is exact.  The error is within a few ulp of max(1, |ln x|)
// in absolute terms (what the rate expressions need: ln T and log10 of the
// Troe quantities enter as addends).  Zero, negative, subnormal, inf and NaN
// arguments go to the library log().  About 13 FP64 operations.
#pragma once
#include "fastexp.cuh"  // small_int_to_double

namespace df {

struct LogEntry {
  double r, hi, lo;
};

static __device__ const LogEntry g_log_tab[128] = {
#include "fastlog_table.inc"
};

__device__ __forceinline__ double log_tab(double x) {
  const int hi = __double2hiint(x);
  if (hi < 0x00100000 || hi >= 0x7ff00000) return log(x);  // <= 0, subnormal, inf, NaN
  constexpr double LN2_HI = 0x1.62e42fefa3000p-1;
  constexpr double LN2_LO = 0x1.3de6af278ece6p-42;
  const int m = (hi >> 20) - 1023;
  const int j = (hi >> 13) & 127;
  const double y = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));
  const double r = __ldg(&g_log_tab[j].r);
  const double lh = __ldg(&g_log_tab[j].hi);
  const double ll = __ldg(&g_log_tab[j].lo);
  const double t = fma(y, r, -1.0);
  double p = 1.0 / 7.0;
  p = fma(p, t, -1.0 / 6.0);
  p = fma(p, t, 0.2);
  p = fma(p, t, -0.25);
  p = fma(p, t, 1.0 / 3.0);
  p = fma(p, t, -0.5);
  const double lp = fma(p, t * t, t);  // log1p(t)
  const double md = small_int_to_double(m);  // exact, on the integer pipes
  return fma(md, LN2_HI, lh) + (fma(md, LN2_LO, ll) + lp);
}

__device__ __forceinline__ double log10_tab(double x) { return log_tab(x) * 0.43429448190325182765; }

}  // namespace df
