// Device-side definitions shared by the library's kernels and by the kernels
// the library generates and compiles at run time for a loaded mechanism
// (runtime compilation has no C++ standard headers: the few types and macros
// used are provided here).  Mechanism blob: one contiguous FP64 array holding
// the species and reaction data of a mechanism (Sec. 2.3 eq. (reaction):
// nu'_{aj}, nu''_{aj}; Arrhenius K_f; third-body efficiencies; Troe falloff;
// NASA-7 thermo).  The same bytes live in device memory and are staged into
// shared memory by the kernels, so every record has a fixed size and an 8-byte
// alignment.
#pragma once
#ifdef __CUDACC_RTC__
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#ifndef INFINITY
#define INFINITY __longlong_as_double(0x7ff0000000000000ULL)
#endif
#ifndef NAN
#define NAN __longlong_as_double(0x7ff8000000000000ULL)
#endif
// per-cell status codes (the values of include/df_chem.h)
#define DF_CELL_OK 0
#define DF_CELL_MAXSTEPS 1
#define DF_CELL_NONFINITE 2
#define DF_CELL_HMIN 3
#else
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/df_chem.h"
#endif

namespace df {

// physical constants (cgs inside the kernels)
constexpr double RU = 8.314462618e7;         // erg/(mol K)
constexpr double RU_SI = 8.314462618;        // J/(mol K)
constexpr double P_STD = 1.01325e6;          // standard-state pressure, dyn/cm^2
constexpr double LN10 = 2.302585092994045684;
constexpr double LOG_PSTD_RU = -4.4074185890025275;     // ln(P_STD / RU), RU in erg/(mol K)

constexpr int MAX_SPECIES = 64;
constexpr int MAX_REACTIONS = 4096;
constexpr int THREAD_PATH_MAX_N = 16;   // N <= this runs one cell per thread

// --- blob layout (all in doubles) -----------------------------------------
// species record k (SP_REC doubles):   W, 1/W, a1..a7, then the NASA-7
//   coefficients as the enthalpy and entropy polynomials use them:
//   a2/2, a3/3, a4/4, a5/5 (h/RT) and a3/2, a4/3, a5/4 (s/R)
constexpr int SP_REC = 16;
constexpr int SP_H = 9;   // offset of a2/2 .. a5/5
constexpr int SP_S = 13;  // offset of a3/2 .. a5/4
// reaction record j (RX_REC doubles):  lnA, beta, Ea/R, meta0, meta1
//   meta0 (8 bytes): reac[3], prod[3] species indices, nr | np << 4, flags
//     flags: bit0-1 type (0 elementary, 1 third-body, 2 Troe), bit2 reversible
//   meta1 (8 bytes): int32 effslot (-1: none), int32 troeslot (-1: none)
constexpr int RX_REC = 5;
// Troe record (TR_REC doubles): lnA0 - lnA, beta0, Ea0/R, alpha, 1/T***, 1/T*, T**, pad
constexpr int TR_REC = 8;
// efficiency record: N doubles per third-body / falloff reaction

struct RxMeta {
  uint8_t reac[3];
  uint8_t prod[3];
  uint8_t nrnp;
  uint8_t flags;
};
static_assert(sizeof(RxMeta) == 8, "meta layout");
struct RxSlots {
  int32_t eff;
  int32_t troe;
};
static_assert(sizeof(RxSlots) == 8, "slot layout");

struct MechDims {
  int N, M, n_eff, n_troe;
  int off_sp, off_rx, off_tr, off_eff, total;  // offsets in doubles
};

inline MechDims mech_dims(int N, int M, int n_eff, int n_troe) {
  MechDims d;
  d.N = N;
  d.M = M;
  d.n_eff = n_eff;
  d.n_troe = n_troe;
  d.off_sp = 0;
  d.off_rx = d.off_sp + SP_REC * N;
  d.off_tr = d.off_rx + RX_REC * M;
  d.off_eff = d.off_tr + TR_REC * n_troe;
  d.total = d.off_eff + n_eff * N;
  return d;
}

#ifdef __CUDACC__
// 1/a in FP64 from an FP32 seed and two Newton-Raphson steps r <- r (2 - a r)
// (the relative error squares at each step: 2^-22 -> 2^-44 -> rounding): four
// FP64 operations where a correctly rounded division takes a longer sequence
// on the narrow FP64 pipe.  For |a| inside the FP32 normal range (pivots,
// temperatures, densities, heat capacities, step sizes and error scales of the
// integrators); a zero or non-finite a gives a non-finite result.
__device__ __forceinline__ double rcp_nr(double a) {
  float r0f;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"((float)a));
  const double r0 = (double)r0f;
  const double r1 = r0 * fma(-a, r0, 2.0);
  return r1 * fma(-a, r1, 2.0);
}

#endif

}  // namespace df
