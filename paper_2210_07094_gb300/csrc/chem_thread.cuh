// Device chemistry for the one-cell-per-thread path (N <= 16 species).
//
// Per-thread vectors whose index is a compile-time constant live in registers;
// vectors indexed by a reaction's species (C, wdot, g/RT, h/RT) and the dense
// (N+1)x(N+1) Jacobian / LU live in shared memory in [index][thread] order, so
// that the 32 lanes of a warp touch 32 consecutive doubles (no bank conflicts).
//
// Equations (cgs units inside):
//   rho = p W/(R T),  C_k = rho Y_k / W_k                        (Sec. 2.3)
//   K_f = A T^b exp(-Ea/RT)  (Arrhenius law, Sec. 2.3)
//   K_r = K_f / K_c,  K_c = exp(-sum_k nu_kj g_k/RT) (p_std/RT)^{sum_k nu_kj}
//   third body: rate x [M], [M] = sum_k eps_k C_k
//   Troe: k = k_inf Pr/(1+Pr) F, Pr = k_0 [M]/k_inf,
//         log F = log F_c / (1 + ((log Pr + c)/(n - d (log Pr + c)))^2)
//   q_j = K_f prod C^nu' - K_r prod C^nu''
//   dY_k/dt = W_k sum_j (nu''_kj - nu'_kj) q_j / rho           (eq. (sourceeq))
//   dT/dt = -sum_k H_k wdot_k / (rho cp)   (constant-pressure adiabatic 0D reactor,
//                                           Sec. 2.2 df0DFoam; h conserved)
#pragma once
#include "common.cuh"

namespace df {

// strided view of a per-thread vector in shared memory
struct SV {
  double* p;
  int s;
  __device__ __forceinline__ double& operator[](int i) const { return p[i * s]; }
};

struct MechView {
  const double* sp;
  const double* rx;
  const double* tr;
  const double* eff;
  int M;
};

__device__ __forceinline__ MechView make_view(const double* blob, const MechDims& d) {
  MechView v;
  v.sp = blob + d.off_sp;
  v.rx = blob + d.off_rx;
  v.tr = blob + d.off_tr;
  v.eff = blob + d.off_eff;
  v.M = d.M;
  return v;
}

__device__ __forceinline__ RxMeta load_meta(const double* r) {
  RxMeta m;
  unsigned long long bits = __double_as_longlong(r[3]);
  memcpy(&m, &bits, 8);
  return m;
}
__device__ __forceinline__ RxSlots load_slots(const double* r) {
  RxSlots s;
  unsigned long long bits = __double_as_longlong(r[4]);
  memcpy(&s, &bits, 8);
  return s;
}

// Evaluate f = dy/dt for y = (T, Y) and, when WITH_J, the analytic Jacobian
// J = df/dy (row-major in the strided view Jv, n x n with n = NS + 1).
// Returns qdot = -sum_k H_k wdot_k in erg/(cm^3 s).
template <int NS, bool WITH_J>
__device__ __forceinline__ double eval_thread(const MechView& mv, const double pc, const double (&y)[NS + 1],
                                              double (&f)[NS + 1], SV C, SV wdot, SV gRT, SV hRT, SV cpR,
                                              SV Jv) {
  constexpr int n = NS + 1;
  const double T = y[0];
  const double lnT = log(T);
  const double invT = 1.0 / T;
  double sumYW = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* a = mv.sp + SP_REC * k + 2;
    cpR[k] = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double hk = a[0] + T * (a[1] * 0.5 + T * (a[2] * (1.0 / 3.0) + T * (a[3] * 0.25 + T * a[4] * 0.2))) +
                      a[5] * invT;
    const double sk = a[0] * lnT + T * (a[1] + T * (a[2] * 0.5 + T * (a[3] * (1.0 / 3.0) + T * a[4] * 0.25))) + a[6];
    hRT[k] = hk;
    gRT[k] = hk - sk;
    sumYW += y[1 + k] * mv.sp[SP_REC * k + 1];
  }
  const double rho = pc * invT / (RU * sumYW);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    C[k] = rho * y[1 + k] * mv.sp[SP_REC * k + 1];
    wdot[k] = 0.0;
  }
  if (WITH_J) {
#pragma unroll
    for (int i = 0; i < n * n; ++i) Jv[i] = 0.0;
  }
  const double lnP0RT = LOG_PSTD_RU - lnT;
  for (int j = 0; j < mv.M; ++j) {
    const double* r = mv.rx + RX_REC * j;
    const double lnA = r[0];
    if (lnA == -INFINITY) continue;  // A = 0: no rate
    const double beta = r[1], EaR = r[2];
    const RxMeta mt = load_meta(r);
    const int nr = mt.nrnp & 15, np = mt.nrnp >> 4;
    const int type = mt.flags & 3;
    const bool rev = (mt.flags & 4) != 0;
    const double lnkf = lnA + beta * lnT - EaR * invT;
    // concentration products
    const double cr0 = C[mt.reac[0]];
    const double cr1 = nr > 1 ? C[mt.reac[1]] : 1.0;
    const double cr2 = nr > 2 ? C[mt.reac[2]] : 1.0;
    const double cp0 = C[mt.prod[0]];
    const double cp1 = np > 1 ? C[mt.prod[1]] : 1.0;
    const double cp2 = np > 2 ? C[mt.prod[2]] : 1.0;
    const double Pf = cr0 * cr1 * cr2;
    const double Pb = cp0 * cp1 * cp2;
    // sum_k nu_kj g_k/RT and sum_k nu_kj h_k/RT (products minus reactants)
    double sg = gRT[mt.prod[0]] - gRT[mt.reac[0]];
    double sh = 0.0;
    if (WITH_J) sh = hRT[mt.prod[0]] - hRT[mt.reac[0]];
    if (np > 1) { sg += gRT[mt.prod[1]]; if (WITH_J) sh += hRT[mt.prod[1]]; }
    if (np > 2) { sg += gRT[mt.prod[2]]; if (WITH_J) sh += hRT[mt.prod[2]]; }
    if (nr > 1) { sg -= gRT[mt.reac[1]]; if (WITH_J) sh -= hRT[mt.reac[1]]; }
    if (nr > 2) { sg -= gRT[mt.reac[2]]; if (WITH_J) sh -= hRT[mt.reac[2]]; }
    const int dnu = np - nr;
    const double lnKcinv = sg - dnu * lnP0RT;  // ln(1/K_c)
    double kf, kr, mult = 1.0, dqdM = 0.0, dlnk = 0.0;
    const RxSlots sl = load_slots(r);
    if (type == 2) {
      const double* tr = mv.tr + TR_REC * sl.troe;
      const double* ef = mv.eff + NS * sl.eff;
      double Mc = 0.0;
#pragma unroll
      for (int l = 0; l < NS; ++l) Mc += ef[l] * C[l];
      const double kinf = exp(lnkf);
      const double lnk0 = lnA + tr[0] + tr[1] * lnT - tr[2] * invT;
      const double k0 = exp(lnk0);
      const double Pr = k0 * Mc / kinf;
      if (!(Pr > 0.0)) continue;  // no low-pressure rate or no collider: k = 0
      const double e3 = exp(-T * tr[4]), e1 = exp(-T * tr[5]), e2 = exp(-tr[6] * invT);
      const double Fc = (1.0 - tr[3]) * e3 + tr[3] * e1 + e2;
      const double Lc = log10(Fc);
      const double cc = -0.4 - 0.67 * Lc;
      const double nn = 0.75 - 1.27 * Lc;
      const double L = log10(Pr);
      const double x = L + cc;
      const double den = nn - 0.14 * x;
      const double f1 = x / den;
      const double q1 = 1.0 / (1.0 + f1 * f1);
      const double log10F = Lc * q1;
      const double F = exp(LN10 * log10F);
      const double onePr = 1.0 / (1.0 + Pr);
      kf = kinf * Pr * onePr * F;
      kr = rev ? kf * exp(lnKcinv) : 0.0;
      if (WITH_J) {
        const double df1_dL = nn / (den * den);
        const double df1_dLc = (-0.67 * den - x * (-1.27 + 0.67 * 0.14)) / (den * den);
        const double dlogF_dL = -Lc * 2.0 * f1 * df1_dL * q1 * q1;
        const double dlogF_dLc = q1 - Lc * 2.0 * f1 * df1_dLc * q1 * q1;
        const double g = onePr + dlogF_dL;  // d ln k / d ln Pr
        const double dlnkinf = (beta + EaR * invT) * invT;
        const double dlnk0 = (tr[1] + tr[2] * invT) * invT;
        const double dFc = -(1.0 - tr[3]) * tr[4] * e3 - tr[3] * tr[5] * e1 + tr[6] * invT * invT * e2;
        dlnk = dlnkinf + g * (dlnk0 - dlnkinf) + dlogF_dLc * dFc / Fc;
        // dk/d[M] = k0 F g / (1 + Pr); rate per unit k is (Pf - Pb/K_c)
        dqdM = k0 * F * g * onePr * (Pf - (rev ? Pb * exp(lnKcinv) : 0.0));
      }
    } else {
      kf = exp(lnkf);
      kr = rev ? exp(lnkf + lnKcinv) : 0.0;
      if (type == 1) {
        const double* ef = mv.eff + NS * sl.eff;
        double Mc = 0.0;
#pragma unroll
        for (int l = 0; l < NS; ++l) Mc += ef[l] * C[l];
        mult = Mc;
        dqdM = kf * Pf - kr * Pb;
      }
      if (WITH_J) dlnk = (beta + EaR * invT) * invT;
    }
    const double q = mult * (kf * Pf - kr * Pb);
    wdot[mt.reac[0]] -= q;
    if (nr > 1) wdot[mt.reac[1]] -= q;
    if (nr > 2) wdot[mt.reac[2]] -= q;
    wdot[mt.prod[0]] += q;
    if (np > 1) wdot[mt.prod[1]] += q;
    if (np > 2) wdot[mt.prod[2]] += q;
    if (WITH_J) {
      const double dlnKc = (sh - dnu) * invT;
      const double dqdT = mult * (kf * Pf * dlnk - kr * Pb * (dlnk - dlnKc));
      // d q / d C of each reactant / product entry (product rule, no division)
      const double fk = mult * kf, rk = mult * kr;
      double dr[3], dp[3];
      dr[0] = fk * cr1 * cr2;
      dr[1] = fk * cr0 * cr2;
      dr[2] = fk * cr0 * cr1;
      dp[0] = -rk * cp1 * cp2;
      dp[1] = -rk * cp0 * cp2;
      dp[2] = -rk * cp0 * cp1;
      const double* ef = (type != 0) ? mv.eff + NS * sl.eff : nullptr;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const bool isr = a < 3;
        const int ia = isr ? a : a - 3;
        if (ia >= (isr ? nr : np)) continue;
        const double sgn = isr ? -1.0 : 1.0;
        const int row = 1 + (isr ? mt.reac[ia] : mt.prod[ia]);
        Jv[row * n] += sgn * dqdT;
        Jv[row * n + 1 + mt.reac[0]] += sgn * dr[0];
        if (nr > 1) Jv[row * n + 1 + mt.reac[1]] += sgn * dr[1];
        if (nr > 2) Jv[row * n + 1 + mt.reac[2]] += sgn * dr[2];
        Jv[row * n + 1 + mt.prod[0]] += sgn * dp[0];
        if (np > 1) Jv[row * n + 1 + mt.prod[1]] += sgn * dp[1];
        if (np > 2) Jv[row * n + 1 + mt.prod[2]] += sgn * dp[2];
        if (ef) {
          const double cM = sgn * dqdM;
#pragma unroll
          for (int l = 0; l < NS; ++l) Jv[row * n + 1 + l] += cM * ef[l];
        }
      }
    }
  }
  // mixture cp (mass) and heat release
  double cpm = 0.0, Hw = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    cpm += y[1 + k] * cpR[k] * mv.sp[SP_REC * k + 1];
    Hw += hRT[k] * wdot[k];
  }
  cpm *= RU;
  Hw *= RU * T;
  const double invrho = 1.0 / rho;
  const double invcp = 1.0 / cpm;
#pragma unroll
  for (int k = 0; k < NS; ++k) f[1 + k] = mv.sp[SP_REC * k] * wdot[k] * invrho;
  f[0] = -Hw * invrho * invcp;
  if (WITH_J) {
    // species rows: concentration-space Jc[k][l] = d wdot_k / d C_l (stored in
    // Jv[1+k][1+l]) and dwdot_k/dT at fixed C (Jv[1+k][0]) -> (T, Y) space
    const double Wbar = 1.0 / sumYW;
#pragma unroll 1
    for (int k = 0; k < NS; ++k) {
      const int row = (1 + k) * n;
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < NS; ++l) s += Jv[row + 1 + l] * C[l];
      const double Wk = mv.sp[SP_REC * k];
      const double wk = wdot[k];
      const double a = Wk * Wbar * invrho * (wk - s);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        const double iWi = mv.sp[SP_REC * i + 1];
        Jv[row + 1 + i] = (Wk * Jv[row + 1 + i] + a) * iWi;
      }
      Jv[row] = Wk * invrho * (Jv[row] + (wk - s) * invT);
    }
    // temperature row: f_T = -sum_k h_k f_Yk / cp (h_k specific enthalpy)
    double dcp = 0.0, cpf = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double* a = mv.sp + SP_REC * k + 2;
      const double iW = mv.sp[SP_REC * k + 1];
      dcp += y[1 + k] * (a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]))) * iW;
      cpf += cpR[k] * iW * f[1 + k];
    }
    dcp *= RU;
    cpf *= RU;
#pragma unroll 1
    for (int jc = 0; jc < n; ++jc) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) acc += hRT[k] * mv.sp[SP_REC * k + 1] * Jv[(1 + k) * n + jc];
      acc *= RU * T;
      if (jc == 0) {
        Jv[0] = -invcp * (acc + cpf) - f[0] * dcp * invcp;
      } else {
        const double cpj = RU * cpR[jc - 1] * mv.sp[SP_REC * (jc - 1) + 1];
        Jv[jc] = -invcp * acc - f[0] * cpj * invcp;
      }
    }
  }
  return -Hw;
}

// LU with partial pivoting of the n x n matrix in the strided view A; whole rows
// are swapped, the reciprocal of each pivot replaces the diagonal.  The matrix
// stays in shared memory, so the pivot loop is not unrolled (register budget).
template <int n>
__device__ __forceinline__ bool lu_factor(SV A, int* piv) {
  bool ok = true;
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      const double v = fabs(A[i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    ok = ok && (best > 0.0) && (best < INFINITY);
    if (p != k) {
#pragma unroll
      for (int j = 0; j < n; ++j) {
        const double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    }
    const double inv = 1.0 / A[k * n + k];
    A[k * n + k] = inv;
    for (int i = k + 1; i < n; ++i) {
      const double l = A[i * n + k] * inv;
      A[i * n + k] = l;
#pragma unroll 4
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return ok;
}

// Solve in place on the strided vector x with the factors of lu_factor: the
// whole row permutation first, then the unit-lower and upper solves.
template <int n>
__device__ __forceinline__ void lu_solve(SV A, const int* piv, SV x) {
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    if (p != k) {
      const double t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
  }
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const double xk = x[k];
    for (int i = k + 1; i < n; ++i) x[i] -= A[i * n + k] * xk;
  }
#pragma unroll 1
  for (int k = n - 1; k >= 0; --k) {
    double acc = x[k];
    for (int j = k + 1; j < n; ++j) acc -= A[k * n + j] * x[j];
    x[k] = acc * A[k * n + k];
  }
}

}  // namespace df
