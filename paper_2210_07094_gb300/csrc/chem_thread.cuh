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
#include "dev_common.cuh"
#include "fastexp.cuh"
#include "fastlog.cuh"
#include "dual.cuh"

namespace df {

// ln and log10 of the rate expressions by the table-driven logarithm (the
// dual-number versions carry the derivative d/x)
__device__ __forceinline__ double fast_log(double x) { return log_tab(x); }
__device__ __forceinline__ Dual fast_log(const Dual& x) { return Dual(log_tab(x.v), x.d / x.v); }
__device__ __forceinline__ double fast_log10(double x) { return log10_tab(x); }
__device__ __forceinline__ Dual fast_log10(const Dual& x) {
  return Dual(log10_tab(x.v), x.d / (x.v * 2.302585092994045684));
}

// strided view of a per-thread vector (any scalar type) in shared memory; a
// stride fixed at compile time (ST > 0, the block size) turns the address of
// every constant index into an immediate offset
template <class S, int ST = 0>
struct SVT {
  S* p;
  int s;
  __device__ __forceinline__ S& operator[](int i) const { return p[i * (ST > 0 ? ST : s)]; }
};
typedef SVT<double> SV;

struct MechView {
  const double* sp;
  const double* rx;
  const double* tr;
  const double* eff;
  const double2* etab;  // 2^(j/64) table of exp_tang (shared memory)
  int M;
};

__device__ __forceinline__ MechView make_view(const double* blob, const MechDims& d, const double2* etab) {
  MechView v;
  v.etab = etab;
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

// exp of two arguments (two independent dependency chains for the scheduler)
__device__ __forceinline__ void exp_pair(double a, double b, const double2* tab, double& ea, double& eb) {
  exp_tang2(a, b, tab, ea, eb);
}
__device__ __forceinline__ void exp_pair(const Dual& a, const Dual& b, const double2* tab, Dual& ea, Dual& eb) {
  ea = exp_tang(a, tab);
  eb = exp_tang(b, tab);
}

// Result of the rate of one reaction; with J also the pieces of dq/dT|_C and
// dq/dC.
template <class S>
struct RateOutT {
  bool active;
  RxMeta mt;
  RxSlots sl;
  S q;       // net rate [mol/cm^3/s]
  S fk, rk;  // effective forward / reverse coefficients (x [M] for third body)
  S dqdT;    // dq/dT at fixed C
  S dqdM;    // dq/d[M] (third body, Troe); multiplies eps_l for dq/dC_l
  S cr[3], cp[3];
};
typedef RateOutT<double> RateOut;

// Everything rate_one reads from memory for reaction j: its record, the
// concentrations of its species, sum_k nu_kj g_k/RT (and h_k/RT with J) and,
// for a third-body or falloff reaction, [M] = sum_l eps_l C_l.  Gathering the
// next reaction's inputs before the current reaction's production rates are
// stored keeps the shared-memory loads off the FP64 dependency chain (the
// concentrations and g/RT do not change during the reaction loop).
template <class S>
struct RxIn {
  double lnA, beta, EaR;
  RxMeta mt;
  RxSlots sl;
  S cr[3], cp[3];  // reactant / product concentrations (1 where absent)
  S sg, sh;        // sum nu g/RT, sum nu h/RT (products minus reactants)
  S Mc;            // [M] (third body, falloff)
};

// Third-body efficiencies as a sum of all concentrations plus sparse
// corrections: [M] = ctot + sum over the species l whose efficiency is not 1 of
// (eps_l - 1) C_l.  off[s] .. off[s + 1] index the (l, low word, high word)
// triples of efficiency slot s in ent (the correction eps_l - 1 as the two
// 32-bit halves of a double).
struct SparseEff {
  const int* off;
  const int* ent;
  double ctot;
};

template <int NS, bool WITH_J, class S, class Vec>
__device__ __forceinline__ void rate_gather(const MechView& mv, const double* r, int Nrt, const Vec& C,
                                            const Vec& gRT, const Vec& hRT, RxIn<S>& g,
                                            const SparseEff* se = nullptr) {
  const int N = NS > 0 ? NS : Nrt;
  g.lnA = r[0];
  g.beta = r[1];
  g.EaR = r[2];
  g.mt = load_meta(r);
  g.sl = load_slots(r);
  const RxMeta mt = g.mt;
  const int nr = mt.nrnp & 15, np = mt.nrnp >> 4;
  const S one(1.0);
  g.cr[0] = C[mt.reac[0]];
  g.cr[1] = nr > 1 ? S(C[mt.reac[1]]) : one;
  g.cr[2] = nr > 2 ? S(C[mt.reac[2]]) : one;
  g.cp[0] = C[mt.prod[0]];
  g.cp[1] = np > 1 ? S(C[mt.prod[1]]) : one;
  g.cp[2] = np > 2 ? S(C[mt.prod[2]]) : one;
  S sg = gRT[mt.prod[0]] - gRT[mt.reac[0]];
  S sh(0.0);
  if (WITH_J) sh = hRT[mt.prod[0]] - hRT[mt.reac[0]];
  if (np > 1) { sg += gRT[mt.prod[1]]; if (WITH_J) sh += hRT[mt.prod[1]]; }
  if (np > 2) { sg += gRT[mt.prod[2]]; if (WITH_J) sh += hRT[mt.prod[2]]; }
  if (nr > 1) { sg -= gRT[mt.reac[1]]; if (WITH_J) sh -= hRT[mt.reac[1]]; }
  if (nr > 2) { sg -= gRT[mt.reac[2]]; if (WITH_J) sh -= hRT[mt.reac[2]]; }
  g.sg = sg;
  g.sh = sh;
  g.Mc = S(0.0);
  if ((mt.flags & 3) != 0) {
    if (se) {
      S Mc(se->ctot);
      for (int t = se->off[g.sl.eff]; t < se->off[g.sl.eff + 1]; ++t) {
        const int* e = se->ent + 3 * t;
        Mc += __hiloint2double(e[2], e[1]) * C[e[0]];
      }
      g.Mc = Mc;
    } else {
      const double* ef = mv.eff + N * g.sl.eff;
      S Mc(0.0);
#pragma unroll
      for (int l = 0; l < N; ++l) Mc += ef[l] * C[l];
      g.Mc = Mc;
    }
  }
}

// The rate of one reaction from its gathered inputs: Arrhenius K_f, K_r = K_f/K_c,
// third-body [M] and Troe falloff; with WITH_J also dq/dT at fixed C and dq/d[M].
template <int NS, bool WITH_J, class S>
__device__ __forceinline__ void rate_compute(const MechView& mv, const RxIn<S>& g, S T, S lnT, S invT,
                                             S lnP0RT, RateOutT<S>& o) {
  o.active = false;
  const double lnA = g.lnA;
  if (lnA == -INFINITY) return;  // A = 0: no rate
  const double beta = g.beta, EaR = g.EaR;
  const RxMeta mt = g.mt;
  o.mt = mt;
  const int nr = mt.nrnp & 15, np = mt.nrnp >> 4;
  const int type = mt.flags & 3;
  const bool rev = (mt.flags & 4) != 0;
  const S lnkf = lnA + beta * lnT - EaR * invT;
  o.cr[0] = g.cr[0]; o.cr[1] = g.cr[1]; o.cr[2] = g.cr[2];
  o.cp[0] = g.cp[0]; o.cp[1] = g.cp[1]; o.cp[2] = g.cp[2];
  const S Pf = g.cr[0] * g.cr[1] * g.cr[2];
  const S Pb = g.cp[0] * g.cp[1] * g.cp[2];
  const S sg = g.sg, sh = g.sh;
  const int dnu = np - nr;
  // ln(1/K_c); a reaction that keeps its mole count has no pressure term (no
  // operation where the counts are known at compile time, as in the kernels
  // generated for a mechanism; the same value either way)
  const S lnKcinv = dnu == 0 ? sg : sg - (double)dnu * lnP0RT;
  S kf, kr, mult(1.0), dqdM(0.0), dlnk(0.0);
  const RxSlots sl = g.sl;
  o.sl = sl;
  if (type == 2) {
    const double* tr = mv.tr + TR_REC * sl.troe;
    const S Mc = g.Mc;
    const S lnk0 = lnA + tr[0] + tr[1] * lnT - tr[2] * invT;
    // Pr = k0 [M] / kinf, as exp(ln k0 - ln kinf) [M] (no division); the
    // exponentials in pairs (see exp_pair)
    S kinf, r0, e3, e1, e2, invKc;
    exp_pair(lnkf, lnk0 - lnkf, mv.etab, kinf, r0);
    const S Pr = r0 * Mc;
    if (!(val(Pr) > 0.0)) return;  // no low-pressure rate or no collider: k = 0
    exp_pair(-T * tr[4], -T * tr[5], mv.etab, e3, e1);
    exp_pair(-tr[6] * invT, lnKcinv, mv.etab, e2, invKc);
    if (!rev) invKc = S(0.0);
    const S Fc = (1.0 - tr[3]) * e3 + tr[3] * e1 + e2;
    const S Lc = fast_log10(Fc);
    const S cc = -0.4 - 0.67 * Lc;
    const S nn = 0.75 - 1.27 * Lc;
    const S L = fast_log10(Pr);
    const S x = L + cc;
    const S den = nn - 0.14 * x;
    // 1 / (1 + (x / den)^2) with one division
    const S den2 = den * den;
    const S q1 = den2 / (den2 + x * x);
    const S log10F = Lc * q1;
    const S F = exp_tang(LN10 * log10F, mv.etab);
    const S onePr = 1.0 / (1.0 + Pr);
    kf = kinf * Pr * onePr * F;
    kr = kf * invKc;
    if (WITH_J) {
      const S k0 = exp_tang(lnk0, mv.etab);
      const S f1 = x / den;
      const S df1_dL = nn / (den * den);
      const S df1_dLc = (-0.67 * den - x * (-1.27 + 0.67 * 0.14)) / (den * den);
      const S dlogF_dL = -2.0 * Lc * f1 * df1_dL * q1 * q1;
      const S dlogF_dLc = q1 - 2.0 * Lc * f1 * df1_dLc * q1 * q1;
      const S gpr = onePr + dlogF_dL;  // d ln k / d ln Pr
      const S dlnkinf = (beta + EaR * invT) * invT;
      const S dlnk0 = (tr[1] + tr[2] * invT) * invT;
      const S dFc = -(1.0 - tr[3]) * tr[4] * e3 - tr[3] * tr[5] * e1 + tr[6] * invT * invT * e2;
      dlnk = dlnkinf + gpr * (dlnk0 - dlnkinf) + dlogF_dLc * dFc / Fc;
      // dk/d[M] = k0 F gpr / (1 + Pr); rate per unit k is (Pf - Pb/K_c)
      dqdM = k0 * F * gpr * onePr * (Pf - Pb * invKc);
    }
  } else {
    exp_pair(lnkf, lnkf + lnKcinv, mv.etab, kf, kr);
    if (!rev) kr = S(0.0);
    if (type == 1) {
      mult = g.Mc;
      dqdM = kf * Pf - kr * Pb;
    }
    if (WITH_J) dlnk = (beta + EaR * invT) * invT;
  }
  o.active = true;
  o.q = mult * (kf * Pf - kr * Pb);
  o.fk = mult * kf;
  o.rk = mult * kr;
  o.dqdM = dqdM;
  if (WITH_J) {
    const S dlnKc = (sh - (double)dnu) * invT;
    o.dqdT = mult * (kf * Pf * dlnk - kr * Pb * (dlnk - dlnKc));
  } else {
    o.dqdT = S(0.0);
  }
}


// Rate of one reaction (Sec. 2.3 eq. (sourceeq) bracket, with the Arrhenius
// K_f, K_r = K_f/K_c, third-body [M] and Troe falloff) at temperature T and
// concentrations C: rate_gather then rate_compute.  S is the scalar type
// (double, or Dual for directional derivatives); Vec is any indexable vector of
// S.  NS > 0 fixes the species count at compile time; otherwise Nrt is used.
template <int NS, bool WITH_J, class S, class Vec>
__device__ __forceinline__ void rate_one(const MechView& mv, const double* r, int Nrt, S T, S lnT, S invT,
                                         S lnP0RT, const Vec& C, const Vec& gRT, const Vec& hRT,
                                         RateOutT<S>& o, const SparseEff* se = nullptr) {
  RxIn<S> g;
  rate_gather<NS, WITH_J>(mv, r, Nrt, C, gRT, hRT, g, se);
  rate_compute<NS, WITH_J>(mv, g, T, lnT, invT, lnP0RT, o);
}

// Optional accumulation of d/d ln A_j of a weighted sum of the right-hand side
// (the discrete adjoint's parameter gradient), inside eval_vjp.  Mode 1: the
// weights are eval_vjp's cotangent r of dy/dt, i.e. th[j] += r . d f / d ln A_j
// = q_j sum_k nu_kj u_k with u_k = (W_k r_{Y_k} - r_T H_k / cp) / rho.  Mode 2:
// heat release, th[j] += g * d qdot / d ln A_j with qdot = -0.1 sum_k H_k wdot_k
// [W/m^3].  With a Dual scalar only the derivative part is accumulated, or,
// with both set, the value part and then the derivative part (a Dual
// evaluation that also stands in for the double one at the same point).  The
// scratch u may be the storage of eval_vjp's cpR vector: eval_vjp reads u only
// in its reaction loop and writes cpR after it.
struct ThetaHook {
  int mode;        // 0: off
  double g;        // mode 2: weight
  SV th;           // per-thread accumulator, M entries
  SV u;            // per-thread scratch, N entries (double evaluation)
  SVT<Dual> uD;    // per-thread scratch, N entries (Dual evaluation)
  int both = 0;    // Dual evaluation: accumulate the value part too
};

__device__ __forceinline__ void th_add(const ThetaHook& h, int j, double x) { h.th[j] += x; }
__device__ __forceinline__ void th_add(const ThetaHook& h, int j, const Dual& x) {
  if (h.both) h.th[j] += x.v;
  h.th[j] += x.d;
}
__device__ __forceinline__ void u_store(const ThetaHook& h, int k, double x) { h.u[k] = x; }
__device__ __forceinline__ void u_store(const ThetaHook& h, int k, const Dual& x) { h.uD[k] = x; }
__device__ __forceinline__ double u_load(const ThetaHook& h, int k, double) { return h.u[k]; }
__device__ __forceinline__ Dual u_load(const ThetaHook& h, int k, const Dual&) { return h.uD[k]; }

// Evaluate f = dy/dt for y = (T, Y) and, when WITH_J, the analytic Jacobian
// J = df/dy (row-major in the strided view Jv, n x n with n = NS + 1).
// Constant-pressure reactor (CONSTV false): pc is the pressure [dyn/cm^2], rho
// follows from the ideal-gas law, and the energy balance conserves h.
// Constant-volume reactor (Sec. 2.2, CONSTV true): pc is the fixed density
// [g/cm^3]; U_k = H_k - R T and cv = cp - R/W replace H_k and cp in the
// temperature equation, and C_k = rho Y_k / W_k no longer depends on T or on
// the mean molar mass.  Returns qdot = -sum_k H_k wdot_k (U_k at constant
// volume) in erg/(cm^3 s).
template <int NS, bool WITH_J, class S = double, bool CONSTV = false, int ST = 0>
__device__ __forceinline__ S eval_thread(const MechView& mv, const double pc, const S (&y)[NS + 1], S (&f)[NS + 1],
                                         SVT<S, ST> C, SVT<S, ST> wdot, SVT<S, ST> gRT, SVT<S, ST> hRT,
                                         SVT<S, ST> cpR, SVT<S, ST> Jv) {
  constexpr int n = NS + 1;
  constexpr double EV = CONSTV ? 1.0 : 0.0;  // U/(RT) = H/(RT) - 1, cv/R = cp/R - 1
  const S T = y[0];
  const S lnT = fast_log(T);
  const S invT = 1.0 / T;
  S sumYW(0.0), cpm(0.0);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* a = mv.sp + SP_REC * k + 2;
    const double* ah = mv.sp + SP_REC * k + SP_H;  // a2/2 .. a5/5
    const double* as = mv.sp + SP_REC * k + SP_S;  // a3/2 .. a5/4
    const S cpk = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    cpR[k] = cpk;
    const S hk = a[0] + T * (ah[0] + T * (ah[1] + T * (ah[2] + T * ah[3]))) + a[5] * invT;
    const S sk = a[0] * lnT + T * (a[1] + T * (as[0] + T * (as[1] + T * as[2]))) + a[6];
    hRT[k] = hk;
    gRT[k] = hk - sk;
    sumYW += y[1 + k] * mv.sp[SP_REC * k + 1];
    cpm += y[1 + k] * (cpk - EV) * mv.sp[SP_REC * k + 1];
  }
  cpm = cpm * RU;  // cp, or cv at constant volume
  const S rho = CONSTV ? S(pc) : pc * invT / (RU * sumYW);
  const S invrho = 1.0 / rho;
  const S invcp = 1.0 / cpm;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    C[k] = rho * y[1 + k] * mv.sp[SP_REC * k + 1];
    wdot[k] = S(0.0);
  }
  if (WITH_J) {
#pragma unroll
    for (int i = 0; i < n * n; ++i) Jv[i] = S(0.0);
  }
  const S lnP0RT = LOG_PSTD_RU - lnT;
  for (int j = 0; j < mv.M; ++j) {
    RateOutT<S> ro;
    rate_one<NS, WITH_J>(mv, mv.rx + RX_REC * j, NS, T, lnT, invT, lnP0RT, C, gRT, hRT, ro);
    if (!ro.active) continue;
    const RxMeta mt = ro.mt;
    const int nr = mt.nrnp & 15, np = mt.nrnp >> 4;
    const S q = ro.q;
    wdot[mt.reac[0]] -= q;
    if (nr > 1) wdot[mt.reac[1]] -= q;
    if (nr > 2) wdot[mt.reac[2]] -= q;
    wdot[mt.prod[0]] += q;
    if (np > 1) wdot[mt.prod[1]] += q;
    if (np > 2) wdot[mt.prod[2]] += q;
    if (WITH_J) {
      // d q / d C of each reactant / product entry (product rule, no division)
      S dr[3], dp[3];
      dr[0] = ro.fk * ro.cr[1] * ro.cr[2];
      dr[1] = ro.fk * ro.cr[0] * ro.cr[2];
      dr[2] = ro.fk * ro.cr[0] * ro.cr[1];
      dp[0] = -(ro.rk * ro.cp[1] * ro.cp[2]);
      dp[1] = -(ro.rk * ro.cp[0] * ro.cp[2]);
      dp[2] = -(ro.rk * ro.cp[0] * ro.cp[1]);
      const int type = mt.flags & 3;
      const double* ef = (type != 0) ? mv.eff + NS * ro.sl.eff : nullptr;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const bool isr = a < 3;
        const int ia = isr ? a : a - 3;
        if (ia >= (isr ? nr : np)) continue;
        const double sgn = isr ? -1.0 : 1.0;
        const int row = 1 + (isr ? mt.reac[ia] : mt.prod[ia]);
        Jv[row * n] += sgn * ro.dqdT;
        Jv[row * n + 1 + mt.reac[0]] += sgn * dr[0];
        if (nr > 1) Jv[row * n + 1 + mt.reac[1]] += sgn * dr[1];
        if (nr > 2) Jv[row * n + 1 + mt.reac[2]] += sgn * dr[2];
        Jv[row * n + 1 + mt.prod[0]] += sgn * dp[0];
        if (np > 1) Jv[row * n + 1 + mt.prod[1]] += sgn * dp[1];
        if (np > 2) Jv[row * n + 1 + mt.prod[2]] += sgn * dp[2];
        if (ef) {
          const S cM = sgn * ro.dqdM;
#pragma unroll
          for (int l = 0; l < NS; ++l) Jv[row * n + 1 + l] += cM * ef[l];
        }
      }
    }
  }
  // heat release
  S Hw(0.0);
#pragma unroll
  for (int k = 0; k < NS; ++k) Hw += (hRT[k] - EV) * wdot[k];
  Hw = Hw * (RU * T);
#pragma unroll
  for (int k = 0; k < NS; ++k) f[1 + k] = mv.sp[SP_REC * k] * wdot[k] * invrho;
  f[0] = -(Hw * invrho * invcp);
  if (WITH_J) {
    // species rows: concentration-space Jc[k][l] = d wdot_k / d C_l (stored in
    // Jv[1+k][1+l]) and dwdot_k/dT at fixed C (Jv[1+k][0]) -> (T, Y) space.
    // At constant pressure C also moves with T and with the mean molar mass;
    // at constant volume it does not.
    const S Wbar = 1.0 / sumYW;
#pragma unroll 1
    for (int k = 0; k < NS; ++k) {
      const int row = (1 + k) * n;
      const double Wk = mv.sp[SP_REC * k];
      if (CONSTV) {
#pragma unroll
        for (int i = 0; i < NS; ++i) Jv[row + 1 + i] = Wk * Jv[row + 1 + i] * mv.sp[SP_REC * i + 1];
        Jv[row] = Wk * invrho * Jv[row];
      } else {
        S s(0.0);
#pragma unroll
        for (int l = 0; l < NS; ++l) s += Jv[row + 1 + l] * C[l];
        const S wk = wdot[k];
        const S a = Wk * Wbar * invrho * (wk - s);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          const double iWi = mv.sp[SP_REC * i + 1];
          Jv[row + 1 + i] = (Wk * Jv[row + 1 + i] + a) * iWi;
        }
        Jv[row] = Wk * invrho * (Jv[row] + (wk - s) * invT);
      }
    }
    // temperature row: f_T = -sum_k e_k f_Yk / c with e_k the specific enthalpy
    // (internal energy) and c = cp (cv)
    S dcp(0.0), cpf(0.0);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double* a = mv.sp + SP_REC * k + 2;
      const double iW = mv.sp[SP_REC * k + 1];
      dcp += y[1 + k] * (a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]))) * iW;
      cpf += (cpR[k] - EV) * iW * f[1 + k];
    }
    dcp = dcp * RU;
    cpf = cpf * RU;
#pragma unroll 1
    for (int jc = 0; jc < n; ++jc) {
      S acc(0.0);
#pragma unroll
      for (int k = 0; k < NS; ++k) acc += (hRT[k] - EV) * mv.sp[SP_REC * k + 1] * Jv[(1 + k) * n + jc];
      acc = acc * (RU * T);
      if (jc == 0) {
        Jv[0] = -(invcp * (acc + cpf)) - f[0] * dcp * invcp;
      } else {
        const double iWj = mv.sp[SP_REC * (jc - 1) + 1];
        const S cpj = RU * (cpR[jc - 1] - EV) * iWj;
        Jv[jc] = -(invcp * acc) - f[0] * cpj * invcp;
      }
    }
  }
  return -Hw;
}

// b = J(y)^T r for a fixed vector r, without forming J: the transpose of the
// assembly in eval_thread, accumulated reaction by reaction (reverse mode).
// With rho_k = r_{1+k} + r_0 c_k, c_k = -R T h_k/(RT) / (W_k cp) the weight of
// species row k in the temperature row, and sigma_k = W_k rho_k:
//   v_i = sum_k sigma_k dwdot_k/dC_i,   v_T = sum_k sigma_k dwdot_k/dT|_C
// (each reaction adds w_j dq_j/dC_i and w_j dq_j/dT, w_j = sum over its
// products of sigma minus sum over its reactants), D = sum_k sigma_k wdot_k -
// sum_l v_l C_l, and then
//   b_T     = (v_T + D / T) / rho + r_0 e_T
//   b_{Y_i} = (v_i + D Wbar / rho) / W_i + r_0 e_i
// with e the temperature row's own terms (e_T = -(cpf + f_T dcp/dT) / cp,
// e_i = -f_T cp_i / cp).  Also returns f = dy/dt (f may alias nothing) and, with
// a hook, its ln A terms.  sig and v are N-entry scratch vectors; cpR receives
// cp_k/R after the reaction loop (the hook's u, ud may share its storage).
template <int NS, class S = double>
__device__ __forceinline__ void eval_vjp(const MechView& mv, const double pc, const S (&y)[NS + 1],
                                         const double (&r)[NS + 1], S (&b)[NS + 1], S (&f)[NS + 1], SVT<S> C,
                                         SVT<S> wdot, SVT<S> gRT, SVT<S> hRT, SVT<S> cpR, SVT<S> sig, SVT<S> v,
                                         const ThetaHook* hook = nullptr) {
  const S T = y[0];
  const S lnT = fast_log(T);
  const S invT = 1.0 / T;
  S sumYW(0.0), cpm(0.0);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* a = mv.sp + SP_REC * k + 2;
    const S cpk = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double* ah = mv.sp + SP_REC * k + SP_H;  // a2/2 .. a5/5
    const double* as = mv.sp + SP_REC * k + SP_S;  // a3/2 .. a5/4
    const S hk = a[0] + T * (ah[0] + T * (ah[1] + T * (ah[2] + T * ah[3]))) + a[5] * invT;
    const S sk = a[0] * lnT + T * (a[1] + T * (as[0] + T * (as[1] + T * as[2]))) + a[6];
    hRT[k] = hk;
    gRT[k] = hk - sk;
    sumYW += y[1 + k] * mv.sp[SP_REC * k + 1];
    cpm += y[1 + k] * cpk * mv.sp[SP_REC * k + 1];
  }
  cpm = cpm * RU;
  const S rho = pc * invT / (RU * sumYW);
  const S invrho = 1.0 / rho;
  const S invcp = 1.0 / cpm;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    C[k] = rho * y[1 + k] * mv.sp[SP_REC * k + 1];
    wdot[k] = S(0.0);
    v[k] = S(0.0);
    const S ck = -(invcp * (RU * T) * hRT[k] * mv.sp[SP_REC * k + 1]);
    sig[k] = mv.sp[SP_REC * k] * (r[1 + k] + r[0] * ck);
  }
  if (hook && hook->mode) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const S Hk = RU * T * hRT[k];
      S uk;
      if (hook->mode == 1) uk = (mv.sp[SP_REC * k] * r[1 + k] - r[0] * Hk * invcp) * invrho;
      else uk = -0.1 * hook->g * Hk;
      u_store(*hook, k, uk);
    }
  }
  S vT(0.0);
  const S lnP0RT = LOG_PSTD_RU - lnT;
  for (int j = 0; j < mv.M; ++j) {
    RateOutT<S> ro;
    rate_one<NS, true>(mv, mv.rx + RX_REC * j, NS, T, lnT, invT, lnP0RT, C, gRT, hRT, ro);
    if (!ro.active) continue;
    const RxMeta mt = ro.mt;
    const int nr = mt.nrnp & 15, np = mt.nrnp >> 4;
    const S q = ro.q;
    wdot[mt.reac[0]] -= q;
    if (nr > 1) wdot[mt.reac[1]] -= q;
    if (nr > 2) wdot[mt.reac[2]] -= q;
    wdot[mt.prod[0]] += q;
    if (np > 1) wdot[mt.prod[1]] += q;
    if (np > 2) wdot[mt.prod[2]] += q;
    if (hook && hook->mode) {
      S w = u_load(*hook, mt.prod[0], q) - u_load(*hook, mt.reac[0], q);
      if (np > 1) w += u_load(*hook, mt.prod[1], q);
      if (np > 2) w += u_load(*hook, mt.prod[2], q);
      if (nr > 1) w -= u_load(*hook, mt.reac[1], q);
      if (nr > 2) w -= u_load(*hook, mt.reac[2], q);
      th_add(*hook, j, q * w);
    }
    S w = sig[mt.prod[0]] - sig[mt.reac[0]];
    if (np > 1) w += sig[mt.prod[1]];
    if (np > 2) w += sig[mt.prod[2]];
    if (nr > 1) w -= sig[mt.reac[1]];
    if (nr > 2) w -= sig[mt.reac[2]];
    vT += w * ro.dqdT;
    const S wf = w * ro.fk, wr = w * ro.rk;
    v[mt.reac[0]] += wf * (ro.cr[1] * ro.cr[2]);
    if (nr > 1) v[mt.reac[1]] += wf * (ro.cr[0] * ro.cr[2]);
    if (nr > 2) v[mt.reac[2]] += wf * (ro.cr[0] * ro.cr[1]);
    v[mt.prod[0]] -= wr * (ro.cp[1] * ro.cp[2]);
    if (np > 1) v[mt.prod[1]] -= wr * (ro.cp[0] * ro.cp[2]);
    if (np > 2) v[mt.prod[2]] -= wr * (ro.cp[0] * ro.cp[1]);
    const int type = mt.flags & 3;
    if (type != 0) {
      const double* ef = mv.eff + NS * ro.sl.eff;
      const S wM = w * ro.dqdM;
#pragma unroll
      for (int l = 0; l < NS; ++l) v[l] += wM * ef[l];
    }
  }
  // cp_k/R, recomputed (the same arithmetic as in the first loop) now that the
  // hook's scratch is no longer read
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* a = mv.sp + SP_REC * k + 2;
    cpR[k] = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
  }
  S Hw(0.0), sw(0.0), svc(0.0);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    Hw += hRT[k] * wdot[k];
    sw += sig[k] * wdot[k];
    svc += v[k] * C[k];
  }
  Hw = Hw * (RU * T);
#pragma unroll
  for (int k = 0; k < NS; ++k) f[1 + k] = mv.sp[SP_REC * k] * wdot[k] * invrho;
  f[0] = -(Hw * invrho * invcp);
  S dcp(0.0), cpf(0.0);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const double* a = mv.sp + SP_REC * k + 2;
    const double iW = mv.sp[SP_REC * k + 1];
    dcp += y[1 + k] * (a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]))) * iW;
    cpf += cpR[k] * iW * f[1 + k];
  }
  dcp = dcp * RU;
  cpf = cpf * RU;
  const S D = sw - svc;
  const S Wbar = 1.0 / sumYW;
  b[0] = invrho * (vT + invT * D) - r[0] * (invcp * (cpf + f[0] * dcp));
  const S DW = Wbar * invrho * D;
  const S fcp = r[0] * f[0] * invcp * RU;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const double iWi = mv.sp[SP_REC * i + 1];
    b[1 + i] = (v[i] + DW) * iWi - fcp * cpR[i] * iWi;
  }
}

// LU with partial pivoting of the n x n matrix in the strided view A; whole rows
// are swapped, the reciprocal of each pivot replaces the diagonal.  The matrix
// stays in shared memory, so the pivot loop is not unrolled (register budget).
template <int n, int ST = 0>
__device__ __forceinline__ bool lu_factor(SVT<double, ST> A, int* piv) {
  bool ok = true;
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    // pivot search on the magnitudes' bit patterns as 64-bit integers
    // (non-negative doubles order like their patterns): integer compares
    // instead of FP64 ones on the narrow pipe; a NaN sorts above every finite
    // value, is picked, and fails the finiteness test
    int p = k;
    long long best = __double_as_longlong(A[k * n + k]) & 0x7FFFFFFFFFFFFFFFLL;
    for (int i = k + 1; i < n; ++i) {
      const long long v = __double_as_longlong(A[i * n + k]) & 0x7FFFFFFFFFFFFFFFLL;
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    ok = ok && (best > 0) && (best < 0x7FF0000000000000LL);
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
template <int n, int ST = 0>
__device__ __forceinline__ void lu_solve(SVT<double, ST> A, const int* piv, SVT<double, ST> x) {
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    if (p != k) {
      const double t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
  }
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const double xk = x[k];
#pragma unroll
    for (int i = k + 1; i < n; ++i) x[i] -= A[i * n + k] * xk;
  }
#pragma unroll
  for (int k = n - 1; k >= 0; --k) {
    double acc = x[k];
#pragma unroll
    for (int j = k + 1; j < n; ++j) acc -= A[k * n + j] * x[j];
    x[k] = acc * A[k * n + k];
  }
}

}  // namespace df
