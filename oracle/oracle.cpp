// CPU oracle for the per-cell chemistry substep.  TEST INFRASTRUCTURE ONLY:
// only the test suite, the smoke check and the benchmark's CPU-baseline leg
// may load this library.  It shares no code with the CUDA path.
//
// What it computes (plain definitions, FP64, no blocking or fusion):
//   * species source terms of the reaction system, Sec. 2.3 eq. (sourceeq):
//       dY_a/dt = W_a sum_j (nu''_aj - nu'_aj) { K_fj prod (rho Y/W)^nu' - K_rj prod (rho Y/W)^nu'' } / rho
//     (the printed equation omits 1/rho; the bracket is a molar rate per volume,
//     so dividing by rho gives dY/dt);
//   * K_f by the Arrhenius law (Sec. 2.3), K_r = K_f / K_c with K_c from NASA-7
//     Gibbs energies, third-body [M] and Troe falloff (Gilbert-Luther-Troe form);
//   * the constant-pressure adiabatic energy balance of the 0D reactor
//     (Sec. 2.2, df0DFoam; T follows h, p, Y as in Sec. 3.2 correctThermo):
//       dT/dt = -sum_k H_k wdot_k / (rho cp)
//   * the Jacobian of that right-hand side by complex-step differentiation
//     (derivative definition, exact to rounding);
//   * the solution of the IVP over [0, dt] with a fully implicit Radau IIA
//     (order 5) method, full stage system solved by simplified Newton with a
//     dense partial-pivot LU, and step-doubling (Richardson) error control.
//     This stands in for CVODE (Sec. 2.3) and is deliberately a different
//     method from the GPU's Rosenbrock scheme;
//   * a Rosenbrock replay (fixed step sequence) of a named published tableau
//     and the complex-step derivative of its output: the reference for the
//     discrete adjoint.
//
// Units inside: cgs (mol/cm^3, erg).  At the interface: T [K], p [Pa],
// heat release [W/m^3], Ea [kJ/mol], A in cm-mol-s.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

typedef std::complex<double> cplx;

static const double RU_SI = 8.314462618;       // J/(mol K)
static const double RU = 8.314462618e7;        // erg/(mol K)
static const double PATM = 1.01325e6;          // dyn/cm^2 (standard-state pressure)
static const double LN10 = 2.302585092994045684;

extern "C" {
struct OMech {
  int N, M;
  const double* W;       // [N] g/mol
  const double* nasa;    // [N*7] a1..a7
  const int* nreac;      // [M] reactant entries (with multiplicity), <= 3
  const int* reac;       // [M*3]
  const int* nprod;      // [M]
  const int* prod;       // [M*3]
  const int* type;       // [M] 0 elementary, 1 three-body, 2 Troe falloff
  const int* rev;        // [M] 1 reversible
  const double* A;       // [M]
  const double* b;       // [M]
  const double* Ea;      // [M] kJ/mol
  const double* eff;     // [M*N] third-body efficiencies
  const double* A0;      // [M] Troe low-pressure limit
  const double* b0;
  const double* Ea0;
  const double* troe;    // [M*4] alpha, T***, T*, T**
};
}

static inline double re(double x) { return x; }
static inline double re(const cplx& x) { return x.real(); }

// ---------------------------------------------------------------------------
// thermo: NASA-7 polynomials (one temperature range)
// ---------------------------------------------------------------------------
template <class S>
static void thermo(const OMech& m, const S& T, S* cp_R, S* h_RT, S* s_R) {
  S lnT = std::log(T);
  for (int k = 0; k < m.N; ++k) {
    const double* a = m.nasa + 7 * k;
    S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    cp_R[k] = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    h_RT[k] = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    s_R[k] = a[0] * lnT + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
  }
}

// ---------------------------------------------------------------------------
// reaction rates: net molar production wdot [mol/cm^3/s], per-reaction data
// ---------------------------------------------------------------------------
// Reaction rates at (T, Y).  Constant-pressure reactor: rho from the pressure
// p_pa [Pa] and the ideal-gas law.  Constant-volume reactor (rho_fixed > 0):
// rho = rho_fixed [g/cm^3] (Sec. 2.2: df0DFoam's constant-volume case).
template <class S>
static void rates(const OMech& m, const S& T, double p_pa, const S* Y, S* wdot, S* rho_out,
                  S* qnet, S* kf_out, S* kr_out, const S* dlnA, double rho_fixed = 0.0) {
  const int N = m.N;
  std::vector<S> cp(N), h(N), s(N), C(N);
  thermo(m, T, cp.data(), h.data(), s.data());
  S sumYW = 0.0;
  for (int k = 0; k < N; ++k) sumYW += Y[k] / m.W[k];
  const double p = 10.0 * p_pa;
  S rho = rho_fixed > 0.0 ? S(rho_fixed) : p / (RU * T * sumYW);
  for (int k = 0; k < N; ++k) C[k] = rho * Y[k] / m.W[k];
  for (int k = 0; k < N; ++k) wdot[k] = 0.0;
  S lnT = std::log(T);
  for (int j = 0; j < m.M; ++j) {
    S shift = dlnA ? dlnA[j] : S(0.0);
    S kf = m.A[j] * std::exp(m.b[j] * lnT - m.Ea[j] * 1e3 / (RU_SI * T) + shift);
    if (m.A[j] == 0.0) kf = 0.0;
    S M3 = 0.0;
    if (m.type[j] != 0)
      for (int k = 0; k < N; ++k) M3 += m.eff[j * N + k] * C[k];
    if (m.type[j] == 1) {
      kf = kf * M3;
    } else if (m.type[j] == 2) {
      S k0 = m.A0[j] * std::exp(m.b0[j] * lnT - m.Ea0[j] * 1e3 / (RU_SI * T) + shift);
      if (m.A0[j] == 0.0) k0 = 0.0;
      S kinf = kf;
      if (re(kinf) == 0.0) {
        kf = 0.0;
      } else {
        S Pr = k0 * M3 / kinf;
        const double* tr = m.troe + 4 * j;
        S Fc = (1.0 - tr[0]) * std::exp(-T / tr[1]) + tr[0] * std::exp(-T / tr[2]) + std::exp(-tr[3] / T);
        S logFc = std::log(Fc) / LN10;
        S c = -0.4 - 0.67 * logFc;
        S nn = 0.75 - 1.27 * logFc;
        const double d = 0.14;
        S logPr = std::log(Pr) / LN10;
        S f1 = (logPr + c) / (nn - d * (logPr + c));
        S logF = logFc / (1.0 + f1 * f1);
        S F = std::exp(logF * LN10);
        kf = kinf * (Pr / (1.0 + Pr)) * F;
        if (re(Pr) == 0.0) kf = 0.0;
      }
    }
    // equilibrium constant in concentration units
    S sum_g = 0.0;
    int dnu = 0;
    for (int i = 0; i < m.nprod[j]; ++i) {
      int k = m.prod[3 * j + i];
      sum_g += h[k] - s[k];
      dnu += 1;
    }
    for (int i = 0; i < m.nreac[j]; ++i) {
      int k = m.reac[3 * j + i];
      sum_g -= h[k] - s[k];
      dnu -= 1;
    }
    S Kc = std::exp(-sum_g) * std::pow(PATM / (RU * T), (double)dnu);
    S kr = m.rev[j] ? kf / Kc : S(0.0);
    S Pf = 1.0, Pb = 1.0;
    for (int i = 0; i < m.nreac[j]; ++i) Pf *= C[m.reac[3 * j + i]];
    for (int i = 0; i < m.nprod[j]; ++i) Pb *= C[m.prod[3 * j + i]];
    S q = kf * Pf - kr * Pb;
    for (int i = 0; i < m.nreac[j]; ++i) wdot[m.reac[3 * j + i]] -= q;
    for (int i = 0; i < m.nprod[j]; ++i) wdot[m.prod[3 * j + i]] += q;
    if (qnet) qnet[j] = q;
    if (kf_out) kf_out[j] = kf;
    if (kr_out) kr_out[j] = kr;
  }
  if (rho_out) *rho_out = rho;
}

// y = (T, Y_1..Y_N); f = dy/dt.  Constant pressure: dT/dt = -sum H_k wdot_k /
// (rho cp), qdot = -sum H_k wdot_k [erg/cm^3/s].  Constant volume (rho_fixed >
// 0): the internal energy is conserved, dT/dt = -sum U_k wdot_k / (rho cv) with
// U_k = H_k - R T and cv = cp - R / W (per unit mass), qdot = -sum U_k wdot_k.
template <class S>
static void rhs(const OMech& m, double p_pa, const S* y, S* f, S* qdot, const S* dlnA,
                double rho_fixed = 0.0) {
  const int N = m.N;
  std::vector<S> wdot(N), cp(N), h(N), s(N);
  S rho;
  rates(m, y[0], p_pa, y + 1, wdot.data(), &rho, (S*)nullptr, (S*)nullptr, (S*)nullptr, dlnA, rho_fixed);
  thermo(m, y[0], cp.data(), h.data(), s.data());
  const double shift = rho_fixed > 0.0 ? 1.0 : 0.0;  // U/(RT) = H/(RT) - 1, cv/R = cp/R - 1
  S cm = 0.0, Hw = 0.0;
  for (int k = 0; k < N; ++k) {
    cm += y[1 + k] * RU * (cp[k] - shift) / m.W[k];
    Hw += RU * y[0] * (h[k] - shift) * wdot[k];
  }
  for (int k = 0; k < N; ++k) f[1 + k] = m.W[k] * wdot[k] / rho;
  f[0] = -Hw / (rho * cm);
  if (qdot) *qdot = -Hw;
}

template <class S>
static void jac_cs(const OMech& m, double p_pa, const double* y, double* J, double rho_fixed = 0.0) {
  const int n = m.N + 1;
  const double hstep = 1e-30;
  std::vector<cplx> yc(n), fc(n);
  for (int jcol = 0; jcol < n; ++jcol) {
    for (int i = 0; i < n; ++i) yc[i] = cplx(y[i], 0.0);
    double scale = std::max(std::fabs(y[jcol]), 1.0);
    yc[jcol] = cplx(y[jcol], hstep * scale);
    rhs<cplx>(m, p_pa, yc.data(), fc.data(), (cplx*)nullptr, (const cplx*)nullptr, rho_fixed);
    for (int i = 0; i < n; ++i) J[i * n + jcol] = fc[i].imag() / (hstep * scale);
  }
}

// ---------------------------------------------------------------------------
// dense LU with partial pivoting (real or complex; pivot by |real part|)
// ---------------------------------------------------------------------------
template <class S>
static bool lu_factor(int n, S* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(re(a[k * n + k]));
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(re(a[i * n + k]));
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0 || !std::isfinite(best)) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
    S inv = 1.0 / a[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      S l = a[i * n + k] * inv;
      a[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return true;
}

template <class S>
static void lu_solve(int n, const S* a, const int* piv, S* x) {
  // the factorization swapped whole rows (multipliers included), so apply the
  // whole permutation before the unit-lower solve
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(x[k], x[piv[k]]);
  for (int k = 0; k < n; ++k)
    for (int i = k + 1; i < n; ++i) x[i] -= a[i * n + k] * x[k];
  for (int k = n - 1; k >= 0; --k) {
    for (int j = k + 1; j < n; ++j) x[k] -= a[k * n + j] * x[j];
    x[k] /= a[k * n + k];
  }
}

// ---------------------------------------------------------------------------
// Radau IIA, 3 stages, order 5 (Hairer & Wanner, Solving ODEs II, Sec. IV.5)
// ---------------------------------------------------------------------------
struct RadauTab {
  double a[3][3];
  RadauTab() {
    const double s6 = std::sqrt(6.0);
    a[0][0] = (88.0 - 7.0 * s6) / 360.0;
    a[0][1] = (296.0 - 169.0 * s6) / 1800.0;
    a[0][2] = (-2.0 + 3.0 * s6) / 225.0;
    a[1][0] = (296.0 + 169.0 * s6) / 1800.0;
    a[1][1] = (88.0 + 7.0 * s6) / 360.0;
    a[1][2] = (-2.0 - 3.0 * s6) / 225.0;
    a[2][0] = (16.0 - s6) / 36.0;
    a[2][1] = (16.0 + s6) / 36.0;
    a[2][2] = 1.0 / 9.0;
  }
};

struct Ctx {
  const OMech* m;
  double p;
  double rho_fixed = 0.0;  // > 0: constant-volume reactor at this density
  int n;
  double rtol, atolY, atolT;
  long nrhs = 0, njac = 0;
};

static double wnorm_max(const Ctx& c, const double* e, const double* ya, const double* yb) {
  double mx = 0.0;
  for (int i = 0; i < c.n; ++i) {
    double at = i == 0 ? c.atolT : c.atolY;
    double sc = at + c.rtol * std::max(std::fabs(ya[i]), std::fabs(yb[i]));
    mx = std::max(mx, std::fabs(e[i]) / sc);
  }
  return mx;
}

// one Radau IIA step y0 -> y1 over h; returns false if Newton fails
static bool radau_step(Ctx& c, const RadauTab& tab, const double* y0, const double* J, double h,
                       double* y1) {
  const int n = c.n, N3 = 3 * n;
  std::vector<double> Mb(N3 * N3), Z(N3, 0.0), F(N3), r(N3), yi(n);
  std::vector<int> piv(N3);
  for (int bi = 0; bi < 3; ++bi)
    for (int bj = 0; bj < 3; ++bj)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          Mb[(bi * n + i) * N3 + bj * n + j] = (bi == bj && i == j ? 1.0 : 0.0) - h * tab.a[bi][bj] * J[i * n + j];
  if (!lu_factor(N3, Mb.data(), piv.data())) return false;
  double prev = 0.0;
  for (int it = 0; it < 25; ++it) {
    for (int s = 0; s < 3; ++s) {
      for (int i = 0; i < n; ++i) yi[i] = y0[i] + Z[s * n + i];
      rhs<double>(*c.m, c.p, yi.data(), F.data() + s * n, (double*)nullptr, (const double*)nullptr, c.rho_fixed);
      c.nrhs++;
    }
    for (int s = 0; s < 3; ++s)
      for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int t = 0; t < 3; ++t) acc += tab.a[s][t] * F[t * n + i];
        r[s * n + i] = -Z[s * n + i] + h * acc;
      }
    for (int i = 0; i < N3; ++i)
      if (!std::isfinite(r[i])) return false;
    lu_solve(N3, Mb.data(), piv.data(), r.data());
    double dn = 0.0;
    for (int s = 0; s < 3; ++s)
      for (int i = 0; i < n; ++i) {
        Z[s * n + i] += r[s * n + i];
        double at = i == 0 ? c.atolT : c.atolY;
        double sc = at + c.rtol * std::fabs(y0[i]);
        dn = std::max(dn, std::fabs(r[s * n + i]) / sc);
      }
    if (dn <= 1e-3) break;
    if (it > 0) {
      double theta = dn / prev;
      if (theta >= 0.9) {
        // no further contraction: the increments sit at the rounding floor of the
        // stage solve; accept when that floor is inside the step tolerance
        if (dn <= 1.0) break;
        return false;
      }
      if (theta / (1.0 - theta) * dn <= 1e-3) break;
    }
    prev = dn;
    if (it == 24) return false;
  }
  for (int i = 0; i < n; ++i) {
    y1[i] = y0[i] + Z[2 * n + i];
    if (!std::isfinite(y1[i])) return false;
  }
  return true;
}

// integrate one cell; returns status (0 ok, 1 max steps, 2 non-finite, 3 step underflow)
static int radau_cell(Ctx& c, double* y, double dt, int max_steps, int* nsteps_out) {
  static const RadauTab tab;
  const int n = c.n;
  std::vector<double> J(n * n), Jm(n * n), yb(n), ym(n), ys(n), e(n);
  double t = 0.0;
  double h = std::min(dt, 1e-12);
  int nacc = 0, nstep = 0;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(y[i])) return 2;
  if (y[0] <= 0.0) return 2;
  while (t < dt) {
    if (nstep >= max_steps) { *nsteps_out = nacc; return 1; }
    nstep++;
    bool last = false;
    if (t + h >= dt) { h = dt - t; last = true; }
    jac_cs<double>(*c.m, c.p, y, J.data(), c.rho_fixed);
    c.njac++;
    bool ok = radau_step(c, tab, y, J.data(), h, yb.data());
    if (ok) ok = radau_step(c, tab, y, J.data(), 0.5 * h, ym.data());
    if (ok) {
      jac_cs<double>(*c.m, c.p, ym.data(), Jm.data(), c.rho_fixed);
      c.njac++;
      ok = radau_step(c, tab, ym.data(), Jm.data(), 0.5 * h, ys.data());
    }
    if (!ok) {
      h *= 0.25;
      if (h < 1e-30) { *nsteps_out = nacc; return 3; }
      continue;
    }
    for (int i = 0; i < n; ++i) e[i] = (ys[i] - yb[i]) / 31.0;
    double err = wnorm_max(c, e.data(), y, ys.data());
    double fac = err > 0.0 ? 0.9 * std::pow(err, -1.0 / 6.0) : 5.0;
    fac = std::min(5.0, std::max(0.1, fac));
    if (err <= 1.0) {
      t = last ? dt : t + h;
      for (int i = 0; i < n; ++i) y[i] = ys[i];
      nacc++;
      h *= fac;
    } else {
      h *= std::min(fac, 0.5);
      if (h < 1e-30) { *nsteps_out = nacc; return 3; }
    }
  }
  *nsteps_out = nacc;
  return 0;
}

// ---------------------------------------------------------------------------
// Rosenbrock replay: s-stage scheme in the form
//   (I/(h g) - J) K_i = f(y + sum_{j<i} a_ij K_j) + sum_{j<i} (c_ij / h) K_j
//   y_new = y + sum m_i K_i
// with the RODAS4 coefficients of Hairer & Wanner (Solving ODEs II, Sec. VI.4),
// written in the transformed variables used by Sandu et al. (1997) "Benchmarking
// stiff ODE solvers for atmospheric chemistry problems II".  Step sequence given.
// ---------------------------------------------------------------------------
struct RosTab {
  int s;
  double gamma;
  double a[6][6];
  double c[6][6];
  double m[6];
  double e[6];
};

static RosTab rodas4_tab() {
  RosTab t;
  std::memset(&t, 0, sizeof(t));
  t.s = 6;
  t.gamma = 0.25;
  double A[15] = {0.1544000000000000e+01, 0.9466785280815826e+00, 0.2557011698983284e+00,
                  0.3314825187068521e+01, 0.2896124015972201e+01, 0.9986419139977817e+00,
                  0.1221224509226641e+01, 0.6019134481288629e+01, 0.1253708332932087e+02,
                  -0.6878860361058950e+00, 0.1221224509226641e+01, 0.6019134481288629e+01,
                  0.1253708332932087e+02, -0.6878860361058950e+00, 1.0};
  double C[15] = {-0.5668800000000000e+01, -0.2430093356833875e+01, -0.2063599157091915e+00,
                  -0.1073529058151375e+00, -0.9594562251023355e+01, -0.2047028614809616e+02,
                  0.7496443313967647e+01, -0.1024680431464352e+02, -0.3399990352819905e+02,
                  0.1170890893206160e+02, 0.8083246795921522e+01, -0.7981132988064893e+01,
                  -0.3152159432874371e+02, 0.1631930543123136e+02, -0.6058818238834054e+01};
  int idx = 0;
  for (int i = 1; i < 6; ++i)
    for (int j = 0; j < i; ++j) {
      t.a[i][j] = A[idx];
      t.c[i][j] = C[idx];
      idx++;
    }
  t.m[0] = A[6]; t.m[1] = A[7]; t.m[2] = A[8]; t.m[3] = A[9]; t.m[4] = 1.0; t.m[5] = 1.0;
  t.e[5] = 1.0;
  return t;
}

template <class S>
static bool ros_step(const OMech& mech, double p, const RosTab& tb, const S* y, const S* J, double h,
                     S* ynew, S* err, const S* dlnA) {
  const int n = mech.N + 1;
  std::vector<S> W(n * n), K(6 * n), ys(n), f(n);
  std::vector<int> piv(n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) W[i * n + j] = (i == j ? 1.0 / (h * tb.gamma) : 0.0) - J[i * n + j];
  if (!lu_factor(n, W.data(), piv.data())) return false;
  for (int st = 0; st < tb.s; ++st) {
    for (int i = 0; i < n; ++i) {
      S acc = y[i];
      for (int j = 0; j < st; ++j) acc += tb.a[st][j] * K[j * n + i];
      ys[i] = acc;
    }
    rhs<S>(mech, p, ys.data(), f.data(), (S*)nullptr, dlnA);
    for (int i = 0; i < n; ++i) {
      S acc = f[i];
      for (int j = 0; j < st; ++j) acc += (tb.c[st][j] / h) * K[j * n + i];
      K[st * n + i] = acc;
    }
    lu_solve(n, W.data(), piv.data(), K.data() + st * n);
  }
  for (int i = 0; i < n; ++i) {
    S acc = y[i], e = 0.0;
    for (int st = 0; st < tb.s; ++st) {
      acc += tb.m[st] * K[st * n + i];
      e += tb.e[st] * K[st * n + i];
    }
    ynew[i] = acc;
    if (err) err[i] = e;
  }
  return true;
}

// analytic-free complex Jacobian at a complex point: for the replay under complex
// step we need J(y) with y complex.  We use the holomorphic extension: a second
// complex-step direction is not available, so J is taken by central finite
// differences of the complex RHS with a real step small enough for the
// truncation error to stay far below the tolerance of the gradient checks.
static void jac_fd_cplx(const OMech& m, double p, const cplx* y, cplx* J, const cplx* dlnA) {
  const int n = m.N + 1;
  std::vector<cplx> yp(n), fp(n), fm(n);
  for (int j = 0; j < n; ++j) {
    double hs = 1e-5 * std::max(std::fabs(y[j].real()), j == 0 ? 1.0 : 1e-8);
    for (int i = 0; i < n; ++i) yp[i] = y[i];
    yp[j] += hs;
    rhs<cplx>(m, p, yp.data(), fp.data(), (cplx*)nullptr, dlnA);
    yp[j] = y[j] - hs;
    rhs<cplx>(m, p, yp.data(), fm.data(), (cplx*)nullptr, dlnA);
    for (int i = 0; i < n; ++i) J[i * n + j] = (fp[i] - fm[i]) / (2.0 * hs);
  }
}

extern "C" {

int or_thermo(const OMech* m, double T, double* cp_R, double* h_RT, double* s_R) {
  thermo<double>(*m, T, cp_R, h_RT, s_R);
  return 0;
}

// single cell rates: wdot [mol/cm^3/s], rho [g/cm^3], q/kf/kr per reaction (may be NULL)
int or_rates(const OMech* m, double T, double p, const double* Y, double* wdot, double* rho,
             double* q, double* kf, double* kr) {
  double r;
  rates<double>(*m, T, p, Y, wdot, &r, q, kf, kr, (const double*)nullptr);
  if (rho) *rho = r;
  return 0;
}

// f = dy/dt for y = (T, Y); qdot in W/m^3 (may be NULL)
int or_rhs(const OMech* m, double p, const double* y, double* f, double* qdot) {
  double q;
  rhs<double>(*m, p, y, f, &q, (const double*)nullptr);
  if (qdot) *qdot = 0.1 * q;
  return 0;
}

int or_jac(const OMech* m, double p, const double* y, double* J) {
  jac_cs<double>(*m, p, y, J);
  return 0;
}

// Integrate ncells cells over dt.  T[c], p[c], Y[k*ncells + c] (species-major).
// T and Y are overwritten.  status[c], nsteps[c] (accepted steps).
int or_integrate(const OMech* m, int64_t ncells, double* T, const double* p, double* Y, double dt,
                 double rtol, double atolY, double atolT, int max_steps, int* status, int* nsteps,
                 int nthreads) {
  const int N = m->N, n = N + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<double> y(n);
    y[0] = T[c];
    for (int k = 0; k < N; ++k) y[1 + k] = Y[(int64_t)k * ncells + c];
    Ctx ctx;
    ctx.m = m;
    ctx.p = p[c];
    ctx.n = n;
    ctx.rtol = rtol;
    ctx.atolY = atolY;
    ctx.atolT = atolT;
    int ns = 0;
    int st = radau_cell(ctx, y.data(), dt, max_steps, &ns);
    status[c] = st;
    if (nsteps) nsteps[c] = ns;
    if (st == 0) {
      T[c] = y[0];
      for (int k = 0; k < N; ++k) Y[(int64_t)k * ncells + c] = y[1 + k];
    }
  }
  return 0;
}

// Constant-volume reactor (Sec. 2.2, df0DFoam): right-hand side and Jacobian at
// density rho [g/cm^3]; qdot = -sum U_k wdot_k [W/m^3].
int or_rhs_v(const OMech* m, double rho, const double* y, double* f, double* qdot) {
  double q;
  rhs<double>(*m, 0.0, y, f, &q, (const double*)nullptr, rho);
  if (qdot) *qdot = 0.1 * q;
  return 0;
}

int or_jac_v(const OMech* m, double rho, const double* y, double* J) {
  jac_cs<double>(*m, 0.0, y, J, rho);
  return 0;
}

// Constant-volume integration: each cell's density is fixed from its initial
// state (p[c] [Pa], T, Y) by the ideal-gas law; T and Y are overwritten.
int or_integrate_v(const OMech* m, int64_t ncells, double* T, const double* p, double* Y, double dt,
                   double rtol, double atolY, double atolT, int max_steps, int* status, int* nsteps,
                   int nthreads) {
  const int N = m->N, n = N + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t c = 0; c < ncells; ++c) {
    std::vector<double> y(n);
    y[0] = T[c];
    double sumYW = 0.0;
    for (int k = 0; k < N; ++k) {
      y[1 + k] = Y[(int64_t)k * ncells + c];
      sumYW += y[1 + k] / m->W[k];
    }
    Ctx ctx;
    ctx.m = m;
    ctx.p = p[c];
    ctx.rho_fixed = 10.0 * p[c] / (RU * y[0] * sumYW);
    ctx.n = n;
    ctx.rtol = rtol;
    ctx.atolY = atolY;
    ctx.atolT = atolT;
    int ns = 0;
    int st = (ctx.rho_fixed > 0.0 && std::isfinite(ctx.rho_fixed)) ? radau_cell(ctx, y.data(), dt, max_steps, &ns) : 2;
    status[c] = st;
    if (nsteps) nsteps[c] = ns;
    if (st == 0) {
      T[c] = y[0];
      for (int k = 0; k < N; ++k) Y[(int64_t)k * ncells + c] = y[1 + k];
    }
  }
  return 0;
}

// RODAS4 replay with the given step sequence (real).  y in/out (n = N+1).
int or_ros_replay(const OMech* m, double p, double* y, int nsteps, const double* hs) {
  const int n = m->N + 1;
  RosTab tb = rodas4_tab();
  std::vector<double> J(n * n), yn(n);
  for (int s = 0; s < nsteps; ++s) {
    jac_cs<double>(*m, p, y, J.data());
    if (!ros_step<double>(*m, p, tb, y, J.data(), hs[s], yn.data(), (double*)nullptr,
                          (const double*)nullptr))
      return -1;
    for (int i = 0; i < n; ++i) y[i] = yn[i];
  }
  return 0;
}

// One RODAS4 step with its embedded error vector (real), J by complex step.
int or_ros_step(const OMech* m, double p, const double* y, double h, double* ynew, double* err) {
  const int n = m->N + 1;
  RosTab tb = rodas4_tab();
  std::vector<double> J(n * n);
  jac_cs<double>(*m, p, y, J.data());
  return ros_step<double>(*m, p, tb, y, J.data(), h, ynew, err, (const double*)nullptr) ? 0 : -1;
}

// Directional derivative of the replayed map by complex step:
//   L = wT * T(end) + sum_k wY[k] * Y_k(end) + wQ * qdot(end)  [qdot in W/m^3]
// perturbed along direction (dy0 [n], dlnA [M]).  Returns dL.
int or_ros_replay_dir(const OMech* m, double p, const double* y0, int nsteps, const double* hs,
                      double wT, const double* wY, double wQ, const double* dy0, const double* dlnA,
                      double* dL) {
  const int n = m->N + 1;
  const double eps = 1e-20;
  RosTab tb = rodas4_tab();
  std::vector<cplx> y(n), yn(n), J(n * n), dA(m->M), f(n);
  for (int i = 0; i < n; ++i) y[i] = cplx(y0[i], eps * (dy0 ? dy0[i] : 0.0));
  for (int j = 0; j < m->M; ++j) dA[j] = cplx(0.0, eps * (dlnA ? dlnA[j] : 0.0));
  for (int s = 0; s < nsteps; ++s) {
    jac_fd_cplx(*m, p, y.data(), J.data(), dA.data());
    if (!ros_step<cplx>(*m, p, tb, y.data(), J.data(), hs[s], yn.data(), (cplx*)nullptr, dA.data()))
      return -1;
    y = yn;
  }
  cplx q;
  rhs<cplx>(*m, p, y.data(), f.data(), &q, dA.data());
  cplx L = wT * y[0] + wQ * 0.1 * q;
  for (int k = 0; k < m->N; ++k) L += (wY ? wY[k] : 0.0) * y[1 + k];
  *dL = L.imag() / eps;
  return 0;
}

}  // extern "C"

extern "C" int or_debug_trace(const OMech* m, double p, double* y, double dt, double rtol, double atolY,
                              double atolT, int max_steps, double* trace /*[max_steps*4]*/) {
  static const RadauTab tab;
  Ctx c; c.m = m; c.p = p; c.n = m->N + 1; c.rtol = rtol; c.atolY = atolY; c.atolT = atolT;
  const int n = c.n;
  std::vector<double> J(n * n), Jm(n * n), yb(n), ym(n), ys(n), e(n);
  double t = 0.0, h = std::min(dt, 1e-12);
  int nstep = 0;
  while (t < dt && nstep < max_steps) {
    bool last = false;
    if (t + h >= dt) { h = dt - t; last = true; }
    jac_cs<double>(*m, p, y, J.data());
    bool ok = radau_step(c, tab, y, J.data(), h, yb.data());
    if (ok) ok = radau_step(c, tab, y, J.data(), 0.5 * h, ym.data());
    if (ok) { jac_cs<double>(*m, p, ym.data(), Jm.data()); ok = radau_step(c, tab, ym.data(), Jm.data(), 0.5 * h, ys.data()); }
    double err = -1;
    if (ok) { for (int i = 0; i < n; ++i) e[i] = (ys[i] - yb[i]) / 31.0; err = wnorm_max(c, e.data(), y, ys.data()); }
    trace[4*nstep] = t; trace[4*nstep+1] = h; trace[4*nstep+2] = err; trace[4*nstep+3] = y[0];
    nstep++;
    if (!ok) { h *= 0.25; continue; }
    double fac = err > 0.0 ? 0.9 * std::pow(err, -1.0 / 6.0) : 5.0;
    fac = std::min(5.0, std::max(0.1, fac));
    if (err <= 1.0) { t = last ? dt : t + h; for (int i = 0; i < n; ++i) y[i] = ys[i]; h *= fac; }
    else h *= std::min(fac, 0.5);
  }
  return nstep;
}
