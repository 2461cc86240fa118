// Rosenbrock schemes in the form of Sandu et al. (1997), "Benchmarking stiff
// ODE solvers for atmospheric chemistry problems II: Rosenbrock solvers":
//   (I/(h gamma) - J) K_i = f(y + sum_{j<i} a_ij K_j) + sum_{j<i} (c_ij/h) K_j
//   y_new = y + sum_i m_i K_i,   err = sum_i e_i K_i
// with the RODAS4 coefficients of Hairer & Wanner (Solving ODEs II, Sec. VI.4)
// and the RODAS3 coefficients of Sandu et al. (1997).  One attempt of one cell
// on the thread-per-cell path, and the step-size control shared by the
// integrator and the adjoint's forward recomputation (so both follow the same
// step sequence).
#pragma once
#include "chem_thread.cuh"

namespace df {

struct RosTab {
  int s;
  int elo;
  double gamma;
  double a[6][6];
  double c[6][6];
  double m[6];
  double e[6];
  int newf[6];
  // stiffly accurate: m is the last row of a plus the last stage (m_j = a_{s-1,j}
  // for j < s - 1, m_{s-1} = 1), the error estimate is the last stage alone and
  // the last stage evaluates f at its own state; then y_new = Y_{s-1} + K_{s-1}
  // and err = K_{s-1}.  Both tables are (mark_stiffly_accurate); the kernels
  // rely on it and the host uploads no other table.
  int stiff_acc;
};

#ifndef __CUDACC_RTC__  // host-side table builders
static void mark_stiffly_accurate(RosTab& t) {
  const int l = t.s - 1;
  bool sa = l > 0 && t.m[l] == 1.0 && t.newf[l] != 0;
  for (int j = 0; j < l; ++j) sa = sa && t.m[j] == t.a[l][j] && t.e[j] == 0.0;
  t.stiff_acc = sa && t.e[l] == 1.0 ? 1 : 0;
}

static RosTab make_rodas4() {
  RosTab t;
  memset(&t, 0, sizeof(t));
  t.s = 6;
  t.elo = 4;
  t.gamma = 0.25;
  const double A[15] = {1.544, 0.9466785280815826, 0.2557011698983284, 3.314825187068521,
                        2.896124015972201, 0.9986419139977817, 1.221224509226641, 6.019134481288629,
                        12.53708332932087, -0.6878860361058950, 1.221224509226641, 6.019134481288629,
                        12.53708332932087, -0.6878860361058950, 1.0};
  const double C[15] = {-5.6688, -2.430093356833875, -0.2063599157091915, -0.1073529058151375,
                        -9.594562251023355, -20.47028614809616, 7.496443313967647, -10.24680431464352,
                        -33.99990352819905, 11.70890893206160, 8.083246795921522, -7.981132988064893,
                        -31.52159432874371, 16.31930543123136, -6.058818238834054};
  int idx = 0;
  for (int i = 1; i < 6; ++i)
    for (int j = 0; j < i; ++j) {
      t.a[i][j] = A[idx];
      t.c[i][j] = C[idx];
      ++idx;
    }
  t.m[0] = A[6];
  t.m[1] = A[7];
  t.m[2] = A[8];
  t.m[3] = A[9];
  t.m[4] = 1.0;
  t.m[5] = 1.0;
  t.e[5] = 1.0;
  for (int i = 0; i < 6; ++i) t.newf[i] = 1;
  mark_stiffly_accurate(t);
  return t;
}

static RosTab make_rodas3() {
  RosTab t;
  memset(&t, 0, sizeof(t));
  t.s = 4;
  t.elo = 3;
  t.gamma = 0.5;
  t.a[1][0] = 0.0;
  t.a[2][0] = 2.0;
  t.a[2][1] = 0.0;
  t.a[3][0] = 2.0;
  t.a[3][1] = 0.0;
  t.a[3][2] = 1.0;
  t.c[1][0] = 4.0;
  t.c[2][0] = 1.0;
  t.c[2][1] = -1.0;
  t.c[3][0] = 1.0;
  t.c[3][1] = -1.0;
  t.c[3][2] = -8.0 / 3.0;
  t.m[0] = 2.0;
  t.m[1] = 0.0;
  t.m[2] = 1.0;
  t.m[3] = 1.0;
  t.e[3] = 1.0;
  t.newf[0] = 1;
  t.newf[1] = 0;  // a[1][*] = 0: stage 2 reuses f(y)
  t.newf[2] = 1;
  t.newf[3] = 1;
  mark_stiffly_accurate(t);
  return t;
}
#endif


// One Rosenbrock attempt from y over h: K stages in Kv (strided, s x n), the
// factorised W = I/(h gamma) - J(y) left in Jv, the candidate state in ynew and
// the weighted RMS norm of the embedded error estimate in en.
// First trial step of a cell: theta over the fastest relative rate
// max_i |f_i| / max(|y_i|, floor_i) at the initial state (floor 1e-6 for mass
// fractions: species that start near zero do not set the scale).  It replaces
// the cuts the error control would otherwise make from h = dt on stiff cells,
// and is taken from f(y0), which the first attempt computes anyway.
constexpr double FIRST_STEP_THETA = 0.5;

template <int n>
__device__ __forceinline__ double first_step_limit(const double (&y)[n], const double (&f)[n]) {
  double r = fabs(f[0]) * rcp_nr(fabs(y[0]));
#pragma unroll
  for (int i = 1; i < n; ++i) r = fmax(r, fabs(f[i]) * rcp_nr(fmax(fabs(y[i]), 1e-6)));
  return r > 0.0 ? FIRST_STEP_THETA / r : INFINITY;
}

// pc: the reactor's fixed state parameter, pressure [dyn/cm^2] (CONSTV false)
// or density [g/cm^3] (CONSTV true; see eval_thread)
// Evaluation of f (and J) for ros_attempt: the mechanism-independent kernels
// read the mechanism from its blob (eval_thread); a kernel generated for one
// mechanism supplies its own policy with the same interface.
struct BlobEval {
  static constexpr bool kSpeciesVectors = true;  // uses the per-thread C, wdot, g, h, cp vectors
  template <int NS, bool WITH_J, bool CONSTV, int ST>
  __device__ __forceinline__ static double run(const MechView& mv, double pc, const double (&y)[NS + 1],
                                               double (&f)[NS + 1], SVT<double, ST> C, SVT<double, ST> wdot,
                                               SVT<double, ST> gRT, SVT<double, ST> hRT, SVT<double, ST> cpR,
                                               SVT<double, ST> Jv) {
    return eval_thread<NS, WITH_J, double, CONSTV, ST>(mv, pc, y, f, C, wdot, gRT, hRT, cpR, Jv);
  }
};

template <int NS, bool CONSTV = false, int ST = 0, class EVAL = BlobEval>
__device__ __forceinline__ bool ros_attempt(const MechView& mv, const RosTab& tb, double pc, const double (&y)[NS + 1],
                                            double& h, double rtol, double atolY, double atolT, SVT<double, ST> C,
                                            SVT<double, ST> wdot, SVT<double, ST> gRT, SVT<double, ST> hRT,
                                            SVT<double, ST> cpR, SVT<double, ST> Jv, SVT<double, ST> Kv, int stride,
                                            double (&ynew)[NS + 1], double& en, int* piv_out = nullptr,
                                            bool first = false, bool* last = nullptr, double* fT = nullptr) {
  constexpr int n = NS + 1;
  double fs[n];
  EVAL::template run<NS, true, CONSTV, ST>(mv, pc, y, fs, C, wdot, gRT, hRT, cpR, Jv);
  if (fT) *fT = fs[0];
  if (first) {
    const double hl = first_step_limit<n>(y, fs);
    if (hl < h) {
      h = hl;
      if (last) *last = false;
    }
  }
  const double hgi = rcp_nr(h * tb.gamma);
#pragma unroll
  for (int i = 0; i < n; ++i) {
#pragma unroll
    for (int j = 0; j < n; ++j) Jv[i * n + j] = i == j ? hgi - Jv[i * n + j] : -Jv[i * n + j];
  }
  int piv_l[n];
  int* piv = piv_out ? piv_out : piv_l;
  bool ok = lu_factor<n, ST>(Jv, piv);
  const double ih = rcp_nr(h);
  for (int s = 0; s < tb.s; ++s) {
    if (s > 0 && tb.newf[s]) {
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double acc = y[i];
        for (int j = 0; j < s; ++j) acc += tb.a[s][j] * Kv[j * n + i];
        ynew[i] = acc;
      }
      EVAL::template run<NS, false, CONSTV, ST>(mv, pc, ynew, fs, C, wdot, gRT, hRT, cpR, Jv);
    }
    // stage right-hand side, solved in place in the K slot of this stage
    SVT<double, ST> Ks{&Kv[s * n], stride};
#pragma unroll
    for (int i = 0; i < n; ++i) {
      double acc = fs[i];
      for (int j = 0; j < s; ++j) acc += (tb.c[s][j] * ih) * Kv[j * n + i];
      Ks[i] = acc;
    }
    lu_solve<n, ST>(Jv, piv, Ks);
  }
  // stiffly accurate tables (see RosTab): ynew holds the last stage's state
  // Y_{s-1} = y + sum_j a_{s-1,j} K_j, accumulated as y + sum_j m_j K_j would be,
  // so y_new = Y_{s-1} + K_{s-1} is that sum's double, and err = K_{s-1}; a
  // non-finite stage shows in y_new (integer test of its exponent), not in err
  double e2 = 0.0;
  bool fin = true;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const double e = Kv[(tb.s - 1) * n + i];
    const double yn = ynew[i] + e;
    fin = fin && (__double2hiint(yn) & 0x7ff00000) != 0x7ff00000;
    ynew[i] = yn;
    const double sc = (i == 0 ? atolT : atolY) + rtol * fmax(fabs(y[i]), fabs(yn));
    const double r = e * rcp_nr(sc);
    e2 += r * r;
  }
  en = sqrt(e2 * (1.0 / n));
  return ok && fin && isfinite(en);
}

// Ignition delay (Sec. 4.1 defines it by [dT/dt]_max): the largest dT/dt
// among the samples of one cell -- the states at which its accepted substeps
// start, in time order, where the integrator evaluates f anyway -- with its
// time refined by the vertex of the parabola through the largest sample and
// its two neighbours, so the delay is resolved below the substep spacing
// where the rate peak is smooth.  Without a neighbour on either side the time
// of the largest sample stands.
struct PeakTrack {
  double tp, fp;  // the sample before the largest
  double tb, fb;  // the largest
  double tn, fn;  // the first sample after the largest
  double tl, fl;  // the latest sample
  int have;       // bit 0: a sample before the largest, bit 1: one after, bit 2: any sample
  __host__ __device__ void reset() {
    tp = fp = tn = fn = tl = fl = tb = 0.0;
    fb = -INFINITY;
    have = 0;
  }
  __host__ __device__ void add(double t, double f) {
    if (f > fb) {
      tp = tl;
      fp = fl;
      tb = t;
      fb = f;
      have = (have & 4) ? 5 : 4;
    } else if (!(have & 2)) {
      tn = t;
      fn = f;
      have |= 2;
    }
    tl = t;
    fl = f;
    have |= 4;
  }
  __host__ __device__ double time() const {
    if ((have & 3) != 3) return tb;
    const double a = tb - tp, b = tb - tn;    // a > 0 > b
    const double fa = fb - fp, fc = fb - fn;  // both >= 0
    const double den = a * fc - b * fa;
    if (!(den > 0.0)) return tb;
    const double tv = tb - 0.5 * (a * a * fc - b * b * fa) / den;
    return fmin(fmax(tv, tp), tn);
  }
};

// accept / reject and the next step size.  Elementary controller (safety 0.9,
// growth limits [0.2, 6], down to 1e-4 before the first accepted step, no
// growth right after a rejection) combined with Gustafsson's predictive
// controller as in RODAS (Hairer & Wanner, Solving ODEs II, Sec. IV.8): after
// an accepted step the growth factor is the smaller of
//   0.9 err^(-1/p)  and  0.9 (h / h_acc) (err_acc / err^2)^(1/p),
// h_acc, err_acc being the previous accepted step and its error (>= 1e-2).
struct StepState {
  double hacc, erracc;
};

template <int n>
__device__ __forceinline__ void step_control(const RosTab& tb, bool ok, double en, bool last, double dt,
                                             double (&y)[n], const double (&ynew)[n], double& t, double& h,
                                             int& nacc, int& nrej, bool& last_rej, bool& done, StepState& ss) {
  // the accept test in FP64, the step-size factors in FP32 (a heuristic's
  // factors need no more; FP32 powf runs on the wide pipes, FP64 pow on the
  // narrow one)
  const float ie = -1.0f / (float)tb.elo;
  if (ok && en <= 1.0) {
#pragma unroll
    for (int i = 0; i < n; ++i) y[i] = ynew[i];
    t = last ? dt : t + h;
    ++nacc;
    const float e = fmaxf((float)en, 1e-10f);
    float fac = 0.9f * powf(e, ie);
    if (nacc > 1) fac = fminf(fac, 0.9f * ((float)h / (float)ss.hacc) * powf(e * e / (float)ss.erracc, ie));
    fac = fminf(last_rej ? 1.0f : 6.0f, fmaxf(0.2f, fac));
    ss.hacc = h;
    ss.erracc = fmax(1e-2, en);
    h *= (double)fac;
    last_rej = false;
    if (t >= dt) done = true;
  } else {
    ++nrej;
    // before the first accepted step the trial step (= dt) may be orders of
    // magnitude too long for a stiff cell: let the error estimate cut it deeply
    const float fmn = nacc == 0 ? 1e-4f : 0.2f;
    const float fac = ok ? fmaxf(fmn, 0.9f * powf((float)en, ie)) : 0.25f;
    h *= (double)fac;
    last_rej = true;
  }
}

}  // namespace df
