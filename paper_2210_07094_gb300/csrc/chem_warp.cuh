// Device chemistry for the one-cell-per-warp path (any N <= 64; used for the
// 50-species mechanism).  The 32 lanes of a warp share one cell:
//   thermo      - lanes over species,
//   rates       - lanes over reactions (rate_one, same math as the thread path),
//   wdot, J     - lanes over species rows, summing their reactions from a
//                 species -> (reaction, nu) list (fixed order: deterministic,
//                 no atomics),
//   LU          - pivot search by warp reduction, trailing update dealt
//                 element by element over the lanes,
//   solves      - column-oriented substitution, one __syncwarp per step.
// All per-cell vectors and the dense (N+1)^2 matrix live in shared memory.
#pragma once
#include "chem_thread.cuh"

namespace df {

constexpr unsigned WFULL = 0xffffffffu;

// plain shared-memory vector with the same indexing interface as SV
struct PV {
  double* p;
  __device__ __forceinline__ double& operator[](int i) const { return p[i]; }
};

// per-warp workspace layout (offsets in doubles)
struct WarpWS {
  int y, ys, f, wdot, C, gRT, hRT, q, fk, rk, dT, dM, J, K, piv, total;
};

// Seven cells of the 50-species mechanism fit an SM where six did with one
// slot per quantity: the production rates share the g/RT slots (the rates
// read g/RT before the per-species sums write the production rates, and the
// temperature row reuses the slots after the last read of the production
// rates); d q / d[M] has one slot per third-body reaction; d q / dT lives in
// the stage vectors while the Jacobian is built (no stage vector is live
// then) where they have room; cp/R is recomputed where it is needed.
__host__ __device__ inline WarpWS warp_ws_layout(int N, int M, int n_eff) {
  const int n = N + 1;
  WarpWS w;
  int o = 0;
  w.y = o; o += n;
  w.f = o; o += n;
  w.C = o; o += N;
  w.gRT = o; o += N;
  w.wdot = w.gRT;
  w.hRT = o; o += N;
  w.q = o; o += M;
  w.fk = o; o += M;
  w.rk = o; o += M;
  w.dM = o; o += n_eff > 0 ? n_eff : 1;
  w.J = o; o += n * n;
  w.K = o; o += 6 * n;
  // the stage state shares the last stage vector's slot: it is read (f(ys))
  // before that stage vector is written, and the candidate state overwrites
  // it element by element after each lane has read its own elements
  w.ys = w.K + 5 * n;
  if (M <= 6 * n) {
    w.dT = w.K;
  } else {
    w.dT = o;
    o += M;
  }
  w.piv = o; o += (n + 1) / 2;  // ints, two per double slot
  w.total = (o + 1) & ~1;
  return w;
}

// cp/R of species k at T (NASA-7)
__device__ __forceinline__ double cp_species(const MechView& mv, int k, double T) {
  const double* a = mv.sp + SP_REC * k + 2;
  return a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
}


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(WFULL, v, o);
  return v;
}

// Evaluate f(y) (and J when WITH_J) for the state at ws + yoff.
// csr: [N+1] row pointers, then (reaction, nu) pairs.  Returns qdot in erg/(cm^3 s).
// pc: pressure [dyn/cm^2], or the fixed density [g/cm^3] of a constant-volume
// reactor (CONSTV; the same closure as eval_thread).
template <bool WITH_J, bool CONSTV = false>
__device__ double warp_eval(const MechView& mv, const int* csr, int N, double pc, double* ws, const WarpWS& L,
                            int yoff) {
  constexpr double EV = CONSTV ? 1.0 : 0.0;  // U/(RT) = H/(RT) - 1, cv/R = cp/R - 1
  const int lane = threadIdx.x & 31;
  const int n = N + 1;
  const double* y = ws + yoff;
  double* f = ws + L.f;
  PV C{ws + L.C}, gRT{ws + L.gRT}, hRT{ws + L.hRT};
  double* wdot = ws + L.wdot;  // the g/RT slots, once the rates have read them
  const double T = y[0];
  const double lnT = log_tab(T);
  const double invT = rcp_nr(T);
  // thermo and sum Y/W
  double sYW = 0.0;
  for (int k = lane; k < N; k += 32) {
    const double* a = mv.sp + SP_REC * k + 2;
    const double* ah = mv.sp + SP_REC * k + SP_H;  // a2/2 .. a5/5
    const double* as = mv.sp + SP_REC * k + SP_S;  // a3/2 .. a5/4
    const double hk = a[0] + T * (ah[0] + T * (ah[1] + T * (ah[2] + T * ah[3]))) + a[5] * invT;
    const double sk = a[0] * lnT + T * (a[1] + T * (as[0] + T * (as[1] + T * as[2]))) + a[6];
    hRT[k] = hk;
    gRT[k] = hk - sk;
    sYW += y[1 + k] * mv.sp[SP_REC * k + 1];
  }
  const double sumYW = warp_sum(sYW);
  const double Wbar = rcp_nr(sumYW);
  const double rho = CONSTV ? pc : pc * invT * Wbar * (1.0 / RU);
  double cs = 0.0;
  for (int k = lane; k < N; k += 32) {
    const double ck = rho * y[1 + k] * mv.sp[SP_REC * k + 1];
    C[k] = ck;
    cs += ck;
  }
  // third-body [M] = sum_l C_l + the sparse corrections (eps_l - 1) C_l; the
  // table follows the species lists and the lane assignment in csr
  const int* effs = csr + N + 1 + 2 * csr[N] + 64;
  const SparseEff se{effs + 1, effs + 2 + effs[0], warp_sum(cs)};
  __syncwarp();
  const double lnP0RT = LOG_PSTD_RU - lnT;
  // reactions: one lane per reaction
  for (int j = lane; j < mv.M; j += 32) {
    RateOut ro;
    rate_one<0, WITH_J>(mv, mv.rx + RX_REC * j, N, T, lnT, invT, lnP0RT, C, gRT, hRT, ro, &se);
    if (ro.active) {
      ws[L.q + j] = ro.q;
      if (WITH_J) {
        ws[L.fk + j] = ro.fk;
        ws[L.rk + j] = ro.rk;
        ws[L.dT + j] = ro.dqdT;
        if ((ro.mt.flags & 3) != 0) ws[L.dM + ro.sl.eff] = ro.dqdM;
      }
    } else {
      ws[L.q + j] = 0.0;
      if (WITH_J) {
        ws[L.fk + j] = 0.0;
        ws[L.rk + j] = 0.0;
        ws[L.dT + j] = 0.0;
        const double* r = mv.rx + RX_REC * j;
        if ((load_meta(r).flags & 3) != 0) ws[L.dM + load_slots(r).eff] = 0.0;
      }
    }
  }
  __syncwarp();
  // species production rates, cp, heat release.  Each lane sums the reaction
  // lists of its (at most two) species in one loop over their concatenation,
  // so the warp waits for the longest pair, not for the longest list of each
  // of two rounds; each list is still summed in its own fixed order.
  const int* asg = csr + N + 1 + 2 * csr[N] + 2 * lane;
  const int ka = asg[0], kb = asg[1];
  const int ba = ka >= 0 ? csr[ka] : 0, la = ka >= 0 ? csr[ka + 1] - ba : 0;
  const int bb = kb >= 0 ? csr[kb] : 0, lb = kb >= 0 ? csr[kb + 1] - bb : 0;
  double cpp = 0.0, hwp = 0.0;
  {
    // one running sum, one multiply-add per entry: the first list's sum is
    // set aside where the second list starts
    double acc = 0.0, wa = 0.0, wb = 0.0;
    for (int t = 0; t < la + lb; ++t) {
      if (t == la) {
        wa = acc;
        acc = 0.0;
      }
      const int e = t < la ? ba + t : bb + (t - la);
      acc = fma(small_int_to_double(csr[N + 2 + 2 * e]), ws[L.q + csr[N + 1 + 2 * e]], acc);
    }
    if (lb > 0) wb = acc;
    else wa = acc;
    if (ka >= 0) {
      wdot[ka] = wa;
      cpp += y[1 + ka] * (cp_species(mv, ka, T) - EV) * mv.sp[SP_REC * ka + 1];
      hwp += (hRT[ka] - EV) * wa;
    }
    if (kb >= 0) {
      wdot[kb] = wb;
      cpp += y[1 + kb] * (cp_species(mv, kb, T) - EV) * mv.sp[SP_REC * kb + 1];
      hwp += (hRT[kb] - EV) * wb;
    }
  }
  __syncwarp();
  const double cpm = RU * warp_sum(cpp);
  const double Hw = RU * T * warp_sum(hwp);
  const double invrho = rcp_nr(rho);
  const double invcp = rcp_nr(cpm);
  for (int k = lane; k < N; k += 32) f[1 + k] = mv.sp[SP_REC * k] * wdot[k] * invrho;
  const double fT = -Hw * invrho * invcp;
  if (lane == 0) f[0] = fT;
  if (WITH_J) {
    double* J = ws + L.J;
    // concentration-space rows of this lane's species: one loop over the
    // concatenation of their reaction lists (as for the production rates)
    if (ka >= 0)
      for (int c = 0; c < n; ++c) J[(1 + ka) * n + c] = 0.0;
    if (kb >= 0)
      for (int c = 0; c < n; ++c) J[(1 + kb) * n + c] = 0.0;
    // collider columns d q_j / d[M] eps_l: the unit part summed per row (sMa,
    // sMb; added to every species column in the conversion below), the
    // corrections eps_l - 1 entered where the efficiency is not 1
    double sMa = 0.0, sMb = 0.0;
    for (int t = 0; t < la + lb; ++t) {
      const bool first = t < la;
      const int e = first ? ba + t : bb + (t - la);
      double* row = J + (1 + (first ? ka : kb)) * n;
      {
        const int j = csr[N + 1 + 2 * e];
        const double nu = small_int_to_double(csr[N + 2 + 2 * e]);
        const double* r = mv.rx + RX_REC * j;
        const RxMeta mt = load_meta(r);
        const int nr = mt.nrnp & 15, np = mt.nrnp >> 4;
        const double fk = ws[L.fk + j], rk = ws[L.rk + j];
        row[0] += nu * ws[L.dT + j];
        const double c0 = C[mt.reac[0]], c1 = nr > 1 ? C[mt.reac[1]] : 1.0, c2 = nr > 2 ? C[mt.reac[2]] : 1.0;
        row[1 + mt.reac[0]] += nu * fk * c1 * c2;
        if (nr > 1) row[1 + mt.reac[1]] += nu * fk * c0 * c2;
        if (nr > 2) row[1 + mt.reac[2]] += nu * fk * c0 * c1;
        const double d0 = C[mt.prod[0]], d1 = np > 1 ? C[mt.prod[1]] : 1.0, d2 = np > 2 ? C[mt.prod[2]] : 1.0;
        row[1 + mt.prod[0]] -= nu * rk * d1 * d2;
        if (np > 1) row[1 + mt.prod[1]] -= nu * rk * d0 * d2;
        if (np > 2) row[1 + mt.prod[2]] -= nu * rk * d0 * d1;
        if ((mt.flags & 3) != 0) {
          const int sl = load_slots(r).eff;
          const double cM = nu * ws[L.dM + sl];
          if (first) sMa += cM;
          else sMb += cM;
          for (int u = se.off[sl]; u < se.off[sl + 1]; ++u) {
            const int* q = se.ent + 3 * u;
            row[1 + q[0]] += cM * __hiloint2double(q[2], q[1]);
          }
        }
      }
    }
    // -> (T, Y) space, row by row
    for (int tk = 0; tk < 2; ++tk) {
      const int k = tk == 0 ? ka : kb;
      if (k < 0) continue;
      double* row = J + (1 + k) * n;
      const double Wk = mv.sp[SP_REC * k];
      const double sM = tk == 0 ? sMa : sMb;  // the row's unit collider part
      if (CONSTV) {  // C does not move with T or the mean molar mass
        const double b = Wk * sM;
        for (int i = 0; i < N; ++i) row[1 + i] = fma(Wk, row[1 + i], b) * mv.sp[SP_REC * i + 1];
        row[0] = Wk * invrho * row[0];
        continue;
      }
      double s = sM * se.ctot;
      for (int l = 0; l < N; ++l) s += row[1 + l] * C[l];
      const double wk = wdot[k];
      const double a = Wk * Wbar * invrho * (wk - s) + Wk * sM;
      for (int i = 0; i < N; ++i) row[1 + i] = (Wk * row[1 + i] + a) * mv.sp[SP_REC * i + 1];
      row[0] = Wk * invrho * (row[0] + (wk - s) * invT);
    }
    __syncwarp();
    // temperature row
    // hw_k = (h_k/RT - EV) / W_k, once per species (into the g/RT slots, which
    // the rates no longer need), for the column sums below
    double dcp = 0.0, cpf = 0.0;
    for (int k = lane; k < N; k += 32) {
      const double* a = mv.sp + SP_REC * k + 2;
      const double iW = mv.sp[SP_REC * k + 1];
      dcp += y[1 + k] * (a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]))) * iW;
      cpf += (cp_species(mv, k, T) - EV) * iW * f[1 + k];
      gRT[k] = (hRT[k] - EV) * iW;
    }
    dcp = RU * warp_sum(dcp);
    cpf = RU * warp_sum(cpf);
    __syncwarp();
    for (int jc = lane; jc < n; jc += 32) {
      double acc = 0.0;
      for (int k = 0; k < N; ++k) acc += gRT[k] * J[(1 + k) * n + jc];
      acc *= RU * T;
      if (jc == 0) J[0] = -invcp * (acc + cpf) - fT * dcp * invcp;
      else J[jc] = -invcp * acc - fT * RU * (cp_species(mv, jc - 1, T) - EV) * mv.sp[SP_REC * (jc - 1) + 1] * invcp;
    }
  }
  __syncwarp();
  return -Hw;
}

// LU with partial pivoting of the n x n row-major matrix A (shared memory),
// whole rows swapped, reciprocal pivots on the diagonal, and the columns of U
// above the diagonal divided by their pivot (U'_ik = U_ik / U_kk, for the
// back substitution of warp_solve).  Returns false if a pivot is zero or not
// finite.  The pivot search compares the magnitudes' bit patterns as 64-bit
// integers (non-negative doubles order like their patterns), so it runs on
// the integer pipe instead of the narrow FP64 one; a NaN sorts above every
// finite value, is picked, and fails the finiteness test.
__device__ bool warp_lu(double* A, int* piv, int n) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    long long best = -1;
    int bi = k;
    for (int i = k + lane; i < n; i += 32) {
      const long long v = __double_as_longlong(A[i * n + k]) & 0x7FFFFFFFFFFFFFFFLL;
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ob = __shfl_xor_sync(WFULL, best, o);
      const int oi = __shfl_xor_sync(WFULL, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    ok = ok && (best > 0) && (best < 0x7FF0000000000000LL);
    if (lane == 0) piv[k] = bi;
    if (bi != k) {
      for (int j = lane; j < n; j += 32) {
        const double t = A[k * n + j];
        A[k * n + j] = A[bi * n + j];
        A[bi * n + j] = t;
      }
    }
    __syncwarp();
    const double inv = rcp_nr(A[k * n + k]);
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) A[i * n + k] *= inv;
    for (int i = lane; i < k; i += 32) A[i * n + k] *= inv;  // U'_ik = U_ik / U_kk (row i < k is final)
    if (lane == 0) A[k * n + k] = inv;
    __syncwarp();
    // trailing update of the m x m block: its elements are dealt to the lanes
    // row by row (element e = i m + j to lane e mod 32), so all 32 lanes stay
    // busy down to a block of 32 elements
    const int m = n - 1 - k;
    if (m > 0) {
      const int di = 32 / m, dj = 32 - di * m;
      int i = lane / m, j = lane - (lane / m) * m;
      const double* urow = A + k * n + k + 1;
      while (i < m) {
        double* row = A + (k + 1 + i) * n;
        row[k + 1 + j] -= row[k] * urow[j];
        i += di;
        j += dj;
        if (j >= m) {
          j -= m;
          ++i;
        }
      }
    }
    __syncwarp();
  }
  return ok;
}

// x <- A^{-1} x with the factors of warp_lu (x in shared memory)
__device__ void warp_solve(const double* A, const int* piv, double* x, int n) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) {
        const double t = x[k];
        x[k] = x[p];
        x[p] = t;
      }
    }
  }
  __syncwarp();
  for (int k = 0; k < n; ++k) {
    const double xk = x[k];
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) x[i] -= A[i * n + k] * xk;
    __syncwarp();
  }
  // back substitution on b~ (x_k = b~_k / U_kk): b~_i -= U'_ik b~_k for i < k,
  // with U' = U scaled by its column pivots, then one scaling pass
  for (int k = n - 1; k > 0; --k) {
    const double bk = x[k];
    __syncwarp();
    for (int i = lane; i < k; i += 32) x[i] -= A[i * n + k] * bk;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) x[i] *= A[i * n + i];
  __syncwarp();
}

}  // namespace df
