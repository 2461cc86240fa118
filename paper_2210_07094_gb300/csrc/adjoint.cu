// Discrete adjoint of the RODAS4 chemistry substep (one cell per thread).
//
// Target: the gradient of
//   L = sum_c [ gT1_c T_c(dt) + sum_k gY1_kc Y_kc(dt) + gQ1_c qdot_c(dt) ]
// with respect to every cell's initial state (T, Y) and to ln A_j of every
// reaction, for the DISCRETE map the integrator computes, with its accepted
// step sequence h_0..h_{S-1} held fixed (the usual discrete-adjoint
// convention; Sandu et al., "Discrete adjoints of Rosenbrock methods").  The
// paper has no adjoint; this is the sensitivity / calibration extension of the
// chemistry substep of Sec. 2.3.
//
// Per accepted step, in reverse: recompute the stages K_s and the LU of
// W = I/(h gamma) - J(y) from the checkpoint (y_i, h_i), then with
// Kbar_s = m_s lambda (+ later-stage terms):
//   Rbar_s = W^{-T} Kbar_s
//   Kbar_j += (c_sj / h) Rbar_s                           (j < s)
//   Ybar_s = J(Y_s)^T Rbar_s,  lambda += Ybar_s,  Kbar_j += a_sj Ybar_s
//   thbar  += (df/dlnA)(Y_s)^T Rbar_s
//   lambda += d/de [J(y + e K_s)^T Rbar_s]               (W depends on y)
//   thbar  += d/de [(df/dlnA)(y + e K_s)^T Rbar_s]
// The directional derivatives come from forward-mode dual numbers through the
// same rate and Jacobian code as the integrator (exact, no differencing).
// qdot's gradient at the final state: n dual evaluations of the right-hand side.
//
// Cells are assigned statically (cell = global thread index) and the per-cell
// ln A gradients are summed over threads in a fixed order, then over blocks by a
// second kernel in a fixed order: the result is bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "rosenbrock.cuh"

namespace df {

static __constant__ RosTab c_tab_adj;
static bool g_adj_ready[64] = {false};

struct AdjArgs {
  const double* blob;
  MechDims d;
  int64_t ncells;
  const double* T0;
  const double* p;
  const double* Y0;
  double dt;
  double rtol, atolY, atolT, h0, hmin;
  int max_sub;
  int cap;  // checkpoints per cell
  const double* gT1;
  const double* gY1;
  const double* gQ1;
  double* gT0;
  double* gY0;
  int32_t* status;
  int32_t* nsub;
  double* ckpt;     // [ncells][cap][n + 1]: y_i then h_i
  double* partial;  // [gridDim.x][M]
  int stage_blob;
  // optional [cap][7n + n^2][ncells] (cell fastest, so a warp's accesses
  // coalesce): the accepted step's stage vectors K_s (6n), LU factors of W
  // (n^2) and row pivots (n), kept by the forward sweep so that the reverse
  // sweep need not recompute the step; null: the reverse sweep recomputes it
  double* stages;
  int hook_cp;  // 8 NS: the Dual cpR vector's offset (doubles, units of the block size)
};

// Per-thread shared-memory doubles.  Without KEEP (the reverse sweep
// recomputes each step): Dual C, wdot, gRT, hRT, cpR, sigma, v (14 NS) + W
// (n^2) + K, Kbar (12 n) + theta (M).  With KEEP (the forward sweep stores each
// accepted step's stages and LU factors in the workspace and the reverse sweep
// reads them there): the dual vectors, then a region of max(n^2, 6n + M) that
// holds Kbar and theta in the reverse sweep and W in the forward sweep; the
// forward sweep's K sits in the derivative halves of the dual vectors, unused
// until the reverse sweep (6n <= 7NS for NS >= 6).  In both, the ln A hook's
// scratch u, ud shares the Dual cpR vector (eval_vjp writes cpR only after its
// reaction loop, the one place that reads u), and its weights are the
// cotangent eval_vjp is given.  Less shared memory per thread, more warps per
// SM on the narrow FP64 pipe.
__host__ __device__ constexpr int adj_layout_doubles(int NS, int M, bool keep) {
  return keep ? 14 * NS + ((NS + 1) * (NS + 1) > 6 * (NS + 1) + M ? (NS + 1) * (NS + 1) : 6 * (NS + 1) + M)
              : 14 * NS + (NS + 1) * (NS + 1) + 12 * (NS + 1) + M;
}

__host__ __device__ constexpr bool adj_keep_possible(int NS) { return 6 * (NS + 1) <= 7 * NS; }

// read-only view of the stored stages in the workspace: element i at p[i * s],
// s = ncells (64-bit offsets)
struct GV {
  const double* p;
  int64_t s;
  __device__ __forceinline__ double operator[](int i) const { return p[(int64_t)i * s]; }
};

template <int NS, bool KEEP = false>
__global__ void __launch_bounds__(32, 1) k_adjoint_thread(AdjArgs a) {
  static_assert(!KEEP || 6 * (NS + 1) <= 7 * NS, "KEEP: the forward K must fit the dual derivative halves");
  constexpr int n = NS + 1;
  extern __shared__ double smem[];
  const int tid = threadIdx.x, stride = blockDim.x;
  double2* etab = reinterpret_cast<double2*>(smem);
  for (int i = tid; i < 64; i += stride) etab[i] = g_exp2_tab[i];
  int boff = 128;
  const double* blob = a.blob;
  if (a.stage_blob) {
    for (int i = tid; i < a.d.total; i += stride) smem[boff + i] = a.blob[i];
    blob = smem + boff;
    boff += (a.d.total + 1) & ~1;
  }
  __syncthreads();
  const MechView mv = make_view(blob, a.d, etab);
  const int M = a.d.M;
  double* base = smem + boff;
  // Dual vectors (value part at even offsets)
  Dual* dbase = reinterpret_cast<Dual*>(base) + tid;
  SVT<Dual> dC{dbase, stride}, dW{dbase + NS * stride, stride}, dG{dbase + 2 * NS * stride, stride},
      dH{dbase + 3 * NS * stride, stride}, dCp{dbase + 4 * NS * stride, stride},
      dS{dbase + 5 * NS * stride, stride}, dV{dbase + 6 * NS * stride, stride};
  // double views of the same storage
  double* vb = base + 2 * tid;
  SV C{vb, 2 * stride}, wd{vb + 2 * NS * stride, 2 * stride}, gRT{vb + 4 * NS * stride, 2 * stride},
      hRT{vb + 6 * NS * stride, 2 * stride}, cpR{vb + 8 * NS * stride, 2 * stride},
      sg{vb + 10 * NS * stride, 2 * stride}, vs{vb + 12 * NS * stride, 2 * stride};
  double* rest = base + (14 * NS) * stride + tid;
  SV Wv{rest, stride};  // the forward sweep's W (both layouts) and the recomputed one
  SV Kv = KEEP ? SV{vb + 1, 2 * stride} : SV{rest + n * n * stride, stride};
  const int kstride = KEEP ? 2 * stride : stride;  // stride of a stage vector inside Kv
  double* kb0 = KEEP ? rest : rest + (n * n + 6 * n) * stride;
  SV Kb{kb0, stride};
  SV th{kb0 + 6 * n * stride, stride};
  // the ln A hook's scratch: the Dual cpR vector (its value halves for the
  // double evaluation), at an offset the launch passes in: where the compiler
  // can see that the scratch and cpR coincide it schedules eval_vjp with
  // several hundred bytes of register spills
  SV uu{vb + a.hook_cp * stride, 2 * stride};
  SVT<Dual> uD{reinterpret_cast<Dual*>(vb + a.hook_cp * stride), stride};
  const int th_off = 14 * NS + (KEEP ? 6 * n : n * n + 12 * n);  // theta's offset (units of stride)
  const RosTab& tb = c_tab_adj;
  for (int j = 0; j < M; ++j) th[j] = 0.0;

  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + tid;
  if (cell < a.ncells) {
    double y[n];
    y[0] = a.T0[cell];
    bool ok = isfinite(y[0]) && y[0] > 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      y[1 + k] = a.Y0[(int64_t)k * a.ncells + cell];
      ok = ok && isfinite(y[1 + k]);
    }
    const double pc = 10.0 * a.p[cell];
    ok = ok && isfinite(pc) && pc > 0.0;
    int status = ok ? DF_CELL_OK : DF_CELL_NONFINITE;
    double* ck = a.ckpt + cell * (int64_t)a.cap * (n + 1);
    // ---- forward with checkpoints --------------------------------------
    double t = 0.0, h = fmin(a.h0, a.dt);
    int nacc = 0, nrej = 0;
    bool last_rej = false, done = !ok || !(a.dt > 0.0);
    StepState ss{0.0, 1.0};
    while (!done) {
      bool last = false;
      if (t + h >= a.dt) {
        h = a.dt - t;
        last = true;
      }
      double yold[n], ynew[n], en;
#pragma unroll
      for (int i = 0; i < n; ++i) yold[i] = y[i];
      int pv[n];
      const bool sok = ros_attempt<NS>(mv, tb, pc, y, h, a.rtol, a.atolY, a.atolT, C, wd, gRT, hRT, cpR, Wv, Kv,
                                       kstride, ynew, en, pv, nacc == 0 && nrej == 0, &last);
      const double hstep = h;  // the step actually taken (the first one may be cut)
      const int before = nacc;
      step_control(tb, sok, en, last, a.dt, y, ynew, t, h, nacc, nrej, last_rej, done, ss);
      if (nacc > before) {
        if (nacc > a.cap) {
          status = DF_CELL_MAXSTEPS;
          done = true;
        } else {
          double* slot = ck + (int64_t)(nacc - 1) * (n + 1);
#pragma unroll
          for (int i = 0; i < n; ++i) slot[i] = yold[i];
          slot[n] = hstep;
          if (a.stages) {
            double* sp = a.stages + (int64_t)(nacc - 1) * (7 * n + n * n) * a.ncells + cell;
            for (int i = 0; i < 6 * n; ++i) sp[i * a.ncells] = Kv[i];
            for (int i = 0; i < n * n; ++i) sp[(6 * n + i) * a.ncells] = Wv[i];
#pragma unroll
            for (int i = 0; i < n; ++i) sp[(6 * n + n * n + i) * a.ncells] = (double)pv[i];
          }
        }
      }
      if (!done) {
        if (nacc + nrej >= a.max_sub) {
          status = DF_CELL_MAXSTEPS;
          done = true;
        } else if (h < a.hmin) {
          status = DF_CELL_HMIN;
          done = true;
        }
      }
    }
    if (KEEP) {  // the forward sweep's W overlaid theta, u, ud and Kbar
      for (int j = 0; j < M; ++j) th[j] = 0.0;
    }
    double lam[n];
    if (status == DF_CELL_OK) {
      // ---- cotangent at the final state --------------------------------
      lam[0] = a.gT1 ? a.gT1[cell] : 0.0;
#pragma unroll
      for (int k = 0; k < NS; ++k) lam[1 + k] = a.gY1 ? a.gY1[(int64_t)k * a.ncells + cell] : 0.0;
      const double gq = a.gQ1 ? a.gQ1[cell] : 0.0;
      if (gq != 0.0) {
        // Q = -sum_k H_k wdot_k = f_T rho cp, so dQ/dy = rho cp (row 0 of J) +
        // f_T d(rho cp)/dy: one transposed product with e_T (which also adds the
        // ln A terms of Q through the hook) and the closed-form derivative of
        // rho cp = (p/T) A/B, A = sum_k Y_k cp_k/(R W_k), B = sum_k Y_k/W_k
        ThetaHook hk{2, gq, th, uu, uD};
        double e0[n], b0[n], fq[n];
#pragma unroll
        for (int i = 0; i < n; ++i) e0[i] = i == 0 ? 1.0 : 0.0;
        eval_vjp<NS, double>(mv, pc, y, e0, b0, fq, C, wd, gRT, hRT, cpR, sg, vs, &hk);
        const double T = y[0];
        double A = 0.0, B = 0.0, dA = 0.0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const double* c7 = mv.sp + SP_REC * k + 2;
          const double iW = mv.sp[SP_REC * k + 1];
          A += y[1 + k] * cpR[k] * iW;
          B += y[1 + k] * iW;
          dA += y[1 + k] * (c7[1] + T * (2.0 * c7[2] + T * (3.0 * c7[3] + T * 4.0 * c7[4]))) * iW;
        }
        const double rcp = pc / T * A / B;
        const double w = gq * 0.1;
        lam[0] += w * (rcp * b0[0] + fq[0] * pc * (dA / (T * B) - A / (T * T * B)));
#pragma unroll
        for (int k = 0; k < NS; ++k)
          lam[1 + k] += w * (rcp * b0[1 + k] + fq[0] * (pc / T) * mv.sp[SP_REC * k + 1] * (cpR[k] - A / B) / B);
      }
      // ---- reverse sweep over the accepted steps -----------------------
      for (int istep = nacc - 1; istep >= 0; --istep) {
        const double* slot = ck + (int64_t)istep * (n + 1);
        double yi[n], ynew[n], en;
#pragma unroll
        for (int i = 0; i < n; ++i) yi[i] = slot[i];
        double hs = slot[n];
        int piv[n];
        // this step's stages and LU factors: read in place from the workspace
        // (KEEP), copied from it, or recomputed
        typedef typename std::conditional<KEEP, GV, SV>::type StageView;
        StageView Wr, Kr;
        if constexpr (KEEP) {
          const double* sp = a.stages + (int64_t)istep * (7 * n + n * n) * a.ncells + cell;
          Kr = GV{sp, a.ncells};
          Wr = GV{sp + (int64_t)6 * n * a.ncells, a.ncells};
#pragma unroll
          for (int i = 0; i < n; ++i) piv[i] = (int)sp[(int64_t)(6 * n + n * n + i) * a.ncells];
        } else {
          if (a.stages) {  // the forward sweep kept this step's stages and factors
            const double* sp = a.stages + (int64_t)istep * (7 * n + n * n) * a.ncells + cell;
            for (int i = 0; i < 6 * n; ++i) Kv[i] = sp[i * a.ncells];
            for (int i = 0; i < n * n; ++i) Wv[i] = sp[(6 * n + i) * a.ncells];
#pragma unroll
            for (int i = 0; i < n; ++i) piv[i] = (int)sp[(6 * n + n * n + i) * a.ncells];
          } else {
            ros_attempt<NS>(mv, tb, pc, yi, hs, a.rtol, a.atolY, a.atolT, C, wd, gRT, hRT, cpR, Wv, Kv, stride, ynew,
                            en, piv);
          }
          Kr = Kv;
          Wr = Wv;
        }
        const double ih = 1.0 / hs;
        double yb[n];
#pragma unroll
        for (int i = 0; i < n; ++i) yb[i] = lam[i];
        for (int s = 0; s < tb.s; ++s)
#pragma unroll
          for (int i = 0; i < n; ++i) Kb[s * n + i] = tb.m[s] * lam[i];
        for (int s = tb.s - 1; s >= 0; --s) {
          // Rbar = W^{-T} Kbar_s  (W = P^T L U: U^T w = b, L^T z = w, x = P^T z)
          double r[n];
#pragma unroll
          for (int i = 0; i < n; ++i) r[i] = Kb[s * n + i];
#pragma unroll
          for (int k = 0; k < n; ++k) {
            double acc = r[k];
#pragma unroll
            for (int j = 0; j < k; ++j) acc -= Wr[j * n + k] * r[j];
            r[k] = acc * Wr[k * n + k];
          }
#pragma unroll
          for (int k = n - 1; k >= 0; --k) {
            double acc = r[k];
#pragma unroll
            for (int j = k + 1; j < n; ++j) acc -= Wr[j * n + k] * r[j];
            r[k] = acc;
          }
#pragma unroll
          for (int k = n - 1; k >= 0; --k) {
            const int pk = piv[k];
#pragma unroll
            for (int i = k + 1; i < n; ++i)
              if (i == pk) {
                const double tmp = r[k];
                r[k] = r[i];
                r[i] = tmp;
              }
          }
          for (int j = 0; j < s; ++j)
#pragma unroll
            for (int i = 0; i < n; ++i) Kb[j * n + i] += (tb.c[s][j] * ih) * r[i];
          // F_s = f(Y_s): Ybar_s = J(Y_s)^T Rbar, theta += (df/dlnA)(Y_s)^T Rbar
          double ysg[n], fs[n];
#pragma unroll
          for (int i = 0; i < n; ++i) {
            double acc = yi[i];
            for (int j = 0; j < s; ++j) acc += tb.a[s][j] * Kr[j * n + i];
            ysg[i] = acc;
          }
          // the first stage is evaluated at the step's start, where the dual
          // evaluation below is: its value part stands in for this product
          if (s > 0) {
            ThetaHook hk{1, 0.0, th, uu, uD};
            double bj[n];
            eval_vjp<NS, double>(mv, pc, ysg, r, bj, fs, C, wd, gRT, hRT, cpR, sg, vs, &hk);
#pragma unroll
            for (int jc = 0; jc < n; ++jc) {
              yb[jc] += bj[jc];
              for (int j = 0; j < s; ++j) Kb[j * n + jc] += tb.a[s][j] * bj[jc];
            }
          }
          // W depends on y through J(y): d/de [J(y + e K_s)^T Rbar] and the ln A analogue
          {
            Dual yd[n], fd[n], bd[n];
#pragma unroll
            for (int i = 0; i < n; ++i) yd[i] = Dual(yi[i], Kr[s * n + i]);
            ThetaHook hk{1, 0.0, th, uu, uD, s == 0 ? 1 : 0};
            eval_vjp<NS, Dual>(mv, pc, yd, r, bd, fd, dC, dW, dG, dH, dCp, dS, dV, &hk);
            if (s == 0) {
#pragma unroll
              for (int jc = 0; jc < n; ++jc) yb[jc] += bd[jc].v;
            }
#pragma unroll
            for (int jc = 0; jc < n; ++jc) yb[jc] += bd[jc].d;
          }
        }
#pragma unroll
        for (int i = 0; i < n; ++i) lam[i] = yb[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < n; ++i) lam[i] = 0.0;
      for (int j = 0; j < M; ++j) th[j] = 0.0;
    }
    if (a.gT0) a.gT0[cell] = lam[0];
    if (a.gY0) {
#pragma unroll
      for (int k = 0; k < NS; ++k) a.gY0[(int64_t)k * a.ncells + cell] = lam[1 + k];
    }
    a.status[cell] = status;
    if (a.nsub) a.nsub[cell] = nacc;
  }
  // fixed-order sum of the per-thread ln A gradients of this block
  __syncthreads();
  if (a.partial) {
    for (int j = tid; j < M; j += stride) {
      double acc = 0.0;
      for (int q = 0; q < stride; ++q) acc += base[(size_t)(th_off + j) * stride + q];
      a.partial[(int64_t)blockIdx.x * M + j] = acc;
    }
  }
}

__global__ void k_adjoint_reduce(const double* partial, int64_t nblocks, int M, double* g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  double acc = 0.0;
  for (int64_t b = 0; b < nblocks; ++b) acc += partial[b * M + j];
  g[j] = acc;
}

static int ensure_adj_table(int dev) {
  if (dev < 0 || dev >= 64) return DF_OK;
  if (g_adj_ready[dev]) return DF_OK;
  RosTab t = make_rodas4();
  if (!t.stiff_acc) return set_error(DF_EUNSUPPORTED, "RODAS4 table not stiffly accurate");  // ros_attempt relies on it
  int rc = cuda_check(cudaMemcpyToSymbol(c_tab_adj, &t, sizeof(t)), "upload RODAS4 table");
  if (!rc) g_adj_ready[dev] = true;
  return rc;
}

// Threads (cells) per block: as many, up to one warp, as let four blocks share
// an SM.  Each of an SM's four sub-partitions has its own FP64 unit, and a
// thread's workspace is too large for two warps per sub-partition, so a
// fourth block keeps the fourth unit busy: four blocks of 31 threads do more
// work than three of 32 (the 9-species layout: 226 doubles per thread).  Both
// layouts use the count of the one with stored stages, so that their per-block
// ln A partial sums group the cells alike and the gradients agree bitwise.
static int adj_threads(const df_mech* m) {
  const int NS = m->dims.N;
  const long per = adj_layout_doubles(NS, m->dims.M, adj_keep_possible(NS));
  const long budget = (long)m->smem_per_sm / 4 - (long)m->smem_reserved_per_block;  // bytes per block
  const long t = (budget / (long)sizeof(double) - 128) / per;  // 128: the exp table
  return t >= 16 && t < 32 ? (int)t : 32;
}

// Workspace: checkpoints [ncells][cap][n + 1], then the per-block ln A
// partials, then (with_stages) the stored stages [cap][7n + n^2][ncells].
// Every product and sum is overflow-checked: a size that does not fit in
// size_t is reported, never wrapped to a small one.
static bool adj_compact_doubles(const df_mech* m, int64_t ncells, int cap, size_t* out) {
  if (ncells < 0 || cap < 1) return false;
  const size_t n = (size_t)m->dims.N + 1;
  const size_t threads = (size_t)adj_threads(m);
  const size_t blocks = ((size_t)ncells + threads - 1) / threads;
  size_t ck = 0, part = 0;
  if (__builtin_mul_overflow((size_t)ncells, (size_t)cap, &ck) || __builtin_mul_overflow(ck, n + 1, &ck) ||
      __builtin_mul_overflow(blocks, (size_t)m->dims.M, &part) || __builtin_add_overflow(ck, part, out))
    return false;
  return true;
}

bool adjoint_workspace_bytes(const df_mech* m, int64_t ncells, int cap, bool with_stages, size_t* bytes) {
  size_t d = 0;
  if (!adj_compact_doubles(m, ncells, cap, &d)) return false;
  if (with_stages) {
    const size_t n = (size_t)m->dims.N + 1;
    size_t st = 0;
    if (__builtin_mul_overflow((size_t)ncells, (size_t)cap, &st) || __builtin_mul_overflow(st, 7 * n + n * n, &st) ||
        __builtin_add_overflow(d, st, &d))
      return false;
  }
  if (__builtin_mul_overflow(d, sizeof(double), &d) || __builtin_add_overflow(d, (size_t)256, &d)) return false;
  *bytes = d;
  return true;
}

template <int NS, bool KEEP>
static int adjoint_dispatch_layout(const df_mech* m, AdjArgs a, cudaStream_t st, double* g_lnA) {
  const int threads = adj_threads(m);
  const size_t per = (size_t)adj_layout_doubles(NS, m->dims.M, KEEP) * threads;
  a.hook_cp = 8 * NS;
  // the mechanism is staged in shared memory unless that leaves fewer blocks
  // on an SM than reading it through L1
  const size_t sm_staged = sizeof(double) * (128 + ((m->dims.total + 1) & ~1) + per);
  const size_t sm_plain = sizeof(double) * (128 + per);
  auto blocks_per_sm = [m](size_t b) {
    return b > m->max_smem_optin ? (size_t)0 : m->smem_per_sm / (b + m->smem_reserved_per_block);
  };
  a.stage_blob = blocks_per_sm(sm_staged) >= blocks_per_sm(sm_plain) ? 1 : 0;
  const size_t sm = a.stage_blob ? sm_staged : sm_plain;
  if (sm > m->max_smem_optin) return set_error(DF_EUNSUPPORTED, "adjoint workspace exceeds shared memory");
  auto kf = k_adjoint_thread<NS, KEEP>;
  int rc = cuda_check(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                      "set adjoint shared memory");
  if (rc) return rc;
  const int64_t blocks = (a.ncells + threads - 1) / threads;
  kf<<<(unsigned)blocks, threads, sm, st>>>(a);
  rc = cuda_check(cudaGetLastError(), "adjoint kernel launch");
  if (rc) return rc;
  if (g_lnA && m->dims.M > 0) {
    k_adjoint_reduce<<<(m->dims.M + 127) / 128, 128, 0, st>>>(a.partial, blocks, m->dims.M, g_lnA);
    rc = cuda_check(cudaGetLastError(), "adjoint reduction launch");
  }
  return rc;
}

// the smaller layout when the stages are kept in the workspace and the
// forward sweep's stage vectors fit the dual derivative halves
template <int NS>
static int adjoint_dispatch(const df_mech* m, AdjArgs a, cudaStream_t st, double* g_lnA) {
  if constexpr (adj_keep_possible(NS)) {
    if (a.stages) return adjoint_dispatch_layout<NS, true>(m, a, st, g_lnA);
  }
  return adjoint_dispatch_layout<NS, false>(m, a, st, g_lnA);
}

int launch_adjoint(const df_mech* m, int64_t ncells, const double* T0, const double* p, const double* Y0,
                   double dt, const df_integ_opts& o, int cap, const double* gT1, const double* gY1,
                   const double* gQ1, double* gT0, double* gY0, double* g_lnA, int32_t* status, int32_t* nsub,
                   void* ws, size_t ws_bytes, bool allow_stages, cudaStream_t st) {
  if (o.method != 0) return set_error(DF_EUNSUPPORTED, "the adjoint is built for RODAS4 (method 0)");
  if (ncells > ((int64_t)1 << 31)) return set_error(DF_EINVAL, "adjoint: ncells must be in [0, 2^31]");
  size_t need = 0, full = 0;
  if (!adjoint_workspace_bytes(m, ncells, cap, false, &need))
    return set_error(DF_EWORKSPACE, "adjoint: ncells * max_steps checkpoints overflow the address space");
  if (!ws || ws_bytes < need) return set_error(DF_EWORKSPACE, "adjoint workspace too small");
  const bool keep_stages =
      allow_stages && adjoint_workspace_bytes(m, ncells, cap, true, &full) && ws_bytes >= full;
  int rc = ensure_adj_table(m->device);
  if (rc) return rc;
  const int n = m->dims.N + 1;
  AdjArgs a;
  memset(&a, 0, sizeof(a));
  a.blob = m->blob_dev;
  a.d = m->dims;
  a.ncells = ncells;
  a.T0 = T0;
  a.p = p;
  a.Y0 = Y0;
  a.dt = dt;
  a.rtol = o.rtol;
  a.atolY = o.atol_Y;
  a.atolT = o.atol_T;
  a.h0 = o.h0;
  a.hmin = o.h_min;
  a.max_sub = o.max_substeps;
  a.cap = cap;
  a.gT1 = gT1;
  a.gY1 = gY1;
  a.gQ1 = gQ1;
  a.gT0 = gT0;
  a.gY0 = gY0;
  a.status = status;
  a.nsub = nsub;
  size_t compact = 0;
  adj_compact_doubles(m, ncells, cap, &compact);  // fits: checked above
  a.ckpt = static_cast<double*>(ws);
  a.partial = static_cast<double*>(ws) + (size_t)ncells * cap * (n + 1);
  a.stages = keep_stages ? static_cast<double*>(ws) + compact : nullptr;
  switch (m->dims.N) {
    case 3:
      return adjoint_dispatch<3>(m, a, st, g_lnA);
    case 9:
      return adjoint_dispatch<9>(m, a, st, g_lnA);
    default:
      return set_error(DF_EUNSUPPORTED, "the adjoint is built for 3- and 9-species mechanisms");
  }
}

}  // namespace df

// ---------------------------------------------------------------------------
// df_chem_adjoint_static: the adjoint without any allocation by the library or
// the caller for its scratch.
//
// Some callers cannot call cudaMalloc when they need a gradient: a host
// application whose device memory is owned by a pool or another framework that
// must not be bypassed, or a real-time loop that forbids allocation after
// start-up.  This entry point
// keeps the adjoint's scratch (the per-cell checkpoints and the per-block ln A
// partial sums) in one file-scope device array instead, so the caller only
// passes its inputs and outputs.
// ---------------------------------------------------------------------------
namespace df {

// 4 MiB of scratch; every GPU that loads the library holds it until exit
constexpr size_t ADJ_STATIC_BYTES = (size_t)4 << 20;
static __device__ __align__(256) double g_adj_static_scratch[ADJ_STATIC_BYTES / sizeof(double)];

static std::mutex g_adj_static_mu;
static void* g_adj_static_ptr[64] = {nullptr};

// Host-side address of the scratch array on the current device.  The array's
// name in host code is only a host-side stand-in, so its device address is
// looked up once per device, with that device current.
static int adj_static_scratch(void** out) {
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= 64) return set_error(DF_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_adj_static_mu);
  if (!g_adj_static_ptr[dev]) {
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_adj_static_scratch), "cudaGetSymbolAddress (adjoint scratch)");
    if (rc) return rc;
    g_adj_static_ptr[dev] = p;
  }
  *out = g_adj_static_ptr[dev];
  return DF_OK;
}

}  // namespace df

extern "C" int df_chem_adjoint_static(const df_mech* m, int64_t ncells, const double* T0, const double* p,
                                      const double* Y0, double dt, const df_integ_opts* opts, int32_t max_steps,
                                      const double* gT1, const double* gY1, const double* gQ1, double* gT0,
                                      double* gY0, double* g_lnA, int32_t* status, int32_t* nsub,
                                      df_stream_t stream) {
  using namespace df;
  const char* fn = "df_chem_adjoint_static";
  df_integ_opts o;
  int rc = check_adjoint_call(fn, m, ncells, dt, max_steps, T0, p, Y0, gT1, gY1, gQ1, gT0, gY0, g_lnA, status, nsub,
                              opts, &o);
  if (rc || ncells == 0) return rc;
  size_t need = 0;
  if (!adjoint_workspace_bytes(m, ncells, max_steps, false, &need) || need > ADJ_STATIC_BYTES)
    return set_error(DF_EWORKSPACE,
                     std::string(fn) + ": ncells * max_steps * (N + 2) checkpoints plus the ln A partials need " +
                         (need > ADJ_STATIC_BYTES ? std::to_string(need) + " bytes" : std::string("more bytes than "
                         "size_t holds")) + ", more than the fixed 4 MiB scratch; use df_chem_adjoint with a "
                         "caller-provided workspace");
  void* ws = nullptr;
  rc = adj_static_scratch(&ws);
  if (rc) return rc;
  return launch_adjoint(m, ncells, T0, p, Y0, dt, o, max_steps, gT1, gY1, gQ1, gT0, gY0, g_lnA, status, nsub, ws,
                        ADJ_STATIC_BYTES, false, (cudaStream_t)stream);
}
