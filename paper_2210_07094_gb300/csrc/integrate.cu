// Kernels of the chemistry substep: RHS / Jacobian diagnostics and the
// persistent adaptive Rosenbrock integrator (one cell per thread, N <= 16).
//
// The integrator stands in for the CVODE call of Sec. 2.3: every cell advances
// its own stiff kinetics ODE over [0, dt].  Method: Rosenbrock schemes in the
// form of Sandu et al. (1997) -- (I/(h gamma) - J) K_i = f(y + sum_j a_ij K_j)
// + sum_j (c_ij/h) K_j,  y_new = y + sum_i m_i K_i, err = sum_i e_i K_i --
// with the RODAS4 coefficients of Hairer & Wanner (Solving ODEs II, Sec. VI.4)
// or the RODAS3 coefficients of Sandu et al. (1997); analytic Jacobian; dense
// LU with partial pivoting per cell in shared memory.
//
// Scheduling: a persistent grid sized to the SMs; each lane takes a new cell
// from a device work counter as soon as its cell is finished (warp-aggregated
// atomics), so cells of very uneven stiffness keep all lanes busy.  This is
// the GPU analogue of the chemistry load balancing of Sec. 3.2 (LoadBalancer).
#include <algorithm>
#include <cmath>

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
};

__constant__ RosTab c_tab[2];

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
  return t;
}

static bool g_tab_ready[64] = {false};

static int ensure_tables(int dev) {
  if (dev < 0 || dev >= 64) return DF_OK;
  if (g_tab_ready[dev]) return DF_OK;
  RosTab t[2] = {make_rodas4(), make_rodas3()};
  int rc = cuda_check(cudaMemcpyToSymbol(c_tab, t, sizeof(t)), "upload Rosenbrock tables");
  if (rc == DF_OK) g_tab_ready[dev] = true;
  return rc;
}

struct IntegArgs {
  const double* blob;
  MechDims d;
  int64_t ncells;
  double* T;
  const double* p;
  double* Y;
  double dt;
  double rtol, atolY, atolT, h0, hmin;
  int max_sub;
  int method;
  int32_t* status;
  int32_t* nsub;
  const int32_t* order;            // optional permutation of cell indices
  unsigned long long* counters;    // [0] next cell, [1] accepted, [2] rejected
  int stage_blob;                  // 1: copy the blob into shared memory
};

constexpr unsigned FULL = 0xffffffffu;

// per-thread shared-memory doubles of the thread path
template <int NS>
__host__ __device__ constexpr int thread_ws_doubles() {
  return 5 * NS + (NS + 1) * (NS + 1) + 6 * (NS + 1);
}

__host__ __device__ inline int blob_smem_doubles(const MechDims& d) { return (d.total + 1) & ~1; }

template <int NS>
__global__ void __launch_bounds__(128, 1) k_integrate_thread(IntegArgs a) {
  constexpr int n = NS + 1;
  extern __shared__ double smem[];
  const int tid = threadIdx.x;
  const int stride = blockDim.x;
  const double* blob = a.blob;
  int boff = 0;
  if (a.stage_blob) {
    for (int i = tid; i < a.d.total; i += stride) smem[i] = a.blob[i];
    blob = smem;
    boff = blob_smem_doubles(a.d);
    __syncthreads();
  }
  const MechView mv = make_view(blob, a.d);
  double* ws = smem + boff + tid;
  SV C{ws, stride};
  SV wdot{ws + NS * stride, stride};
  SV gRT{ws + 2 * NS * stride, stride};
  SV hRT{ws + 3 * NS * stride, stride};
  SV cpR{ws + 4 * NS * stride, stride};
  SV Jv{ws + 5 * NS * stride, stride};
  SV Kv{ws + (5 * NS + n * n) * stride, stride};
  const RosTab& tb = c_tab[a.method];
  const int lane = tid & 31;

  int64_t cell = -1;
  bool exhausted = false, done = false, last_rej = false;
  int status = 0, nacc = 0, nrej = 0;
  double y[n];
  double t = 0.0, h = 0.0;
  unsigned long long tot_acc = 0, tot_rej = 0;

  for (;;) {
    // finished cell: store
    if (cell >= 0 && done) {
      if (status == DF_CELL_OK) {
        a.T[cell] = y[0];
#pragma unroll
        for (int k = 0; k < NS; ++k) a.Y[(int64_t)k * a.ncells + cell] = y[1 + k];
      }
      a.status[cell] = status;
      if (a.nsub) a.nsub[cell] = nacc;
      tot_acc += nacc;
      tot_rej += nrej;
      cell = -1;
    }
    // lane refill from the device work counter
    const bool want = (cell < 0) && !exhausted;
    const unsigned m = __ballot_sync(FULL, want);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&a.counters[0], (unsigned long long)__popc(m));
      base = __shfl_sync(FULL, base, leader);
      if (want) {
        const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
        if (idx < (unsigned long long)a.ncells) {
          cell = a.order ? (int64_t)a.order[idx] : (int64_t)idx;
          y[0] = a.T[cell];
          bool ok = isfinite(y[0]) && y[0] > 0.0;
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            y[1 + k] = a.Y[(int64_t)k * a.ncells + cell];
            ok = ok && isfinite(y[1 + k]);
          }
          const double pc = a.p[cell];
          ok = ok && isfinite(pc) && pc > 0.0;
          t = 0.0;
          h = fmin(a.h0, a.dt);
          nacc = nrej = 0;
          last_rej = false;
          status = ok ? DF_CELL_OK : DF_CELL_NONFINITE;
          done = !ok || !(a.dt > 0.0);
        } else {
          exhausted = true;
        }
      }
    }
    if (__ballot_sync(FULL, cell >= 0 || !exhausted) == 0) break;
    if (cell < 0 || done) continue;

    // ---- one substep attempt ------------------------------------------------
    const double pc = 10.0 * a.p[cell];  // Pa -> dyn/cm^2
    bool last = false;
    if (t + h >= a.dt) {
      h = a.dt - t;
      last = true;
    }
    // f(y) and J(y); W = I/(h gamma) - J factorised in place
    double fs[n];
    eval_thread<NS, true>(mv, pc, y, fs, C, wdot, gRT, hRT, cpR, Jv);
    const double hgi = 1.0 / (h * tb.gamma);
#pragma unroll
    for (int i = 0; i < n; ++i) {
#pragma unroll
      for (int j = 0; j < n; ++j) Jv[i * n + j] = (i == j ? hgi : 0.0) - Jv[i * n + j];
    }
    int piv[n];
    bool ok = lu_factor<n>(Jv, piv);
    const double ih = 1.0 / h;
    double ys[n];
    for (int s = 0; s < tb.s; ++s) {
      if (s > 0 && tb.newf[s]) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
          double acc = y[i];
          for (int j = 0; j < s; ++j) acc += tb.a[s][j] * Kv[j * n + i];
          ys[i] = acc;
        }
        eval_thread<NS, false>(mv, pc, ys, fs, C, wdot, gRT, hRT, cpR, Jv);
      }
      // stage right-hand side, solved in place in the K slot of this stage
      SV Ks{&Kv[s * n], stride};
#pragma unroll
      for (int i = 0; i < n; ++i) {
        double acc = fs[i];
        for (int j = 0; j < s; ++j) acc += (tb.c[s][j] * ih) * Kv[j * n + i];
        Ks[i] = acc;
      }
      lu_solve<n>(Jv, piv, Ks);
    }
    // new state and weighted RMS norm of the embedded error estimate
    double en = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      double yn = y[i], e = 0.0;
      for (int s = 0; s < tb.s; ++s) {
        const double kv = Kv[s * n + i];
        yn += tb.m[s] * kv;
        e += tb.e[s] * kv;
      }
      ys[i] = yn;
      const double sc = (i == 0 ? a.atolT : a.atolY) + a.rtol * fmax(fabs(y[i]), fabs(yn));
      const double r = e / sc;
      en += r * r;
    }
    en = sqrt(en / n);
    ok = ok && isfinite(en);
    if (ok && en <= 1.0) {
#pragma unroll
      for (int i = 0; i < n; ++i) y[i] = ys[i];
      t = last ? a.dt : t + h;
      ++nacc;
      double fac = 0.9 * pow(fmax(en, 1e-10), -1.0 / tb.elo);
      fac = fmin(last_rej ? 1.0 : 6.0, fmax(0.2, fac));
      h *= fac;
      last_rej = false;
      if (t >= a.dt) done = true;
    } else {
      ++nrej;
      const double fac = ok ? fmax(0.2, 0.9 * pow(en, -1.0 / tb.elo)) : 0.25;
      h *= fac;
      last_rej = true;
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
  // statistics: one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot_acc += __shfl_down_sync(FULL, tot_acc, o);
    tot_rej += __shfl_down_sync(FULL, tot_rej, o);
  }
  if (lane == 0) {
    atomicAdd(&a.counters[1], tot_acc);
    atomicAdd(&a.counters[2], tot_rej);
  }
}

// ----------------------------------------------------------------------------
// diagnostics: f and J per cell (one thread per cell)
// ----------------------------------------------------------------------------
struct EvalArgs {
  const double* blob;
  MechDims d;
  int64_t ncells;
  const double* T;
  const double* p;
  const double* Y;
  double* dydt;
  double* qdot;
  double* J;
  int stage_blob;
};

template <int NS, bool WITH_J>
__global__ void __launch_bounds__(128) k_eval_thread(EvalArgs a) {
  constexpr int n = NS + 1;
  extern __shared__ double smem[];
  const int tid = threadIdx.x, stride = blockDim.x;
  const double* blob = a.blob;
  int boff = 0;
  if (a.stage_blob) {
    for (int i = tid; i < a.d.total; i += stride) smem[i] = a.blob[i];
    blob = smem;
    boff = blob_smem_doubles(a.d);
    __syncthreads();
  }
  const MechView mv = make_view(blob, a.d);
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + tid;
  if (c >= a.ncells) return;
  double* ws = smem + boff + tid;
  SV C{ws, stride}, wdot{ws + NS * stride, stride}, gRT{ws + 2 * NS * stride, stride},
      hRT{ws + 3 * NS * stride, stride}, cpR{ws + 4 * NS * stride, stride}, Jv{ws + 5 * NS * stride, stride};
  double y[n], f[n];
  y[0] = a.T[c];
#pragma unroll
  for (int k = 0; k < NS; ++k) y[1 + k] = a.Y[(int64_t)k * a.ncells + c];
  const double q = eval_thread<NS, WITH_J>(mv, 10.0 * a.p[c], y, f, C, wdot, gRT, hRT, cpR, Jv);
  if (a.dydt) {
#pragma unroll
    for (int i = 0; i < n; ++i) a.dydt[(int64_t)i * a.ncells + c] = f[i];
  }
  if (a.qdot) a.qdot[c] = 0.1 * q;  // erg/(cm^3 s) -> W/m^3
  if (WITH_J) {
    double* out = a.J + c * n * n;
#pragma unroll
    for (int i = 0; i < n * n; ++i) out[i] = Jv[i];
  }
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
namespace {

template <int NS>
size_t thread_smem_bytes(const MechDims& d, int threads, bool stage) {
  return sizeof(double) * ((stage ? blob_smem_doubles(d) : 0) + (size_t)thread_ws_doubles<NS>() * threads);
}

template <int NS>
int eval_dispatch(const df_mech* m, int64_t ncells, const double* T, const double* p,
                  const double* Y, double* dydt, double* qdot, double* J, cudaStream_t st) {
  EvalArgs a{m->blob_dev, m->dims, ncells, T, p, Y, dydt, qdot, J, 1};
  const int threads = 64;
  size_t sm = thread_smem_bytes<NS>(m->dims, threads, true);
  if (sm > m->max_smem_optin) {
    a.stage_blob = 0;
    sm = thread_smem_bytes<NS>(m->dims, threads, false);
  }
  const int64_t blocks = (ncells + threads - 1) / threads;
  if (J) {
    auto kf = k_eval_thread<NS, true>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<(unsigned)blocks, threads, sm, st>>>(a);
  } else {
    auto kf = k_eval_thread<NS, false>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<(unsigned)blocks, threads, sm, st>>>(a);
  }
  return cuda_check(cudaGetLastError(), "chemistry evaluation kernel");
}

template <int NS>
int integrate_dispatch(df_mech* m, const IntegArgs& a0, cudaStream_t st, int threads, int bps) {
  IntegArgs a = a0;
  a.stage_blob = 1;
  size_t sm = thread_smem_bytes<NS>(m->dims, threads, true);
  if (sm > m->max_smem_optin) {
    a.stage_blob = 0;
    sm = thread_smem_bytes<NS>(m->dims, threads, false);
  }
  if (sm > m->max_smem_optin)
    return set_error(DF_EUNSUPPORTED, "integrator shared memory exceeds the per-block limit");
  auto kf = k_integrate_thread<NS>;
  int rc = cuda_check(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                      "set integrator shared memory");
  if (rc) return rc;
  int occ = 0;
  rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf, threads, sm), "occupancy");
  if (rc) return rc;
  if (occ < 1) return set_error(DF_EUNSUPPORTED, "integrator launch shape does not fit on an SM");
  const int per_sm = bps > 0 ? std::min(bps, occ) : occ;
  int64_t blocks = (int64_t)m->num_sms * per_sm;
  const int64_t need = (a.ncells + threads - 1) / threads;
  if (blocks > need) blocks = std::max<int64_t>(1, need);
  rc = cuda_check(cudaMemsetAsync(m->counters, 0, 4 * sizeof(unsigned long long), st), "reset work counter");
  if (rc) return rc;
  kf<<<(unsigned)blocks, threads, sm, st>>>(a);
  return cuda_check(cudaGetLastError(), "integrator kernel launch");
}

}  // namespace

#define DF_THREAD_NS_LIST(X) X(3) X(9)

int launch_rhs(const df_mech* m, int64_t ncells, const double* T, const double* p,
               const double* Y, double* dydt, double* qdot, cudaStream_t st) {
  switch (m->dims.N) {
#define X(NS) \
  case NS:    \
    return eval_dispatch<NS>(m, ncells, T, p, Y, dydt, qdot, nullptr, st);
    DF_THREAD_NS_LIST(X)
#undef X
    default:
      return set_error(DF_EUNSUPPORTED, "no kernel built for this species count");
  }
}

int launch_jacobian(const df_mech* m, int64_t ncells, const double* T, const double* p,
                    const double* Y, double* J, cudaStream_t st) {
  switch (m->dims.N) {
#define X(NS) \
  case NS:    \
    return eval_dispatch<NS>(m, ncells, T, p, Y, nullptr, nullptr, J, st);
    DF_THREAD_NS_LIST(X)
#undef X
    default:
      return set_error(DF_EUNSUPPORTED, "no kernel built for this species count");
  }
}

int launch_integrate(df_mech* m, int64_t ncells, double* T, const double* p, double* Y,
                     double dt, const df_integ_opts& o, int32_t* status, int32_t* nsub,
                     cudaStream_t st) {
  int rc = ensure_tables(m->device);
  if (rc) return rc;
  IntegArgs a;
  memset(&a, 0, sizeof(a));
  a.blob = m->blob_dev;
  a.d = m->dims;
  a.ncells = ncells;
  a.T = T;
  a.p = p;
  a.Y = Y;
  a.dt = dt;
  a.rtol = o.rtol;
  a.atolY = o.atol_Y;
  a.atolT = o.atol_T;
  a.h0 = o.h0;
  a.hmin = o.h_min;
  a.max_sub = o.max_substeps;
  a.method = o.method;
  a.status = status;
  a.nsub = nsub;
  a.order = nullptr;
  a.counters = m->counters;
  const int threads = o.block_threads > 0 ? o.block_threads : 64;
  const int bps = o.blocks_per_sm;
  switch (m->dims.N) {
#define X(NS) \
  case NS:    \
    return integrate_dispatch<NS>(m, a, st, threads, bps);
    DF_THREAD_NS_LIST(X)
#undef X
    default:
      return set_error(DF_EUNSUPPORTED, "no integrator built for this species count");
  }
}

__global__ void k_set_lnA(double* blob, int off_rx, int M, const double* lnA) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < M) blob[off_rx + RX_REC * j] = lnA[j];
}

int launch_set_lnA(df_mech* m, const double* lnA, cudaStream_t st) {
  const int M = m->dims.M;
  if (M == 0) return DF_OK;
  if (lnA == nullptr) {
    // restore the file's values: copy the host records back
    for (int j = 0; j < M; ++j) m->blob_host[m->dims.off_rx + RX_REC * j] = m->lnA_file[j];
    return cuda_check(cudaMemcpyAsync(m->blob_dev, m->blob_host.data(), sizeof(double) * m->dims.total,
                                      cudaMemcpyHostToDevice, st),
                      "restore lnA");
  }
  k_set_lnA<<<(M + 127) / 128, 128, 0, st>>>(m->blob_dev, m->dims.off_rx, M, lnA);
  return cuda_check(cudaGetLastError(), "set lnA kernel");
}

}  // namespace df
