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

#include "common.cuh"
#include "chem_warp.cuh"
#include "integrate_thread.cuh"

namespace df {


static bool g_tab_ready[64] = {false};

static int ensure_tables(int dev) {
  if (dev < 0 || dev >= 64) return DF_OK;
  if (g_tab_ready[dev]) return DF_OK;
  RosTab t[2] = {make_rodas4(), make_rodas3()};
  // the thread path forms y_new and the error estimate from the last stage
  if (!t[0].stiff_acc || !t[1].stiff_acc) return set_error(DF_EUNSUPPORTED, "Rosenbrock table not stiffly accurate");
  int rc = cuda_check(cudaMemcpyToSymbol(c_tab, t, sizeof(t)), "upload Rosenbrock tables");
  if (rc == DF_OK) g_tab_ready[dev] = true;
  return rc;
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
  double2* etab = reinterpret_cast<double2*>(smem);
  for (int i = tid; i < 64; i += stride) etab[i] = g_exp2_tab[i];
  int boff = 128;
  if (a.stage_blob) {
    for (int i = tid; i < a.d.total; i += stride) smem[boff + i] = a.blob[i];
    blob = smem + boff;
    boff += blob_smem_doubles(a.d);
  }
  __syncthreads();
  const MechView mv = make_view(blob, a.d, etab);
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
// one cell per warp (any N <= 64)
// ----------------------------------------------------------------------------
template <bool CONSTV>
__global__ void __launch_bounds__(256, 1) k_integrate_warp(IntegArgs a, const int* csr, WarpWS L) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double2* etab = reinterpret_cast<double2*>(smem);
  for (int i = tid; i < 64; i += blockDim.x) etab[i] = g_exp2_tab[i];
  int boff = 128;
  const double* blob = a.blob;
  if (a.stage_blob) {
    for (int i = tid; i < a.d.total; i += blockDim.x) smem[boff + i] = a.blob[i];
    blob = smem + boff;
    boff += blob_smem_doubles(a.d);
  }
  __syncthreads();
  const MechView mv = make_view(blob, a.d, etab);
  const int N = a.d.N, n = N + 1;
  double* ws = smem + boff + (size_t)warp * L.total;
  double* y = ws + L.y;
  double* ys = ws + L.ys;
  double* f = ws + L.f;
  double* J = ws + L.J;
  double* K = ws + L.K;
  int* piv = reinterpret_cast<int*>(ws + L.piv);
  const RosTab& tb = c_tab[a.method];
  unsigned long long tot_acc = 0, tot_rej = 0;
  const unsigned long long nwork = a.nwork_dev ? *a.nwork_dev : (unsigned long long)a.nwork;

  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(&a.counters[0], 1ull);
    idx = __shfl_sync(WFULL, idx, 0);
    if (idx >= nwork) break;
    const int64_t cell = a.order ? (int64_t)a.order[idx] : (int64_t)idx;
    bool okin = true;
    for (int i = lane; i < n; i += 32) {
      const double v = i == 0 ? a.T[cell] : a.Y[(int64_t)(i - 1) * a.ncells + cell];
      y[i] = v;
      okin = okin && isfinite(v) && (i > 0 || v > 0.0);
    }
    double pc = 10.0 * a.p[cell];  // Pa -> dyn/cm^2
    okin = __all_sync(WFULL, okin) && isfinite(pc) && pc > 0.0;
    __syncwarp();
    if (CONSTV) {  // density of the initial state, fixed from here on
      double s = 0.0;
      for (int k = lane; k < N; k += 32) s += y[1 + k] * mv.sp[SP_REC * k + 1];
      pc = pc / (RU * y[0] * warp_sum(s));
      okin = okin && isfinite(pc) && pc > 0.0;
    }
    int status = okin ? DF_CELL_OK : DF_CELL_NONFINITE;
    bool done = !okin || !(a.dt > 0.0);
    double t = 0.0, h = fmin(a.h0, a.dt);
    double hacc = 0.0, erracc = 1.0;
    int nacc = 0, nrej = 0, istep = 0;
    PeakTrack pk;
    pk.reset();
    bool last_rej = false;
    while (!done) {
      bool last = false;
      if (t + h >= a.dt) {
        h = a.dt - t;
        last = true;
      }
      warp_eval<true, CONSTV>(mv, csr, N, pc, ws, L, L.y);
      const double fT = f[0], t0 = t;
      if (nacc == 0 && nrej == 0) {
        // first trial step from the fastest relative rate (see first_step_limit)
        double r = 0.0;
        for (int i = lane; i < n; i += 32)
          r = fmax(r, fabs(f[i]) / (i == 0 ? fabs(y[0]) : fmax(fabs(y[i]), 1e-6)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(WFULL, r, o));
        if (r > 0.0 && FIRST_STEP_THETA / r < h) {
          h = FIRST_STEP_THETA / r;
          last = false;
        }
      }
      const double ih = rcp_nr(h);
      const double hgi = rcp_nr(h * tb.gamma);
      for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e - i * n;
        J[e] = i == j ? hgi - J[e] : -J[e];
      }
      __syncwarp();
      bool ok = warp_lu(J, piv, n);
      for (int s = 0; s < tb.s; ++s) {
        if (s > 0 && tb.newf[s]) {
          for (int i = lane; i < n; i += 32) {
            double acc = y[i];
            for (int j = 0; j < s; ++j) acc += tb.a[s][j] * K[j * n + i];
            ys[i] = acc;
          }
          __syncwarp();
          warp_eval<false, CONSTV>(mv, csr, N, pc, ws, L, L.ys);
        }
        for (int i = lane; i < n; i += 32) {
          double acc = f[i];
          for (int j = 0; j < s; ++j) acc += (tb.c[s][j] * ih) * K[j * n + i];
          K[s * n + i] = acc;
        }
        __syncwarp();
        warp_solve(J, piv, K + s * n, n);
      }
      double e2 = 0.0;
      for (int i = lane; i < n; i += 32) {
        double yn = y[i], e = 0.0;
        for (int s = 0; s < tb.s; ++s) {
          yn += tb.m[s] * K[s * n + i];
          e += tb.e[s] * K[s * n + i];
        }
        ys[i] = yn;
        const double r = e * rcp_nr((i == 0 ? a.atolT : a.atolY) + a.rtol * fmax(fabs(y[i]), fabs(yn)));
        e2 += r * r;
      }
      // WRMS error norm: the accept test in FP64 (sum <= n), the step-size
      // factors of the controller (see step_control) in FP32 on the wide pipe
      const double esum = warp_sum(e2);
      ok = ok && isfinite(esum);
      const float en = sqrtf((float)esum * (1.0f / (float)n));
      __syncwarp();
      if (ok && esum <= (double)n) {
        for (int i = lane; i < n; i += 32) y[i] = ys[i];
        t = last ? a.dt : t + h;
        ++nacc;
        // elementary + Gustafsson predictive controller (see step_control)
        const float e = fmaxf(en, 1e-10f), ie = -1.0f / (float)tb.elo;
        float fac = 0.9f * powf(e, ie);
        if (nacc > 1) fac = fminf(fac, 0.9f * ((float)h / (float)hacc) * powf(e * e / (float)erracc, ie));
        fac = fminf(last_rej ? 1.0f : 6.0f, fmaxf(0.2f, fac));
        hacc = h;
        erracc = fmax(1e-2, (double)en);
        h *= (double)fac;
        last_rej = false;
        pk.add(istep * a.dt + t0, fT);  // dT/dt at the start of an accepted substep
        if (t >= a.dt) {
          if (++istep < a.nsteps) t = 0.0;  // next consecutive step of dt
          else done = true;
        }
      } else {
        ++nrej;
        const float fmn = nacc == 0 ? 1e-4f : 0.2f;
        const float fac = ok ? fmaxf(fmn, 0.9f * powf(en, -1.0f / (float)tb.elo)) : 0.25f;
        h *= (double)fac;
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
      __syncwarp();
    }
    if (status == DF_CELL_OK) {
      for (int i = lane; i < n; i += 32) {
        if (i == 0) a.T[cell] = y[0];
        else a.Y[(int64_t)(i - 1) * a.ncells + cell] = y[i];
      }
    }
    if (lane == 0) {
      if (a.t_ign) a.t_ign[cell] = status == DF_CELL_OK ? pk.time() : NAN;
      a.status[cell] = status;
      if (a.nsub) a.nsub[cell] = nacc;
      tot_acc += nacc;
      tot_rej += nrej;
    }
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&a.counters[1], tot_acc);
    atomicAdd(&a.counters[2], tot_rej);
  }
}

template <bool WITH_J>
__global__ void __launch_bounds__(256) k_eval_warp(EvalArgs a, const int* csr, WarpWS L) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double2* etab = reinterpret_cast<double2*>(smem);
  for (int i = tid; i < 64; i += blockDim.x) etab[i] = g_exp2_tab[i];
  __syncthreads();
  const MechView mv = make_view(a.blob, a.d, etab);
  const int N = a.d.N, n = N + 1;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= a.ncells) return;
  double* ws = smem + 128 + (size_t)warp * L.total;
  for (int i = lane; i < n; i += 32) ws[L.y + i] = i == 0 ? a.T[c] : a.Y[(int64_t)(i - 1) * a.ncells + c];
  __syncwarp();
  const double q = warp_eval<WITH_J>(mv, csr, N, 10.0 * a.p[c], ws, L, L.y);
  if (a.dydt)
    for (int i = lane; i < n; i += 32) a.dydt[(int64_t)i * a.ncells + c] = ws[L.f + i];
  if (a.qdot && lane == 0) a.qdot[c] = 0.1 * q;
  if (WITH_J)
    for (int e = lane; e < n * n; e += 32) a.J[c * n * n + e] = ws[L.J + e];
}

// ----------------------------------------------------------------------------
// work order by temperature (hottest first): a counting sort over 1 K bins.
// Hot cells take the most substeps, so handing them out first shortens the
// tail of the persistent launch, and lanes that refill together get cells of
// similar stiffness (similar substep counts).
// ----------------------------------------------------------------------------
constexpr int ORDER_BINS = 4096;
constexpr double ORDER_T_TOP = 4000.0;

__device__ __forceinline__ int t_bin(double T) {
  const double b = ORDER_T_TOP - T;
  if (!(b >= 0.0)) return 0;  // T >= top
  return b >= ORDER_BINS - 1 ? ORDER_BINS - 1 : (int)b;
}

__global__ void k_order_hist(const double* T, int64_t n, unsigned* hist) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) atomicAdd(&hist[t_bin(T[c])], 1u);
}

__global__ void k_order_scan(unsigned* hist) {
  // one block of 1024 threads, 4 bins each: exclusive prefix sum in place
  __shared__ unsigned part[1024];
  const int t = threadIdx.x;
  unsigned v[4], s = 0;
  for (int i = 0; i < 4; ++i) {
    v[i] = hist[4 * t + i];
    s += v[i];
  }
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned add = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  unsigned base = part[t] - s;
  for (int i = 0; i < 4; ++i) {
    hist[4 * t + i] = base;
    base += v[i];
  }
}

__global__ void k_order_scatter(const double* T, int64_t n, unsigned* offs, int32_t* order) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) order[atomicAdd(&offs[t_bin(T[c])], 1u)] = (int32_t)c;
}

// the same order for a list of cells whose length is on the device (at most
// cap entries): list entries are cell indices, the order holds cell indices
__global__ void k_order_hist_list(const double* T, const int32_t* list, const unsigned long long* count, int64_t cap,
                                  unsigned* hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long n = *count;
  if (i < cap && (unsigned long long)i < n) atomicAdd(&hist[t_bin(T[list[i]])], 1u);
}

__global__ void k_order_scatter_list(const double* T, const int32_t* list, const unsigned long long* count,
                                     int64_t cap, unsigned* offs, int32_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long n = *count;
  if (i < cap && (unsigned long long)i < n) {
    const int32_t c = list[i];
    order[atomicAdd(&offs[t_bin(T[c])], 1u)] = c;
  }
}

static int ensure_order_buffers(df_mech* m, int64_t n) {
  if (m->order_cap < n) {
    if (m->order) cudaFree(m->order);
    m->order = nullptr;
    m->order_cap = 0;
    int rc = cuda_check(cudaMalloc(&m->order, sizeof(int32_t) * n), "cudaMalloc order");
    if (rc) return rc;
    m->order_cap = n;
  }
  if (!m->bins) return cuda_check(cudaMalloc(&m->bins, sizeof(unsigned) * ORDER_BINS), "cudaMalloc bins");
  return DF_OK;
}

static int build_order_list(df_mech* m, const double* T, const int32_t* list, const unsigned long long* count,
                            int64_t cap, cudaStream_t st, int32_t** out) {
  int rc = ensure_order_buffers(m, cap);
  if (!rc) rc = cuda_check(cudaMemsetAsync(m->bins, 0, sizeof(unsigned) * ORDER_BINS, st), "clear bins");
  if (rc) return rc;
  const unsigned blocks = (unsigned)((cap + 255) / 256);
  k_order_hist_list<<<blocks, 256, 0, st>>>(T, list, count, cap, m->bins);
  k_order_scan<<<1, 1024, 0, st>>>(m->bins);
  k_order_scatter_list<<<blocks, 256, 0, st>>>(T, list, count, cap, m->bins, m->order);
  *out = m->order;
  return cuda_check(cudaGetLastError(), "list order kernels");
}

static int build_order(df_mech* m, const double* T, int64_t ncells, cudaStream_t st, int32_t** out) {
  int rc = ensure_order_buffers(m, ncells);
  if (!rc) rc = cuda_check(cudaMemsetAsync(m->bins, 0, sizeof(unsigned) * ORDER_BINS, st), "clear bins");
  if (rc) return rc;
  const unsigned blocks = (unsigned)((ncells + 255) / 256);
  k_order_hist<<<blocks, 256, 0, st>>>(T, ncells, m->bins);
  k_order_scan<<<1, 1024, 0, st>>>(m->bins);
  k_order_scatter<<<blocks, 256, 0, st>>>(T, ncells, m->bins, m->order);
  *out = m->order;
  return cuda_check(cudaGetLastError(), "order kernels");
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
namespace {

template <int NS>
size_t thread_smem_bytes(const MechDims& d, int threads, bool stage) {
  return sizeof(double) * (2 * EXP_TAB_SIZE + (stage ? blob_smem_doubles(d) : 0) + (size_t)thread_ws_doubles<NS>() * threads);
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
int integrate_dispatch(df_mech* m, const IntegArgs& a0, cudaStream_t st, int threads, int bps, bool constv,
                       bool jit) {
  m->jit_used = 0;
  if (jit && !constv) {  // the kernel generated for this mechanism, if it can run
    bool launched = false;
    const int rc = jit_thread_launch(m, threads, bps, a0, st, &launched);
    if (rc || launched) return rc;
  }
  IntegArgs a = a0;
  a.stage_blob = 1;
  size_t sm = thread_smem_bytes<NS>(m->dims, threads, true);
  if (sm > m->max_smem_optin) {
    a.stage_blob = 0;
    sm = thread_smem_bytes<NS>(m->dims, threads, false);
  }
  if (sm > m->max_smem_optin)
    return set_error(DF_EUNSUPPORTED, "integrator shared memory exceeds the per-block limit");
  // block sizes with a compile-time stride (constant pressure); others take
  // the run-time stride; with t_ign the kernels that refine the ignition time
  auto kf = a.t_ign ? (constv ? k_integrate_thread<NS, true, 0, BlobEval, true>
                              : k_integrate_thread<NS, false, 0, BlobEval, true>)
            : constv          ? k_integrate_thread<NS, true>
            : threads == 32  ? k_integrate_thread<NS, false, 32>
            : threads == 64  ? k_integrate_thread<NS, false, 64>
            : threads == 128 ? k_integrate_thread<NS, false, 128>
                             : k_integrate_thread<NS, false>;
  int rc = cuda_check(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                      "set integrator shared memory");
  if (rc) return rc;
  int occ = 0;
  rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf, threads, sm), "occupancy");
  if (rc) return rc;
  if (occ < 1) return set_error(DF_EUNSUPPORTED, "integrator launch shape does not fit on an SM");
  const int per_sm = bps > 0 ? std::min(bps, occ) : occ;
  int64_t blocks = (int64_t)m->num_sms * per_sm;
  const int64_t need = (a.nwork + threads - 1) / threads;
  if (blocks > need) blocks = std::max<int64_t>(1, need);
  rc = cuda_check(cudaMemsetAsync(m->counters, 0, 4 * sizeof(unsigned long long), st), "reset work counter");
  if (rc) return rc;
  kf<<<(unsigned)blocks, threads, sm, st>>>(a);
  return cuda_check(cudaGetLastError(), "integrator kernel launch");
}

}  // namespace

#define DF_THREAD_NS_LIST(X) X(3) X(9)

static bool has_thread_kernel(int N) {
  switch (N) {
#define X(NS) case NS:
    DF_THREAD_NS_LIST(X)
#undef X
    return true;
    default:
      return false;
  }
}

namespace {

// warp path launch shape: warps per block from the shared-memory budget
int warp_shape(const df_mech* m, const WarpWS& L, bool want_stage, int max_warps, int* warps, int* stage,
               size_t* smem) {
  const size_t per_warp = sizeof(double) * (size_t)L.total;
  const size_t fixed = sizeof(double) * 128;
  const size_t blob = sizeof(double) * (size_t)blob_smem_doubles(m->dims);
  // the mechanism staged in shared memory where that costs no warp; where
  // leaving it in global memory (read through L1) fits one more warp per
  // block, more warps win (they keep the narrow FP64 pipe busier)
  int best_w = 0, best_st = 0;
  for (int st = want_stage ? 1 : 0; st >= 0; --st) {
    const size_t base = fixed + (st ? blob : 0);
    if (base + per_warp > m->max_smem_optin) continue;
    const int w = std::min((int)((m->max_smem_optin - base) / per_warp), max_warps);
    if (w > best_w) {
      best_w = w;
      best_st = st;
    }
  }
  if (best_w > 0) {
    *warps = best_w;
    *stage = best_st;
    *smem = fixed + (best_st ? blob : 0) + per_warp * best_w;
    return DF_OK;
  }
  return set_error(DF_EUNSUPPORTED, "warp-path workspace exceeds shared memory");
}

int eval_warp_dispatch(const df_mech* m, int64_t ncells, const double* T, const double* p, const double* Y,
                       double* dydt, double* qdot, double* J, cudaStream_t st) {
  const WarpWS L = warp_ws_layout(m->dims.N, m->dims.M, m->dims.n_eff);
  int warps, stage;
  size_t sm;
  int rc = warp_shape(m, L, false, 4, &warps, &stage, &sm);
  if (rc) return rc;
  EvalArgs a{m->blob_dev, m->dims, ncells, T, p, Y, dydt, qdot, J, 0};
  const int64_t blocks = (ncells + warps - 1) / warps;
  if (J) {
    auto kf = k_eval_warp<true>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<(unsigned)blocks, 32 * warps, sm, st>>>(a, m->csr_dev, L);
  } else {
    auto kf = k_eval_warp<false>;
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kf<<<(unsigned)blocks, 32 * warps, sm, st>>>(a, m->csr_dev, L);
  }
  return cuda_check(cudaGetLastError(), "warp evaluation kernel");
}

int integrate_warp_dispatch(df_mech* m, const IntegArgs& a0, cudaStream_t st, int threads, bool constv) {
  const WarpWS L = warp_ws_layout(m->dims.N, m->dims.M, m->dims.n_eff);
  int warps, stage;
  size_t sm;
  const int max_warps = threads > 0 ? threads / 32 : 8;
  int rc = warp_shape(m, L, true, max_warps, &warps, &stage, &sm);
  if (rc) return rc;
  IntegArgs a = a0;
  a.stage_blob = stage;
  auto kf = constv ? k_integrate_warp<true> : k_integrate_warp<false>;
  rc = cuda_check(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                  "set warp integrator shared memory");
  if (rc) return rc;
  int occ = 0;
  rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf, 32 * warps, sm), "occupancy");
  if (rc) return rc;
  if (occ < 1) return set_error(DF_EUNSUPPORTED, "warp integrator does not fit on an SM");
  int64_t blocks = (int64_t)m->num_sms * occ;
  const int64_t need = (a.nwork + warps - 1) / warps;
  if (blocks > need) blocks = std::max<int64_t>(1, need);
  rc = cuda_check(cudaMemsetAsync(m->counters, 0, 4 * sizeof(unsigned long long), st), "reset work counter");
  if (rc) return rc;
  kf<<<(unsigned)blocks, 32 * warps, sm, st>>>(a, m->csr_dev, L);
  return cuda_check(cudaGetLastError(), "warp integrator kernel launch");
}

}  // namespace

int launch_rhs(const df_mech* m, int64_t ncells, const double* T, const double* p,
               const double* Y, double* dydt, double* qdot, cudaStream_t st) {
  switch (m->dims.N) {
#define X(NS) \
  case NS:    \
    return eval_dispatch<NS>(m, ncells, T, p, Y, dydt, qdot, nullptr, st);
    DF_THREAD_NS_LIST(X)
#undef X
    default:
      return eval_warp_dispatch(m, ncells, T, p, Y, dydt, qdot, nullptr, st);
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
      return eval_warp_dispatch(m, ncells, T, p, Y, nullptr, nullptr, J, st);
  }
}

int launch_integrate(df_mech* m, int64_t ncells, double* T, const double* p, double* Y,
                     double dt, const df_integ_opts& o, int32_t* status, int32_t* nsub,
                     cudaStream_t st) {
  return launch_integrate_list(m, ncells, T, p, Y, dt, o, status, nsub, nullptr, ncells, st, nullptr);
}

int launch_integrate_steps(df_mech* m, int64_t ncells, double* T, const double* p, double* Y, double dt,
                           int nsteps, const df_integ_opts& o, int32_t* status, int32_t* nsub, double* t_ign,
                           cudaStream_t st) {
  return launch_integrate_list(m, ncells, T, p, Y, dt, o, status, nsub, nullptr, ncells, st, nullptr, nsteps,
                               t_ign);
}

int launch_integrate_list(df_mech* m, int64_t ncells, double* T, const double* p, double* Y, double dt,
                          const df_integ_opts& o, int32_t* status, int32_t* nsub, const int32_t* order,
                          int64_t nwork, cudaStream_t st, const unsigned long long* nwork_dev, int nsteps,
                          double* t_ign) {
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
  a.nsteps = nsteps;
  a.t_ign = t_ign;
  if (!order && o.order_by_T && nwork == ncells && ncells > 1) {
    int32_t* ord = nullptr;
    rc = build_order(m, T, ncells, st, &ord);
    if (rc) return rc;
    order = ord;
  } else if (order && nwork_dev && o.order_by_T && nwork > 1) {
    // a cell list counted on the device (the surrogate's fallback cells):
    // hottest first as well, so its stiffest cells do not start last
    int32_t* ord = nullptr;
    rc = build_order_list(m, T, order, nwork_dev, nwork, st, &ord);
    if (rc) return rc;
    order = ord;
  }
  a.order = order;
  a.nwork = nwork;
  a.nwork_dev = nwork_dev;
  a.counters = m->counters;
  // thread-per-cell kernels: built for the species counts of
  // DF_THREAD_NS_LIST; for any other N <= 16 only the kernel generated for the
  // mechanism (constant pressure, jit on)
  const bool thread_ok = has_thread_kernel(m->dims.N);
  const bool gen_only = !thread_ok && o.jit == 0 && o.reactor == 0 && m->dims.N <= THREAD_PATH_MAX_N;
  if (o.path == 1 && !thread_ok && !gen_only)
    return set_error(DF_EUNSUPPORTED, "no thread-per-cell kernel for this species count and options");
  // zero shape fields: the path and shape df_chem_autotune chose, if any
  int bt = o.block_threads, bps = o.blocks_per_sm, path = o.path;
  const bool tuned = bt == 0 && bps == 0 && m->tuned_threads > 0;
  if (tuned && path == 0) path = m->tuned_path;
  const bool warp_path = path == 2 || (!thread_ok && !gen_only);
  if (tuned && m->tuned_path == (warp_path ? 2 : 1)) {
    bt = m->tuned_threads;
    bps = m->tuned_bps;
  }
  if (warp_path) {
    m->jit_used = 0;
    return integrate_warp_dispatch(m, a, st, bt, o.reactor == 1);
  }
  if (!thread_ok) {  // the generated kernel only (32- or 64-thread blocks)
    bool launched = false;
    m->jit_used = 0;
    const int rc = jit_thread_launch(m, bt == 64 ? 64 : 32, bps, a, st, &launched);
    if (rc || launched) return rc;
    if (o.path == 1)
      return set_error(DF_EUNSUPPORTED, "thread-per-cell path: the generated kernel is unavailable (" +
                                            m->jit_note + ")");
    return integrate_warp_dispatch(m, a, st, 0, false);
  }
  // default block: 32 threads (5 warps per SM for the generated kernel; the
  // mechanism-independent kernel runs as fast at 32 as at 64)
  const int threads = bt > 0 ? bt : 32;
  switch (m->dims.N) {
#define X(NS) \
  case NS:    \
    return integrate_dispatch<NS>(m, a, st, threads, bps, o.reactor == 1, o.jit == 0);
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

namespace df {

// Time candidate launch shapes of the integrator on a copy of the first
// `sample` cells and keep the fastest (the GPU form of the paper's load
// balancing, Sec. 3.2: the shape that keeps the lanes busiest on this cell mix).
int autotune_integrate(df_mech* m, int64_t ncells, const double* T, const double* p, const double* Y, double dt,
                       const df_integ_opts& base, int64_t sample, df_integ_opts* best, float* best_ms,
                       cudaStream_t st) {
  const int N = m->dims.N;
  const int64_t n = std::min<int64_t>(ncells, sample > 0 ? sample : 65536);
  // species counts without a compiled thread kernel: the generated thread
  // kernel (if it can run) competes with the warp path
  const bool gen_only = !has_thread_kernel(N) && base.jit == 0 && base.reactor == 0 && N <= THREAD_PATH_MAX_N &&
                        base.path != 2;
  const bool warp_path = base.path == 2 || !has_thread_kernel(N);
  double *T0 = nullptr, *p0 = nullptr, *Y0 = nullptr, *Tw = nullptr, *Yw = nullptr;
  int32_t* stt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_check(cudaMalloc(&T0, sizeof(double) * n * (3 + 2 * (int64_t)N)), "autotune scratch");
  if (!rc) {
    p0 = T0 + n;
    Tw = p0 + n;
    Y0 = Tw + n;
    Yw = Y0 + n * N;
    rc = cuda_check(cudaMalloc(&stt, sizeof(int32_t) * n), "autotune scratch");
  }
  if (!rc) rc = cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = cuda_check(cudaEventCreate(&e1), "event");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(T0, T, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy T");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(p0, p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "copy p");
  if (!rc)
    rc = cuda_check(cudaMemcpy2DAsync(Y0, sizeof(double) * n, Y, sizeof(double) * ncells, sizeof(double) * n, N,
                                      cudaMemcpyDeviceToDevice, st),
                    "copy Y");
  std::vector<df_integ_opts> cand;
  for (int order = 0; order <= 1; ++order) {
    if (gen_only) {
      for (int bt : {32, 64})
        for (int bps : {0, 1, 2}) {
          df_integ_opts o = base;
          o.block_threads = bt;
          o.blocks_per_sm = bps;
          o.order_by_T = order;
          o.path = 1;
          cand.push_back(o);
        }
    }
    if (warp_path) {
      for (int bt : {64, 128, 256}) {
        df_integ_opts o = base;
        o.block_threads = bt;
        o.blocks_per_sm = 0;
        o.order_by_T = order;
        o.path = 2;
        cand.push_back(o);
      }
    } else {
      for (int bt : {32, 64, 96, 128})
        for (int bps : {0, 1, 2}) {
          df_integ_opts o = base;
          o.block_threads = bt;
          o.blocks_per_sm = bps;
          o.order_by_T = order;
          o.path = 1;
          cand.push_back(o);
        }
    }
  }
  float tbest = INFINITY;
  df_integ_opts obest = base;
  for (size_t c = 0; c < cand.size() && !rc; ++c) {
    float tmin = INFINITY;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok && !rc; ++rep) {
      rc = cuda_check(cudaMemcpyAsync(Tw, T0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "reset T");
      if (!rc)
        rc = cuda_check(cudaMemcpyAsync(Yw, Y0, sizeof(double) * n * N, cudaMemcpyDeviceToDevice, st), "reset Y");
      if (!rc) rc = cuda_check(cudaEventRecord(e0, st), "event");
      if (rc) break;
      if (launch_integrate(m, n, Tw, p0, Yw, dt, cand[c], stt, nullptr, st) != DF_OK) {
        ok = false;  // a shape that does not fit this device: skip it
        break;
      }
      rc = cuda_check(cudaEventRecord(e1, st), "event");
      if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "synchronise");
      float ms = 0.0f;
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "elapsed time");
      if (!rc) tmin = std::min(tmin, ms);
    }
    if (!rc && ok && tmin < tbest) {
      tbest = tmin;
      obest = cand[c];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (T0) cudaFree(T0);
  if (stt) cudaFree(stt);
  if (rc) return rc;
  if (!(tbest < INFINITY)) return set_error(DF_EUNSUPPORTED, "df_chem_autotune: no launch shape fits this device");
  m->tuned_threads = obest.block_threads;
  m->tuned_bps = obest.blocks_per_sm;
  m->tuned_path = obest.path;
  m->tuned_for_ncells = n;
  if (best) *best = obest;
  if (best_ms) *best_ms = tbest;
  set_error(DF_OK, "");
  return DF_OK;
}

}  // namespace df
