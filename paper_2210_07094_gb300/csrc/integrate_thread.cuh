// The persistent thread-per-cell integrator kernel (one cell per thread,
// N <= 16) and its arguments, shared by the library's own build and by the
// kernels it generates for a loaded mechanism and compiles at run time.
//
// Scheduling: a persistent grid sized to the SMs; each lane takes a new cell
// from a device work counter as soon as its cell is finished (warp-aggregated
// atomics), so cells of very uneven stiffness keep all lanes busy (the GPU
// analogue of the chemistry load balancing of Sec. 3.2).
#pragma once
#include "rosenbrock.cuh"

namespace df {

// Rosenbrock coefficient tables (RODAS4, RODAS3), uploaded by the host into
// each module that holds the kernel (external linkage in a runtime-compiled
// module, so that the host can look it up by name)
#ifdef __CUDACC_RTC__
__constant__ RosTab c_tab[2];
#else
static __constant__ RosTab c_tab[2];
#endif

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
  const int32_t* order;            // optional list of the cell indices to advance
  int64_t nwork;                   // number of cells to advance (entries of order)
  const unsigned long long* nwork_dev;  // if set, the number of cells is read from here
  unsigned long long* counters;    // [0] next cell, [1] accepted, [2] rejected
  int stage_blob;                  // 1: copy the blob into shared memory
  int nsteps;                      // consecutive steps of dt per cell (>= 1)
  double* t_ign;                   // optional: time of the largest dT/dt per cell
};

constexpr unsigned FULL = 0xffffffffu;

// per-thread shared-memory doubles of the thread path: the species vectors C,
// wdot, g/RT, h/RT, cp/R (when the evaluation policy keeps them there), the
// matrix J / W and the six stage vectors
template <int NS, class EVAL = BlobEval>
__host__ __device__ constexpr int thread_ws_doubles() {
  return (EVAL::kSpeciesVectors ? 5 * NS : 0) + (NS + 1) * (NS + 1) + 6 * (NS + 1);
}

__host__ __device__ inline int blob_smem_doubles(const MechDims& d) { return (d.total + 1) & ~1; }

// BT > 0: the kernel is launched with exactly BT threads per block, the
// stride of the per-thread shared-memory vectors is a compile-time constant.
// EVAL: the evaluation policy of f and J (see BlobEval).  IGN: track the
// largest dT/dt with the neighbouring samples that refine its time (a.t_ign);
// without it only the time of the largest sample is kept (fewer registers).
template <int NS, bool CONSTV = false, int BT = 0, class EVAL = BlobEval, bool IGN = false>
__global__ void __launch_bounds__(128, 1) k_integrate_thread(IntegArgs a) {
  constexpr int n = NS + 1;
  extern __shared__ double smem[];
  const int tid = threadIdx.x;
  const int stride = BT > 0 ? BT : blockDim.x;
  const double* blob = a.blob;
  double2* etab = reinterpret_cast<double2*>(smem);
  for (int i = tid; i < EXP_TAB_SIZE; i += stride) etab[i] = exp_table_src()[i];
  int boff = 2 * EXP_TAB_SIZE;
  if (a.stage_blob) {
    for (int i = tid; i < a.d.total; i += stride) smem[boff + i] = a.blob[i];
    blob = smem + boff;
    boff += blob_smem_doubles(a.d);
  }
  __syncthreads();
  const MechView mv = make_view(blob, a.d, etab);
  double* ws = smem + boff + tid;
  typedef SVT<double, BT> V;
  constexpr int nv = EVAL::kSpeciesVectors ? NS : 0;
  // without species vectors in shared memory (the generated evaluation) the
  // first view is the evaluation's scratch while J is built: the stage vectors'
  // storage, idle then
  V C{ws + (nv > 0 ? 0 : (n * n) * stride), stride};
  V wdot{ws + nv * stride, stride};
  V gRT{ws + 2 * nv * stride, stride};
  V hRT{ws + 3 * nv * stride, stride};
  V cpR{ws + 4 * nv * stride, stride};
  V Jv{ws + 5 * nv * stride, stride};
  V Kv{ws + (5 * nv + n * n) * stride, stride};
  const RosTab& tb = c_tab[a.method];
  const int lane = tid & 31;
  const unsigned long long nwork = a.nwork_dev ? *a.nwork_dev : (unsigned long long)a.nwork;

  int64_t cell = -1;
  bool exhausted = false, done = false, last_rej = false;
  int status = 0, nacc = 0, nrej = 0, istep = 0;
  double y[n];
  double t = 0.0, h = 0.0, fbest = -INFINITY, tbest = 0.0;
  PeakTrack pk;
  if (IGN) pk.reset();
  double prm = 0.0;  // pressure [dyn/cm^2], or the fixed density [g/cm^3] at constant volume
  StepState ss{0.0, 1.0};
  unsigned long long tot_acc = 0, tot_rej = 0;

  for (;;) {
    // finished cell: store
    if (cell >= 0 && done) {
      if (status == DF_CELL_OK) {
        a.T[cell] = y[0];
#pragma unroll
        for (int k = 0; k < NS; ++k) a.Y[(int64_t)k * a.ncells + cell] = y[1 + k];
      }
      if (a.t_ign) a.t_ign[cell] = status == DF_CELL_OK ? (IGN ? pk.time() : tbest) : NAN;
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
        if (idx < nwork) {
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
          prm = 10.0 * pc;  // Pa -> dyn/cm^2
          if (CONSTV) {  // density of the initial state, fixed from here on
            double sYW = 0.0;
#pragma unroll
            for (int k = 0; k < NS; ++k) sYW += y[1 + k] * mv.sp[SP_REC * k + 1];
            prm = prm / (RU * y[0] * sYW);
            ok = ok && isfinite(prm) && prm > 0.0;
          }
          t = 0.0;
          h = fmin(a.h0, a.dt);
          nacc = nrej = istep = 0;
          fbest = -INFINITY;
          tbest = 0.0;
          if (IGN) pk.reset();
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
    const double pc = prm;
    bool last = false;
    if (t + h >= a.dt) {
      h = a.dt - t;
      last = true;
    }
    double ys[n];
    double en;
    double fT;
    const double t0 = t;
    const bool ok = ros_attempt<NS, CONSTV, BT, EVAL>(mv, tb, pc, y, h, a.rtol, a.atolY, a.atolT, C, wdot, gRT, hRT,
                                                cpR, Jv, Kv, stride, ys, en, nullptr, nacc == 0 && nrej == 0, &last,
                                                &fT);
    const int nacc0 = nacc;
    step_control(tb, ok, en, last, a.dt, y, ys, t, h, nacc, nrej, last_rej, done, ss);
    if (nacc > nacc0) {  // dT/dt at the start of an accepted substep
      if (IGN) {
        pk.add(istep * a.dt + t0, fT);
      } else if (fT > fbest) {
        fbest = fT;
        tbest = istep * a.dt + t0;
      }
    }
    if (done && ++istep < a.nsteps) {  // next consecutive step of dt
      done = false;
      t = 0.0;
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

}  // namespace df
