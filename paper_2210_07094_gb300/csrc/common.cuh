// Internal definitions shared by the library's translation units (host side;
// the device-side definitions and the mechanism blob layout are in
// dev_common.cuh).
#pragma once
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/df_chem.h"

#include "dev_common.cuh"


// the opaque handle
struct df_mech {
  df::MechDims dims;
  std::vector<double> blob_host;  // as parsed (lnA from the file)
  std::vector<double> lnA_file;
  std::vector<int> csr_host;      // species -> (reaction, net nu) lists: [N+1] ptr, pairs
  double* blob_dev = nullptr;     // device copy (lnA may be overridden)
  int* csr_dev = nullptr;
  int device = 0;
  // persistent-queue and statistics scratch (device): [0] work counter,
  // [1] accepted, [2] rejected, [3] error flag
  unsigned long long* counters = nullptr;
  // work order scratch (cells sorted hottest first) and its histogram
  int32_t* order = nullptr;
  int64_t order_cap = 0;
  unsigned* bins = nullptr;
  // autotune cache: the launch shape df_chem_autotune chose, and for which path
  // (1 thread per cell, 2 warp per cell) and sample size
  int tuned_threads = 0, tuned_bps = 0, tuned_path = 0;
  int64_t tuned_for_ncells = -1;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  size_t smem_per_sm = 0, smem_reserved_per_block = 0;
  // generated thread-path kernel (codegen.cu): 1 when the last thread-path
  // launch used it, and its state (compile time, or why it is unavailable)
  int jit_used = 0;
  std::string jit_note;
  // the module compiled for this mechanism on each device (owned by the
  // process-wide cache in codegen.cu; null until the first launch)
  void* jit_module[64] = {nullptr};
};

namespace df {
// thread-local last-error text (api.cu)
int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);

// parse a mechanism JSON file into host arrays (mech.cu)
int parse_mechanism(const char* path, df_mech* m);

// launchers (integrate.cu)
int launch_rhs(const df_mech* m, int64_t ncells, const double* T, const double* p,
               const double* Y, double* dydt, double* qdot, cudaStream_t st);
int launch_jacobian(const df_mech* m, int64_t ncells, const double* T, const double* p,
                    const double* Y, double* J, cudaStream_t st);
int launch_integrate(df_mech* m, int64_t ncells, double* T, const double* p, double* Y,
                     double dt, const df_integ_opts& o, int32_t* status, int32_t* nsub,
                     cudaStream_t st);
int launch_set_lnA(df_mech* m, const double* lnA, cudaStream_t st);
int launch_integrate_steps(df_mech* m, int64_t ncells, double* T, const double* p, double* Y, double dt,
                           int nsteps, const df_integ_opts& o, int32_t* status, int32_t* nsub, double* t_ign,
                           cudaStream_t st);
int autotune_integrate(df_mech* m, int64_t ncells, const double* T, const double* p, const double* Y, double dt,
                       const df_integ_opts& base, int64_t sample, df_integ_opts* best, float* best_ms,
                       cudaStream_t st);
// advance the cells order[0 .. nwork) (nwork read from nwork_dev on the device
// when given; nwork is then an upper bound used to size the launch)
int launch_integrate_list(df_mech* m, int64_t ncells, double* T, const double* p, double* Y, double dt,
                          const df_integ_opts& o, int32_t* status, int32_t* nsub, const int32_t* order,
                          int64_t nwork, cudaStream_t st, const unsigned long long* nwork_dev = nullptr,
                          int nsteps = 1, double* t_ign = nullptr);

// generated thread-per-cell integrator (codegen.cu)
struct IntegArgs;
std::string jit_thread_source(const df_mech* m);
// launch the kernel generated for m with `threads` per block if it can (NVRTC
// available, the module compiled, a generated kernel for that block size);
// *launched says whether it did.  Errors only for a failed launch.
int jit_thread_launch(df_mech* m, int threads, int bps, const IntegArgs& a, cudaStream_t st, bool* launched);

// adjoint (adjoint.cu)
// with_stages: also room for the stored stages and LU factors of every
// accepted step (the reverse sweep then skips recomputing the step); false
// when the size does not fit in size_t
bool adjoint_workspace_bytes(const df_mech* m, int64_t ncells, int cap, bool with_stages, size_t* bytes);
// argument checks shared by df_chem_adjoint and df_chem_adjoint_static (api.cu):
// the cell count, dt, max_steps, every pointer (device memory; the cotangents,
// gradients and nsub may be NULL) and the options, which *o receives
int check_adjoint_call(const char* fn, const df_mech* m, int64_t ncells, double dt, int32_t max_steps,
                       const double* T0, const double* p, const double* Y0, const double* gT1, const double* gY1,
                       const double* gQ1, const double* gT0, const double* gY0, const double* g_lnA,
                       const int32_t* status, const int32_t* nsub, const df_integ_opts* opts, df_integ_opts* o);
// allow_stages: keep the stages when ws_bytes has room for them
int launch_adjoint(const df_mech* m, int64_t ncells, const double* T0, const double* p, const double* Y0,
                   double dt, const df_integ_opts& o, int cap, const double* gT1, const double* gY1,
                   const double* gQ1, double* gT0, double* gY0, double* g_lnA, int32_t* status, int32_t* nsub,
                   void* ws, size_t ws_bytes, bool allow_stages, cudaStream_t st);
}  // namespace df
