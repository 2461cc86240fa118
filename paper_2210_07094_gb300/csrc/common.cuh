// Internal definitions shared by the library's translation units.
//
// Mechanism blob: one contiguous FP64 array holding the species and reaction
// data of a mechanism (Sec. 2.3 eq. (reaction): nu'_{aj}, nu''_{aj}; Arrhenius
// K_f; third-body efficiencies; Troe falloff; NASA-7 thermo).  The same bytes
// live in device memory and are staged into shared memory by the kernels, so
// every record has a fixed size and an 8-byte alignment.
#pragma once
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/df_chem.h"

namespace df {

// physical constants (cgs inside the kernels)
constexpr double RU = 8.314462618e7;         // erg/(mol K)
constexpr double RU_SI = 8.314462618;        // J/(mol K)
constexpr double P_STD = 1.01325e6;          // standard-state pressure, dyn/cm^2
constexpr double LN10 = 2.302585092994045684;
constexpr double LOG_PSTD_RU = -4.4074185890025275;     // ln(P_STD / RU), RU in erg/(mol K)

constexpr int MAX_SPECIES = 64;
constexpr int MAX_REACTIONS = 4096;
constexpr int THREAD_PATH_MAX_N = 16;   // N <= this runs one cell per thread

// --- blob layout (all in doubles) -----------------------------------------
// species record k (SP_REC doubles):   W, 1/W, a1..a7, then the NASA-7
//   coefficients as the enthalpy and entropy polynomials use them:
//   a2/2, a3/3, a4/4, a5/5 (h/RT) and a3/2, a4/3, a5/4 (s/R)
constexpr int SP_REC = 16;
constexpr int SP_H = 9;   // offset of a2/2 .. a5/5
constexpr int SP_S = 13;  // offset of a3/2 .. a5/4
// reaction record j (RX_REC doubles):  lnA, beta, Ea/R, meta0, meta1
//   meta0 (8 bytes): reac[3], prod[3] species indices, nr | np << 4, flags
//     flags: bit0-1 type (0 elementary, 1 third-body, 2 Troe), bit2 reversible
//   meta1 (8 bytes): int32 effslot (-1: none), int32 troeslot (-1: none)
constexpr int RX_REC = 5;
// Troe record (TR_REC doubles): lnA0 - lnA, beta0, Ea0/R, alpha, 1/T***, 1/T*, T**, pad
constexpr int TR_REC = 8;
// efficiency record: N doubles per third-body / falloff reaction

struct RxMeta {
  uint8_t reac[3];
  uint8_t prod[3];
  uint8_t nrnp;
  uint8_t flags;
};
static_assert(sizeof(RxMeta) == 8, "meta layout");
struct RxSlots {
  int32_t eff;
  int32_t troe;
};
static_assert(sizeof(RxSlots) == 8, "slot layout");

struct MechDims {
  int N, M, n_eff, n_troe;
  int off_sp, off_rx, off_tr, off_eff, total;  // offsets in doubles
};

inline MechDims mech_dims(int N, int M, int n_eff, int n_troe) {
  MechDims d;
  d.N = N;
  d.M = M;
  d.n_eff = n_eff;
  d.n_troe = n_troe;
  d.off_sp = 0;
  d.off_rx = d.off_sp + SP_REC * N;
  d.off_tr = d.off_rx + RX_REC * M;
  d.off_eff = d.off_tr + TR_REC * n_troe;
  d.total = d.off_eff + n_eff * N;
  return d;
}

}  // namespace df

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

// adjoint (adjoint.cu)
// with_stages: also room for the stored stages and LU factors of every
// accepted step (the reverse sweep then skips recomputing the step)
size_t adjoint_workspace_bytes(const df_mech* m, int64_t ncells, int cap, bool with_stages);
// allow_stages: keep the stages when ws_bytes has room for them
int launch_adjoint(const df_mech* m, int64_t ncells, const double* T0, const double* p, const double* Y0,
                   double dt, const df_integ_opts& o, int cap, const double* gT1, const double* gY1,
                   const double* gQ1, double* gT0, double* gY0, double* g_lnA, int32_t* status, int32_t* nsub,
                   void* ws, size_t ws_bytes, bool allow_stages, cudaStream_t st);
}  // namespace df
