/*
 * df_chem.h - C ABI of the GB300 per-cell chemistry substep library.
 *
 * The library advances the thermochemical state of many independent cells
 * over one CFD step dt: each cell is a constant-pressure adiabatic 0D reactor
 * (the df0DFoam problem of Sec. 2.2), whose species obey the reaction-system
 * source term of Sec. 2.3 eq. (sourceeq) and whose temperature follows from the
 * conserved enthalpy (Sec. 3.2, correctThermo from h, p, Y).  This is the work
 * that dfChemistryModel::solve() hands to CVODE (Sec. 2.3) or to the DNN
 * integrator (Sec. 2.3, Sec. 3.2 DNNInferencer).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: 0 on success, a negative DF_E* code on a whole-call error.
 *    df_strerror() names a code; df_get_last_error_detail() gives the message
 *    of the last failing call of the calling thread.
 *  - Per-cell numerical failures do NOT fail the call: they are reported in
 *    status[c] (DF_CELL_*), and that cell's state is left as it was on input.
 *  - Device arrays: every array argument named as device memory is a pointer
 *    into the memory of the current CUDA device, owned by the caller,
 *    contiguous, FP64 unless stated.  The library never frees them.
 *  - Cell layout (structure of arrays): T[c], p[c] have ncells entries;
 *    Y is species-major, Y[k * ncells + c] for species k of cell c.
 *  - Units at the boundary: T in K, p in Pa, dt in s, Y mass fractions,
 *    heat release in W/m^3.  The mechanism file gives A in cm-mol-s units and
 *    Ea in kJ/mol.
 *  - Streams: calls are asynchronous on the given stream (a cudaStream_t passed
 *    as void*; NULL is the legacy default stream) unless stated otherwise.
 *  - Handles (df_mech, df_dnn) own their device copies and scratch memory.
 *    A handle may be used by one stream at a time.
 */
#ifndef DF_CHEM_H
#define DF_CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* whole-call error codes */
#define DF_OK 0
#define DF_EINVAL (-1)     /* bad argument (null pointer, size, option)            */
#define DF_ENOMEM (-2)     /* device or host allocation failed                     */
#define DF_ECUDA (-3)      /* a CUDA runtime call failed                           */
#define DF_EMECH (-4)      /* mechanism file missing, unparsable or inconsistent   */
#define DF_EWORKSPACE (-5) /* workspace too small                                  */
#define DF_ETIMEOUT (-6)   /* a bounded device wait ran out                        */
#define DF_EUNSUPPORTED (-7) /* size or feature outside what the library builds    */

/* per-cell status codes (status[c]) */
#define DF_CELL_OK 0
#define DF_CELL_MAXSTEPS 1  /* max_substeps reached before t = dt                  */
#define DF_CELL_NONFINITE 2 /* non-finite or non-positive-T input, or a NaN state  */
#define DF_CELL_HMIN 3      /* step size fell below h_min                          */

typedef void* df_stream_t; /* a cudaStream_t */
typedef struct df_mech df_mech;

/* Integrator options.  Fill with df_integ_opts_default() and override. */
typedef struct df_integ_opts {
  double rtol;          /* relative tolerance of the local error test          */
  double atol_Y;        /* absolute tolerance on mass fractions                */
  double atol_T;        /* absolute tolerance on temperature [K]               */
  double h0;            /* first substep [s]                                   */
  double h_min;         /* smallest allowed substep [s]                        */
  int32_t max_substeps; /* accepted + rejected substeps allowed per cell       */
  int32_t method;       /* 0: RODAS4 (Hairer & Wanner), 1: RODAS3 (Sandu 1997) */
  int32_t block_threads;  /* 0: autotune; else threads per block               */
  int32_t blocks_per_sm;  /* 0: autotune; else resident blocks per SM          */
  int32_t order_by_T;     /* 1: hand out hot cells first (longest-work first)  */
  int32_t path;           /* 0: auto (thread per cell if N <= 16), 1: thread per
                             cell, 2: warp per cell                            */
  int32_t reserved[2];
} df_integ_opts;

void df_integ_opts_default(df_integ_opts* opts);

/* ---------------------------------------------------------------------------
 * Mechanism: species (W, NASA-7) and reactions (nu', nu'', Arrhenius A, b, Ea,
 * third-body efficiencies, Troe falloff), Sec. 2.3 eq. (reaction).
 * ------------------------------------------------------------------------- */

/* Parse the mechanism JSON at `path` and upload it to the current device.
 * On success *out owns the host and device copies; free with df_mech_free.
 * Errors: DF_EINVAL (null argument), DF_EMECH (file or content), DF_ECUDA,
 * DF_ENOMEM.  Limits: up to 64 species, 4096 reactions, 3 species entries per
 * side.  Not asynchronous (synchronises the device once). */
int df_mech_load(const char* path, df_mech** out);

/* Release a mechanism handle (NULL is ignored). */
void df_mech_free(df_mech* mech);

/* Species and reaction counts. */
int df_mech_info(const df_mech* mech, int* n_species, int* n_reactions);

/* Replace the natural logs of the pre-exponential factors by the M values at
 * the device pointer lnA (device memory, M doubles; copied on `stream` before
 * any later call on that stream reads them).  For Troe reactions the same
 * shift ln A - ln A_file scales k_inf and k_0 together.  lnA == NULL restores
 * the file's values. */
int df_mech_set_lnA(df_mech* mech, const double* lnA, df_stream_t stream);

/* ---------------------------------------------------------------------------
 * Right-hand side and Jacobian (diagnostic entry points; same device code as
 * the integrator).
 * ------------------------------------------------------------------------- */

/* dydt[(i) * ncells + c], i = 0 for dT/dt [K/s], i = 1 + k for dY_k/dt [1/s]
 * (Sec. 2.3 eq. (sourceeq) divided by rho; dT/dt = -sum_k H_k wdot_k/(rho cp)).
 * qdot[c] = -sum_k H_k wdot_k [W/m^3] (may be NULL).  All device memory. */
int df_chem_rhs(const df_mech* mech, int64_t ncells, const double* T, const double* p,
                const double* Y, double* dydt, double* qdot, df_stream_t stream);

/* Analytic Jacobian d(dT/dt, dY/dt)/d(T, Y) at constant p.
 * J[c * n * n + i * n + j] = d f_i / d y_j, n = N + 1, y = (T, Y_1..Y_N).
 * Device memory. */
int df_chem_jacobian(const df_mech* mech, int64_t ncells, const double* T, const double* p,
                     const double* Y, double* J, df_stream_t stream);

/* ---------------------------------------------------------------------------
 * Integrator: advance every cell from t = 0 to t = dt (the chemistry substep
 * that Sec. 2.3 hands to CVODE), with an adaptive L-stable Rosenbrock method,
 * analytic Jacobian and per-cell dense LU.
 *
 *  T [ncells] in/out, p [ncells] in, Y [N * ncells] in/out   (device)
 *  status [ncells] out (DF_CELL_*)                            (device)
 *  nsub  [ncells] out, accepted substeps per cell; may be NULL (device)
 *  opts: NULL means df_integ_opts_default().
 *
 * Cells run in one persistent launch in which each lane takes a new cell from
 * a device work counter as soon as its cell finishes (cells of very different
 * stiffness share the GPU without idle lanes).  N <= 16 runs one cell per
 * thread; larger mechanisms run one cell per warp.
 * ------------------------------------------------------------------------- */
int df_chem_integrate(const df_mech* mech, int64_t ncells, double* T, const double* p, double* Y,
                      double dt, const df_integ_opts* opts, int32_t* status, int32_t* nsub,
                      df_stream_t stream);

/* ---------------------------------------------------------------------------
 * Discrete adjoint of the integrator (an extension beyond the paper: kinetic
 * sensitivity and calibration of the chemistry substep of Sec. 2.3).
 *
 * Gradient of L = sum_c [ gT1[c] T_c(dt) + sum_k gY1[k*ncells+c] Y_kc(dt)
 *                         + gQ1[c] qdot_c(dt) ]
 * (qdot = -sum_k H_k wdot_k in W/m^3 at the final state) with respect to each
 * cell's initial T, Y and to ln A_j of every reaction, for the map the
 * integrator computes with RODAS4 and the given options, its accepted step
 * sequence held fixed (discrete adjoint).  The call recomputes the forward
 * pass, storing one checkpoint per accepted step, then sweeps back.
 *
 *  T0, p, Y0     inputs as for df_chem_integrate (device, not modified)
 *  gT1, gY1, gQ1 cotangents (device; each may be NULL = 0)
 *  gT0 [ncells], gY0 [N*ncells] (device, may be NULL): dL/dT0, dL/dY0
 *  g_lnA [M] (device, may be NULL): dL/d ln A_j summed over cells (summation
 *                order fixed: bitwise reproducible)
 *  status, nsub [ncells] (device; nsub may be NULL): per-cell status and number
 *                of accepted steps; a cell with more than max_steps accepted
 *                steps gets DF_CELL_MAXSTEPS and a zero gradient
 *  workspace     device memory of at least df_chem_adjoint_workspace_size()
 *                bytes, owned by the caller.  On return its first
 *                ncells*max_steps*(N+2) doubles hold the checkpoints
 *                [cell][step][T, Y_1..Y_N, h] of the accepted steps.
 * Built for mechanisms of 3 and 9 species (one cell per thread); other sizes
 * return DF_EUNSUPPORTED.  Errors: DF_EINVAL, DF_EWORKSPACE, DF_EUNSUPPORTED,
 * DF_ECUDA. */
int df_chem_adjoint_workspace_size(const df_mech* mech, int64_t ncells, int32_t max_steps, size_t* bytes);
int df_chem_adjoint(const df_mech* mech, int64_t ncells, const double* T0, const double* p, const double* Y0,
                    double dt, const df_integ_opts* opts, int32_t max_steps, const double* gT1,
                    const double* gY1, const double* gQ1, double* gT0, double* gY0, double* g_lnA,
                    int32_t* status, int32_t* nsub, void* workspace, size_t ws_bytes, df_stream_t stream);

/* Work counters of the last df_chem_integrate on this handle (host values; the
 * call synchronises `stream`): accepted and rejected substeps summed over all
 * cells. */
int df_chem_last_stats(const df_mech* mech, int64_t* accepted, int64_t* rejected,
                       df_stream_t stream);

/* ---------------------------------------------------------------------------
 * errors
 * ------------------------------------------------------------------------- */
const char* df_strerror(int code);
/* Copy the last error message of the calling thread into buf (NUL-terminated,
 * truncated to n bytes).  Returns its full length. */
int df_get_last_error_detail(char* buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* DF_CHEM_H */
