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
  int32_t block_threads;  /* 0 (with blocks_per_sm 0): the shape df_chem_autotune
                             chose for this mechanism and path, else 32; >0:
                             threads per block (a multiple of 32)             */
  int32_t blocks_per_sm;  /* 0: as many resident blocks as fit (or the tuned
                             value, see block_threads); >0: at most this many */
  int32_t order_by_T;     /* 1 (default): hand out cells hottest first (a device
                             counting sort; longest work first, lanes refilled
                             together get cells of similar stiffness)          */
  int32_t path;           /* 0: auto -- the path df_chem_autotune chose, else
                             thread per cell where a thread kernel exists (the
                             built species counts 3 and 9; with jit = 0 at
                             constant pressure the generated kernel for any
                             N <= 16, the warp path if it cannot be compiled),
                             else warp per cell; 1: thread per cell (error if
                             no thread kernel can run), 2: warp per cell       */
  int32_t reactor;        /* 0 (default): constant pressure, p[c] fixed and h
                             conserved; 1: constant volume (Sec. 2.2), the
                             density fixed from the initial p[c], T, Y and the
                             internal energy conserved (df_chem_integrate,
                             df_chem_integrate_steps, df_chem_autotune; the
                             adjoint and the DNN integrator are constant
                             pressure and reject 1 with DF_EUNSUPPORTED)       */
  int32_t jit;            /* 0 (default): on the thread-per-cell path at constant
                             pressure, use a kernel generated for the loaded
                             mechanism (its reaction structure as straight-line
                             code, compiled with NVRTC on first use and cached;
                             32- and 64-thread blocks; the same operations as
                             the mechanism-independent kernel, cells equal to
                             rounding), falling back to
                             that kernel when runtime compilation is
                             unavailable (df_chem_jit_info says why); compiled
                             modules are kept in an on-disk cache
                             ($DF_JIT_CACHE, "0" disables; else
                             $XDG_CACHE_HOME/df_chem_jit or
                             ~/.cache/df_chem_jit) keyed by the generated
                             source, the device headers, the architecture, the
                             NVRTC version, the compile options and the cache
                             entry format; 1: always the
                             mechanism-independent kernel                     */
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
 * pass, storing one checkpoint per accepted step, then sweeps back.  When the
 * workspace has room (df_chem_adjoint_workspace_size), the forward pass also
 * keeps each accepted step's stage vectors and LU factors and the reverse
 * sweep reads them back; with only the compact size (checkpoints and partials,
 * below) it recomputes each step instead.  Both give bitwise the same result.
 *
 *  T0, p, Y0     inputs as for df_chem_integrate (device, not modified)
 *  gT1, gY1, gQ1 cotangents (device; each may be NULL = 0)
 *  gT0 [ncells], gY0 [N*ncells] (device, may be NULL): dL/dT0, dL/dY0
 *  g_lnA [M] (device, may be NULL): dL/d ln A_j summed over cells (summation
 *                order fixed: bitwise reproducible)
 *  status, nsub [ncells] (device; nsub may be NULL): per-cell status and number
 *                of accepted steps; a cell with more than max_steps accepted
 *                steps gets DF_CELL_MAXSTEPS and a zero gradient
 *  workspace     device memory owned by the caller: at least the compact size
 *                8 * (ncells*max_steps*(N+2) + ceil(ncells/16)*M) + 256
 *                bytes (the ln A partial sums take ceil(ncells/B)*M doubles,
 *                B the 16 to 32 cells of one block, which the library picks
 *                from the device's shared memory); df_chem_adjoint_workspace_size() returns the size with
 *                the stored stages, 8 * ncells*max_steps*(7n + n^2) bytes more
 *                (n = N + 1).  On return its first ncells*max_steps*(N+2)
 *                doubles hold the checkpoints [cell][step][T, Y_1..Y_N, h] of
 *                the accepted steps.
 * Built for mechanisms of 3 and 9 species (one cell per thread); other sizes
 * return DF_EUNSUPPORTED.  Errors: DF_EINVAL, DF_EWORKSPACE, DF_EUNSUPPORTED,
 * DF_ECUDA. */
int df_chem_adjoint_workspace_size(const df_mech* mech, int64_t ncells, int32_t max_steps, size_t* bytes);
int df_chem_adjoint(const df_mech* mech, int64_t ncells, const double* T0, const double* p, const double* Y0,
                    double dt, const df_integ_opts* opts, int32_t max_steps, const double* gT1,
                    const double* gY1, const double* gQ1, double* gT0, double* gY0, double* g_lnA,
                    int32_t* status, int32_t* nsub, void* workspace, size_t ws_bytes, df_stream_t stream);

/* df_chem_adjoint without a workspace argument, for callers that cannot
 * allocate device memory when they need the gradient (an application whose
 * device memory belongs to a pool or framework that must not be bypassed, a
 * real-time loop that forbids allocation after start-up).  The paper has no
 * counterpart.
 *
 * Arguments, argument checks (every pointer must be device memory; the
 * cotangents, gradients and nsub may be NULL) and results as for
 * df_chem_adjoint.  The scratch (checkpoints and
 * ln A partial sums) lives in one fixed 4 MiB device array inside the library,
 * held by every GPU that loads it until the process exits; nothing is
 * allocated.  Requests that need more (ncells * max_steps * (N + 2) doubles of
 * checkpoints plus at most ceil(ncells / 16) * M doubles of partials, in total
 * more than 4 MiB) return DF_EWORKSPACE with the size in the error detail.  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the one array: calls whose kernels
 * overlap on the GPU (different streams, or several threads) race on it and
 * must be serialised by the caller. */
int df_chem_adjoint_static(const df_mech* mech, int64_t ncells, const double* T0, const double* p,
                           const double* Y0, double dt, const df_integ_opts* opts, int32_t max_steps,
                           const double* gT1, const double* gY1, const double* gQ1, double* gT0, double* gY0,
                           double* g_lnA, int32_t* status, int32_t* nsub, df_stream_t stream);

/* Advance every cell by nsteps consecutive steps of dt (the repeated CFD step
 * of the 0D ignition runs, Sec. 4.1) in one persistent launch, and report each
 * cell's ignition delay as the paper defines it (Sec. 4.1: from [dT/dt]_max).
 * Same arguments and per-cell status as df_chem_integrate, plus:
 *   nsteps >= 1: the substep sequence stops at every multiple of dt (the
 *     step-size controller carries h across the boundaries); max_substeps in
 *     opts bounds the total over all steps;
 *   nsub [ncells] (may be NULL): accepted substeps over all steps;
 *   t_ign [ncells] (device, may be NULL): the time in [0, nsteps*dt) of the
 *     largest dT/dt: the largest among the states at which accepted substeps
 *     start (the integrator evaluates f there anyway), its time refined by the
 *     vertex of the parabola through that sample and its two neighbours (the
 *     sample's own time at either end of the run); NaN for a failed cell.
 * With nsteps = 1 the result equals df_chem_integrate's.  Errors: DF_EINVAL
 * (also nsteps < 1), DF_ECUDA.  Asynchronous on `stream`. */
int df_chem_integrate_steps(const df_mech* mech, int64_t ncells, double* T, const double* p, double* Y,
                            double dt, int32_t nsteps, const df_integ_opts* opts, int32_t* status,
                            int32_t* nsub, double* t_ign, df_stream_t stream);

/* Choose the integrator's launch shape for this mechanism by timing (the GPU
 * form of the paper's dynamic load balancing, Sec. 3.2: the shape that keeps
 * the lanes of a persistent launch busiest on a given mix of cell stiffness).
 * The first `sample` cells (0: min(ncells, 65536)) of T, p, Y (device, layout
 * of df_chem_integrate, ncells the array stride) are copied to library scratch
 * (the inputs are not modified) and advanced over dt with every candidate:
 * thread per cell 32/64/96/128 threads per block x at most 0 (all that fit)/1/2
 * blocks per SM; warp per cell 64/128/256 threads per block; each with and
 * without hottest-first ordering; two timed runs each, fastest kept.  The
 * winner is cached in the handle: later df_chem_integrate calls whose options
 * leave block_threads and blocks_per_sm at 0 use it (order_by_T stays as the
 * caller passes it).  *best (may be NULL) receives `base` with the winning
 * block_threads, blocks_per_sm, order_by_T and path; *best_ms (may be NULL)
 * its time on the sample.  Synchronous (waits for `stream`); allocates and
 * frees device scratch, so do not call it during a stream capture.  Errors:
 * DF_EINVAL, DF_ECUDA, DF_ENOMEM, DF_EUNSUPPORTED (no candidate fits). */
int df_chem_autotune(df_mech* mech, int64_t ncells, const double* T, const double* p, const double* Y,
                     double dt, const df_integ_opts* base, int64_t sample, df_integ_opts* best,
                     float* best_ms, df_stream_t stream);

/* The kernel generated for this mechanism (df_integ_opts.jit): *used = 1 when
 * the last thread-per-cell integrator launch on this handle ran it, else 0;
 * detail (may be NULL, n bytes, NUL-terminated) receives its state: the NVRTC
 * compile time, or why it is unavailable (NVRTC or the device headers not
 * found, a compilation failure) -- then the mechanism-independent kernel ran.
 * Errors: DF_EINVAL (null handle or used). */
int df_chem_jit_info(const df_mech* mech, int32_t* used, char* detail, size_t n);

/* The CUDA C++ source of the kernel generated for a mechanism file (what
 * df_integ_opts.jit = 0 compiles; host only, no device needed), for
 * inspection and for compiling it ahead of use.  The file is parsed as by
 * df_mech_load.  buf (may be NULL) receives up to n bytes, NUL-terminated;
 * *needed (may be NULL) the full size including the NUL.  Errors: DF_EINVAL,
 * DF_EMECH (file or content). */
int df_mech_generated_source(const char* mech_json_path, char* buf, size_t n, size_t* needed);

/* Work counters of the last df_chem_integrate on this handle (host values; the
 * call synchronises `stream`): accepted and rejected substeps summed over all
 * cells. */
int df_chem_last_stats(const df_mech* mech, int64_t* accepted, int64_t* rejected,
                       df_stream_t stream);

/* ---------------------------------------------------------------------------
 * DNN chemistry integrator (Sec. 2.3 and Sec. 3.2 DNNInferencer): a fully
 * connected network with three hidden layers maps x = {T, p, F(Y_1..Y_N)} to the
 * change u of F(Y) over dt, F the Box-Cox transform F(Y) = (max(Y,0)^lambda - 1)
 * / lambda.  Inference follows the three stages of DNNInferencer.inference:
 * (1) Box-Cox + normalisation of (p, T, Y), (2) the network, (3) the inverse
 * transform to Y(t + dt); then T(t + dt) from h(T', Y') = h(T, Y) at fixed p
 * (correctThermo, Sec. 3.2).  Cells outside the training range are advanced
 * by df_chem_integrate instead (FP64 fallback).
 *
 * Network: BF16 weights and activations, FP32 accumulation on the tensor
 * cores, FP32 bias + exact-erf GELU, then rounding to BF16 (the rounding
 * points of every layer); FP32 master weights and Adam moments for training.
 * ------------------------------------------------------------------------- */
typedef struct df_dnn df_dnn;

typedef struct df_dnn_opts {
  int32_t n_species;   /* N: 2 + N inputs (<= 16), N outputs (<= 16)               */
  int32_t width[3];    /* hidden widths, multiples of 8 (default 1600, 800, 400)   */
  double lambda;       /* Box-Cox lambda (default 0.1); 1/lambda must be an integer */
  int32_t batch;       /* rows per training step (default 4096)                    */
  int32_t infer_chunk; /* cells per inference chunk (default 262144)               */
  double beta1, beta2, adam_eps; /* Adam (0.9, 0.999, 1e-8)                        */
  double range_margin; /* fraction of the training range accepted outside it (0)  */
  int32_t reserved[4];
} df_dnn_opts;

void df_dnn_opts_default(df_dnn_opts* opts);

/* Create a network with Glorot-uniform weights drawn from `seed` (the library's
 * own counter-based generator) and zero biases; normalisation identity. */
int df_dnn_create(const df_dnn_opts* opts, uint64_t seed, df_dnn** out);
void df_dnn_free(df_dnn* dnn);

/* Normalisation and range statistics (host arrays): mean_in, std_in, in_min,
 * in_max have 2 + N entries (T, p, F(Y_1..N)); mean_out, std_out have N
 * entries (the change of F(Y) over dt).  Any pointer may be NULL (keep). */
int df_dnn_set_norm(df_dnn* dnn, const float* mean_in, const float* std_in, const float* mean_out,
                    const float* std_out, const float* in_min, const float* in_max);
int df_dnn_get_norm(const df_dnn* dnn, float* mean_in, float* std_in, float* mean_out, float* std_out,
                    float* in_min, float* in_max);

/* Compute the statistics above from n training pairs (T, p, Y) -> Y_next on the
 * device (FP64 accumulation, fixed summation order) and store them in the
 * handle.  Device arrays, SoA as for the integrator.  Synchronises `stream`. */
int df_dnn_fit_norm(df_dnn* dnn, int64_t n, const double* T, const double* p, const double* Y,
                    const double* Y_next, df_stream_t stream);

/* One Adam step on a batch of n pairs (n <= opts.batch): loss = mean over rows
 * and the N outputs of the squared error of the normalised change of F(Y).
 * lr: learning rate of this step.  loss_out (host, may be NULL): the batch loss
 * before the update (synchronises `stream`). */
int df_dnn_train_step(df_dnn* dnn, int64_t n, const double* T, const double* p, const double* Y,
                      const double* Y_next, float lr, float* loss_out, df_stream_t stream);

/* The training step in two halves, for data-parallel training over several
 * GPUs (each rank holds a shard of the training pairs; the paper names
 * multi-GPU DNN work as future work, Sec. 6):
 *  df_dnn_grad: the forward and backward pass of df_dnn_train_step on n pairs
 *    (same arguments, no lr), leaving in the handle's FP32 gradient buffer the
 *    gradient of this shard's share of a loss averaged over n_total >= n rows:
 *    sum over the n rows and N outputs of the squared error / (n_total N).
 *    With n_total = n it is df_dnn_train_step's gradient; with n_total the
 *    rows of all ranks, summing the buffers over the ranks gives the gradient
 *    of the whole batch (every row's output gradient, and its BF16 rounding,
 *    the same as in one pass over the union).  loss_out (host, may be NULL):
 *    this shard's share of the loss, same normalisation.  The parameters are
 *    not changed.
 *  df_dnn_grad_buffer: *grads receives the device address of that buffer
 *    (df_dnn_param_count() floats, layout of df_dnn_get_params), *count (may be
 *    NULL) its length, so the caller can all-reduce it in place (sum over the
 *    ranks) between the two halves.  The handle owns the buffer.
 *  df_dnn_adam_step: one Adam step (the handle's step counter advances, as in
 *    df_dnn_train_step) with the gradient now in the buffer, then the BF16
 *    weight copies.
 * df_dnn_grad (n_total = n) then df_dnn_adam_step equals df_dnn_train_step.
 * Asynchronous on `stream` except for loss_out, which synchronises it. */
int df_dnn_grad(df_dnn* dnn, int64_t n, int64_t n_total, const double* T, const double* p, const double* Y,
                const double* Y_next, float* loss_out, df_stream_t stream);
int df_dnn_grad_buffer(df_dnn* dnn, float** grads, int64_t* count);
int df_dnn_adam_step(df_dnn* dnn, float lr, df_stream_t stream);

/* Adam state (host buffers of df_dnn_param_count() floats each, may be NULL):
 * the first and second moment estimates, and the number of steps taken. */
int df_dnn_get_adam_state(const df_dnn* dnn, float* m1, float* m2, int64_t* step);

/* Advance ncells cells over dt with the network (T, Y in/out, device).  Cells
 * whose inputs leave the training range [in_min, in_max] (widened by
 * range_margin) are advanced by df_chem_integrate with fallback_opts (NULL =
 * defaults) on `mech`.  used_fallback [ncells] (device, may be NULL): 1 for
 * those cells.  n_fallback (host, may be NULL): their count.  status [ncells]
 * (device, may be NULL): DF_CELL_* (network cells are DF_CELL_OK).
 * Synchronises `stream` once (to size the fallback launch). */
int df_dnn_infer(df_dnn* dnn, const df_mech* mech, int64_t ncells, double* T, const double* p, double* Y,
                 double dt, const df_integ_opts* fallback_opts, int32_t* used_fallback, int64_t* n_fallback,
                 int32_t* status, df_stream_t stream);

/* The network's raw output for prepared inputs: X [n][16] bf16 features as the
 * network sees them (device), U [n][16] f32 (device).  For checking the layers. */
int df_dnn_forward_raw(df_dnn* dnn, int64_t n, const void* X, float* U, df_stream_t stream);

/* FP32 master parameters in the order W1[w1][16], b1[w1], W2[w2][w1], b2, W3[w3][w2],
 * b3, W4[16][w3], b4[16] (host buffer of df_dnn_param_count() floats).  get_grads
 * copies the gradients of the last training step in the same layout. */
int64_t df_dnn_param_count(const df_dnn* dnn);
int df_dnn_get_params(const df_dnn* dnn, float* host);
int df_dnn_set_params(df_dnn* dnn, const float* host);
int df_dnn_get_grads(const df_dnn* dnn, float* host);

/* Save / load options, normalisation and parameters (binary file). */
int df_dnn_save(const df_dnn* dnn, const char* path);
int df_dnn_load(const char* path, df_dnn** out);

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
