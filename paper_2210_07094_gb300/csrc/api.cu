// C-ABI entry points: argument checks, handle life cycle, error reporting.
// Every compute step runs in the kernels of integrate.cu (and the other .cu
// files); this file only validates and forwards.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"

namespace df {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DF_OK;
  return set_error(e == cudaErrorMemoryAllocation ? DF_ENOMEM : DF_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

static bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace df

using namespace df;

extern "C" {

void df_integ_opts_default(df_integ_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  // tolerances chosen against the CPU oracle: on the seeded 9- and 50-species
  // workloads they keep |dT| <= 1e-7 K and |dY| <= 4e-11 max Y (three orders of
  // magnitude inside 1e-3 K and 1e-7 max Y)
  o->rtol = 1e-6;
  o->atol_Y = 1e-10;
  o->atol_T = 1e-6;
  o->h0 = 1e-6;
  o->h_min = 1e-22;
  o->max_substeps = 100000;
  o->method = 0;
  o->block_threads = 0;
  o->blocks_per_sm = 0;
  o->order_by_T = 1;
}

const char* df_strerror(int code) {
  switch (code) {
    case DF_OK: return "success";
    case DF_EINVAL: return "invalid argument";
    case DF_ENOMEM: return "out of memory";
    case DF_ECUDA: return "CUDA error";
    case DF_EMECH: return "invalid mechanism";
    case DF_EWORKSPACE: return "workspace too small";
    case DF_ETIMEOUT: return "bounded device wait ran out";
    case DF_EUNSUPPORTED: return "unsupported size or feature";
    default: return "unknown error";
  }
}

int df_get_last_error_detail(char* buf, size_t n) {
  const std::string& s = g_last_error;
  if (buf && n > 0) {
    size_t k = s.size() < n - 1 ? s.size() : n - 1;
    memcpy(buf, s.data(), k);
    buf[k] = 0;
  }
  return (int)s.size();
}

int df_mech_load(const char* path, df_mech** out) {
  if (!path || !out) return set_error(DF_EINVAL, "df_mech_load: null argument");
  *out = nullptr;
  df_mech* m = new (std::nothrow) df_mech();
  if (!m) return set_error(DF_ENOMEM, "df_mech_load: host allocation");
  int rc = parse_mechanism(path, m);
  if (rc) {
    delete m;
    return rc;
  }
  rc = cuda_check(cudaGetDevice(&m->device), "cudaGetDevice");
  cudaDeviceProp prop;
  if (!rc) rc = cuda_check(cudaGetDeviceProperties(&prop, m->device), "cudaGetDeviceProperties");
  if (!rc) {
    m->num_sms = prop.multiProcessorCount;
    m->max_smem_optin = prop.sharedMemPerBlockOptin;
    m->smem_per_sm = prop.sharedMemPerMultiprocessor;
    m->smem_reserved_per_block = prop.reservedSharedMemPerBlock;
  }
  if (!rc) rc = cuda_check(cudaMalloc(&m->blob_dev, sizeof(double) * m->dims.total + 8), "cudaMalloc blob");
  if (!rc)
    rc = cuda_check(cudaMemcpy(m->blob_dev, m->blob_host.data(), sizeof(double) * m->dims.total,
                               cudaMemcpyHostToDevice),
                    "upload mechanism");
  if (!rc) rc = cuda_check(cudaMalloc(&m->csr_dev, sizeof(int) * m->csr_host.size()), "cudaMalloc csr");
  if (!rc)
    rc = cuda_check(cudaMemcpy(m->csr_dev, m->csr_host.data(), sizeof(int) * m->csr_host.size(),
                               cudaMemcpyHostToDevice),
                    "upload species lists");
  if (!rc) rc = cuda_check(cudaMalloc(&m->counters, 4 * sizeof(unsigned long long)), "cudaMalloc counters");
  if (!rc) rc = cuda_check(cudaMemset(m->counters, 0, 4 * sizeof(unsigned long long)), "clear counters");
  if (rc) {
    df_mech_free(m);
    return rc;
  }
  *out = m;
  return DF_OK;
}

void df_mech_free(df_mech* m) {
  if (!m) return;
  if (m->blob_dev) cudaFree(m->blob_dev);
  if (m->counters) cudaFree(m->counters);
  if (m->csr_dev) cudaFree(m->csr_dev);
  if (m->order) cudaFree(m->order);
  if (m->bins) cudaFree(m->bins);
  delete m;
}

int df_mech_info(const df_mech* m, int* n_species, int* n_reactions) {
  if (!m) return set_error(DF_EINVAL, "df_mech_info: null handle");
  if (n_species) *n_species = m->dims.N;
  if (n_reactions) *n_reactions = m->dims.M;
  return DF_OK;
}

int df_mech_set_lnA(df_mech* m, const double* lnA, df_stream_t stream) {
  if (!m) return set_error(DF_EINVAL, "df_mech_set_lnA: null handle");
  if (lnA && !is_device_ptr(lnA)) return set_error(DF_EINVAL, "df_mech_set_lnA: lnA must be device memory");
  return launch_set_lnA(m, lnA, (cudaStream_t)stream);
}

static int check_cells(const char* fn, const df_mech* m, int64_t ncells) {
  if (!m) return set_error(DF_EINVAL, std::string(fn) + ": null mechanism");
  if (ncells < 0 || ncells > (int64_t)1 << 31)
    return set_error(DF_EINVAL, std::string(fn) + ": ncells must be in [0, 2^31]");
  return DF_OK;
}

static int check_dev(const char* fn, const char* name, const void* p) {
  if (!is_device_ptr(p)) return set_error(DF_EINVAL, std::string(fn) + ": " + name + " must be device memory");
  return DF_OK;
}

}  // extern "C"

namespace df {
int check_adjoint_call(const char* fn, const df_mech* m, int64_t ncells, double dt, int32_t max_steps,
                       const double* T0, const double* p, const double* Y0, const double* gT1, const double* gY1,
                       const double* gQ1, const double* gT0, const double* gY0, const double* g_lnA,
                       const int32_t* status, const int32_t* nsub, const df_integ_opts* opts, df_integ_opts* o) {
  int rc = check_cells(fn, m, ncells);
  if (rc || ncells == 0) return rc;
  if (!(dt >= 0.0) || !std::isfinite(dt) || max_steps < 1)
    return set_error(DF_EINVAL, std::string(fn) + ": dt must be finite and >= 0, max_steps >= 1");
  if ((rc = check_dev(fn, "T0", T0)) || (rc = check_dev(fn, "p", p)) || (rc = check_dev(fn, "Y0", Y0)) ||
      (rc = check_dev(fn, "status", status)))
    return rc;
  const void* opt_ptrs[] = {gT1, gY1, gQ1, gT0, gY0, g_lnA, nsub};
  const char* opt_names[] = {"gT1", "gY1", "gQ1", "gT0", "gY0", "g_lnA", "nsub"};
  for (int i = 0; i < 7; ++i)
    if (opt_ptrs[i] && (rc = check_dev(fn, opt_names[i], opt_ptrs[i]))) return rc;
  if (opts) *o = *opts;
  else df_integ_opts_default(o);
  if (o->reactor != 0) return set_error(DF_EUNSUPPORTED, std::string(fn) + ": constant-pressure reactor only");
  if (!(o->rtol > 0.0) || !(o->atol_Y > 0.0) || !(o->atol_T > 0.0) || !(o->h0 > 0.0) || !(o->h_min >= 0.0) ||
      o->max_substeps < 1)
    return set_error(DF_EINVAL, std::string(fn) + ": invalid options");
  return DF_OK;
}
}  // namespace df

extern "C" {

int df_chem_rhs(const df_mech* m, int64_t ncells, const double* T, const double* p, const double* Y,
                double* dydt, double* qdot, df_stream_t stream) {
  int rc = check_cells("df_chem_rhs", m, ncells);
  if (rc || ncells == 0) return rc;
  if ((rc = check_dev("df_chem_rhs", "T", T)) || (rc = check_dev("df_chem_rhs", "p", p)) ||
      (rc = check_dev("df_chem_rhs", "Y", Y)) || (rc = check_dev("df_chem_rhs", "dydt", dydt)))
    return rc;
  if (qdot && (rc = check_dev("df_chem_rhs", "qdot", qdot))) return rc;
  return launch_rhs(m, ncells, T, p, Y, dydt, qdot, (cudaStream_t)stream);
}

int df_chem_jacobian(const df_mech* m, int64_t ncells, const double* T, const double* p,
                     const double* Y, double* J, df_stream_t stream) {
  int rc = check_cells("df_chem_jacobian", m, ncells);
  if (rc || ncells == 0) return rc;
  if ((rc = check_dev("df_chem_jacobian", "T", T)) || (rc = check_dev("df_chem_jacobian", "p", p)) ||
      (rc = check_dev("df_chem_jacobian", "Y", Y)) || (rc = check_dev("df_chem_jacobian", "J", J)))
    return rc;
  return launch_jacobian(m, ncells, T, p, Y, J, (cudaStream_t)stream);
}

int df_chem_integrate(const df_mech* mc, int64_t ncells, double* T, const double* p, double* Y, double dt,
                      const df_integ_opts* opts, int32_t* status, int32_t* nsub, df_stream_t stream) {
  df_mech* m = const_cast<df_mech*>(mc);
  int rc = check_cells("df_chem_integrate", m, ncells);
  if (rc || ncells == 0) return rc;
  if (!(dt >= 0.0) || !std::isfinite(dt)) return set_error(DF_EINVAL, "df_chem_integrate: dt must be finite and >= 0");
  if ((rc = check_dev("df_chem_integrate", "T", T)) || (rc = check_dev("df_chem_integrate", "p", p)) ||
      (rc = check_dev("df_chem_integrate", "Y", Y)) || (rc = check_dev("df_chem_integrate", "status", status)))
    return rc;
  if (nsub && (rc = check_dev("df_chem_integrate", "nsub", nsub))) return rc;
  df_integ_opts o;
  if (opts) o = *opts;
  else df_integ_opts_default(&o);
  if (!(o.rtol > 0.0) || !(o.atol_Y > 0.0) || !(o.atol_T > 0.0) || !(o.h0 > 0.0) || !(o.h_min >= 0.0) ||
      o.max_substeps < 1 || o.method < 0 || o.method > 1 || o.block_threads < 0 || o.block_threads > 1024 ||
      (o.block_threads % 32) != 0 || o.blocks_per_sm < 0 || o.path < 0 || o.path > 2 ||
      o.reactor < 0 || o.reactor > 1)
    return set_error(DF_EINVAL, "df_chem_integrate: invalid options");
  return launch_integrate(m, ncells, T, p, Y, dt, o, status, nsub, (cudaStream_t)stream);
}

int df_chem_integrate_steps(const df_mech* mc, int64_t ncells, double* T, const double* p, double* Y, double dt,
                            int32_t nsteps, const df_integ_opts* opts, int32_t* status, int32_t* nsub,
                            double* t_ign, df_stream_t stream) {
  df_mech* m = const_cast<df_mech*>(mc);
  const char* fn = "df_chem_integrate_steps";
  int rc = check_cells(fn, m, ncells);
  if (rc || ncells == 0) return rc;
  if (!(dt >= 0.0) || !std::isfinite(dt) || nsteps < 1)
    return set_error(DF_EINVAL, "df_chem_integrate_steps: dt must be finite and >= 0, nsteps >= 1");
  if ((rc = check_dev(fn, "T", T)) || (rc = check_dev(fn, "p", p)) || (rc = check_dev(fn, "Y", Y)) ||
      (rc = check_dev(fn, "status", status)))
    return rc;
  if (nsub && (rc = check_dev(fn, "nsub", nsub))) return rc;
  if (t_ign && (rc = check_dev(fn, "t_ign", t_ign))) return rc;
  df_integ_opts o;
  if (opts) o = *opts;
  else df_integ_opts_default(&o);
  if (!(o.rtol > 0.0) || !(o.atol_Y > 0.0) || !(o.atol_T > 0.0) || !(o.h0 > 0.0) || !(o.h_min >= 0.0) ||
      o.max_substeps < 1 || o.method < 0 || o.method > 1 || o.block_threads < 0 || o.block_threads > 1024 ||
      (o.block_threads % 32) != 0 || o.blocks_per_sm < 0 || o.path < 0 || o.path > 2 ||
      o.reactor < 0 || o.reactor > 1)
    return set_error(DF_EINVAL, "df_chem_integrate_steps: invalid options");
  return launch_integrate_steps(m, ncells, T, p, Y, dt, nsteps, o, status, nsub, t_ign, (cudaStream_t)stream);
}

int df_chem_autotune(df_mech* m, int64_t ncells, const double* T, const double* p, const double* Y, double dt,
                     const df_integ_opts* base, int64_t sample, df_integ_opts* best, float* best_ms,
                     df_stream_t stream) {
  int rc = check_cells("df_chem_autotune", m, ncells);
  if (rc) return rc;
  if (ncells == 0 || sample < 0) return set_error(DF_EINVAL, "df_chem_autotune: no cells to tune on");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return set_error(DF_EINVAL, "df_chem_autotune: dt must be finite and >= 0");
  if ((rc = check_dev("df_chem_autotune", "T", T)) || (rc = check_dev("df_chem_autotune", "p", p)) ||
      (rc = check_dev("df_chem_autotune", "Y", Y)))
    return rc;
  df_integ_opts o;
  if (base) o = *base;
  else df_integ_opts_default(&o);
  if (!(o.rtol > 0.0) || !(o.atol_Y > 0.0) || !(o.atol_T > 0.0) || !(o.h0 > 0.0) || !(o.h_min >= 0.0) ||
      o.max_substeps < 1 || o.method < 0 || o.method > 1 || o.path < 0 || o.path > 2 ||
      o.reactor < 0 || o.reactor > 1)
    return set_error(DF_EINVAL, "df_chem_autotune: invalid options");
  return autotune_integrate(m, ncells, T, p, Y, dt, o, sample, best, best_ms, (cudaStream_t)stream);
}

int df_chem_adjoint_workspace_size(const df_mech* m, int64_t ncells, int32_t max_steps, size_t* bytes) {
  int rc = check_cells("df_chem_adjoint_workspace_size", m, ncells);
  if (rc) return rc;
  if (max_steps < 1 || !bytes) return set_error(DF_EINVAL, "df_chem_adjoint_workspace_size: bad arguments");
  if (!adjoint_workspace_bytes(m, ncells, max_steps, true, bytes))
    return set_error(DF_EWORKSPACE, "df_chem_adjoint_workspace_size: the size does not fit in size_t");
  return DF_OK;
}

int df_chem_adjoint(const df_mech* m, int64_t ncells, const double* T0, const double* p, const double* Y0,
                    double dt, const df_integ_opts* opts, int32_t max_steps, const double* gT1,
                    const double* gY1, const double* gQ1, double* gT0, double* gY0, double* g_lnA,
                    int32_t* status, int32_t* nsub, void* workspace, size_t ws_bytes, df_stream_t stream) {
  const char* fn = "df_chem_adjoint";
  df_integ_opts o;
  int rc = check_adjoint_call(fn, m, ncells, dt, max_steps, T0, p, Y0, gT1, gY1, gQ1, gT0, gY0, g_lnA, status, nsub,
                              opts, &o);
  if (rc || ncells == 0) return rc;
  if (workspace && (rc = check_dev(fn, "workspace", workspace))) return rc;
  return launch_adjoint(m, ncells, T0, p, Y0, dt, o, max_steps, gT1, gY1, gQ1, gT0, gY0, g_lnA, status, nsub,
                        workspace, ws_bytes, true, (cudaStream_t)stream);
}

int df_mech_generated_source(const char* path, char* buf, size_t n, size_t* needed) {
  if (!path) return set_error(DF_EINVAL, "df_mech_generated_source: null path");
  df_mech m;
  int rc = parse_mechanism(path, &m);
  if (rc) return rc;
  const std::string src = jit_thread_source(&m);
  if (needed) *needed = src.size() + 1;
  if (buf && n > 0) {
    const size_t k = std::min(n - 1, src.size());
    memcpy(buf, src.data(), k);
    buf[k] = '\0';
  }
  return DF_OK;
}

int df_chem_jit_info(const df_mech* m, int32_t* used, char* detail, size_t n) {
  if (!m || !used) return set_error(DF_EINVAL, "df_chem_jit_info: null handle or output");
  *used = m->jit_used;
  if (detail && n > 0) {
    const size_t k = std::min(n - 1, m->jit_note.size());
    memcpy(detail, m->jit_note.data(), k);
    detail[k] = '\0';
  }
  return DF_OK;
}

int df_chem_last_stats(const df_mech* m, int64_t* accepted, int64_t* rejected, df_stream_t stream) {
  if (!m) return set_error(DF_EINVAL, "df_chem_last_stats: null handle");
  unsigned long long h[4];
  int rc = cuda_check(cudaMemcpyAsync(h, m->counters, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream),
                      "read counters");
  if (!rc) rc = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "synchronise stream");
  if (rc) return rc;
  if (accepted) *accepted = (int64_t)h[1];
  if (rejected) *rejected = (int64_t)h[2];
  return DF_OK;
}

}  // extern "C"
