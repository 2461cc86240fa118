// Mechanism-specific thread-per-cell integrator, generated and compiled at run
// time.
//
// The mechanism-independent kernel reads each reaction's species indices,
// stoichiometry and type from the mechanism blob and keeps the per-thread
// species vectors (C, wdot, g/RT, h/RT, cp/R) in shared memory, because those
// indices are only known at run time.  For a loaded mechanism the library can
// instead emit the evaluation of f and J as straight-line code with the
// species indices, the reactant / product counts and the reaction types as
// literals (the numbers -- ln A, beta, Ea/R, efficiencies, Troe parameters,
// NASA-7 coefficients -- are still read from the blob, so df_mech_set_lnA keeps
// working), compile it with NVRTC into a module holding the same persistent
// kernel (integrate_thread.cuh) with that evaluation policy, and launch it
// through the driver API.  The species vectors then live in registers, no
// reaction metadata is decoded and no branch depends on the reaction, and the
// shared memory per thread drops to J and the six stage vectors.  The
// operations are the mechanism-independent kernel's, in the same order; the
// two compilations may contract different multiply-adds, so cells agree to
// rounding.
//
// NVRTC is opened at run time (dlopen); the driver entry points come through
// cudaGetDriverEntryPointByVersion.  If either is missing, the headers cannot
// be found, or the compilation fails, the integrator uses the
// mechanism-independent kernel and df_chem_jit_info reports why.
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "integrate_thread.cuh"

namespace df {

namespace {

// ---------------------------------------------------------------------------
// source generation
// ---------------------------------------------------------------------------
RxMeta meta_of(const df_mech* m, int j) {
  RxMeta mt;
  memcpy(&mt, &m->blob_host[m->dims.off_rx + RX_REC * j + 3], 8);
  return mt;
}
RxSlots slots_of(const df_mech* m, int j) {
  RxSlots sl;
  memcpy(&sl, &m->blob_host[m->dims.off_rx + RX_REC * j + 4], 8);
  return sl;
}

// exact decimal-free spelling of a double (C++17 hexadecimal literal)
std::string lit(double v) {
  char b[64];
  snprintf(b, sizeof b, "%a", v);
  return std::string("(") + b + ")";
}

// Horner form c[0] + x (c[1] + x (c[2] + ...)) with the trailing coefficients
// that are exactly zero dropped (for finite x they add exactly zero)
std::string horner(const std::vector<double>& c, const char* x) {
  int top = (int)c.size() - 1;
  while (top > 0 && c[top] == 0.0) --top;
  std::string e = lit(c[top]);
  for (int i = top - 1; i >= 0; --i) e = lit(c[i]) + " + " + x + " * (" + e + ")";
  return e;
}

// f and J of the loaded mechanism as straight-line code: the mechanism-
// independent eval_thread (chem_thread.cuh) at constant pressure with every
// reaction's indices and type resolved and the mechanism's numbers as literals
// (except ln A, read from the blob so that df_mech_set_lnA applies), in the
// same order of operations
void emit_eval(std::ostringstream& o, const df_mech* m) {
  const int N = m->dims.N, n = N + 1, M = m->dims.M;
  o << "template <bool WITH_J, int ST>\n"
    << "__device__ __forceinline__ double gen_eval(const MechView& mv, const double pc, const double (&y)[" << n
    << "], double (&f)[" << n << "], SVT<double, ST> Jv, SVT<double, ST> sM) {\n"
    << "  constexpr int NS = " << N << ";\n  constexpr int n = NS + 1;\n"
    << "  const double T = y[0];\n  const double lnT = fast_log(T);\n  const double invT = 1.0 / T;\n"
    << "  double C[NS], wdot[NS], gRT[NS], hRT[NS], cpW[NS];  // cpW: cp_k / (R W_k)\n"
    << "  double sumYW = 0.0, cpm = 0.0;\n";
  auto sp = [&](int k, int i) { return m->blob_host[m->dims.off_sp + SP_REC * k + i]; };
  for (int k = 0; k < N; ++k) {
    const std::vector<double> a = {sp(k, 2), sp(k, 3), sp(k, 4), sp(k, 5), sp(k, 6)};
    // cp_k / (R W_k) directly: the NASA-7 coefficients times 1 / W_k
    std::vector<double> aw(a);
    for (double& v : aw) v *= sp(k, 1);
    const std::vector<double> ah = {sp(k, SP_H), sp(k, SP_H + 1), sp(k, SP_H + 2), sp(k, SP_H + 3)};
    const std::vector<double> as = {sp(k, SP_S), sp(k, SP_S + 1), sp(k, SP_S + 2)};
    std::vector<double> hs = {sp(k, 2)};
    hs.insert(hs.end(), ah.begin(), ah.end());
    // g/RT = h/RT - s/R in one polynomial: (a1 - a7) - a1 ln T
    // + T (-a2/2 + T (-a3/6 + T (-a4/12 + T (-a5/20)))) + a6 / T
    const std::vector<double> gs = {-0.5 * a[1], -a[2] / 6.0, -a[3] / 12.0, -a[4] / 20.0};
    o << "  {  // species " << k << "\n"
      << "    const double cpw = " << horner(aw, "T") << ";\n    cpW[" << k << "] = cpw;\n"
      << "    const double hk = " << horner(hs, "T") << " + " << lit(sp(k, 7)) << " * invT;\n"
      << "    const double gk = " << lit(sp(k, 2) - sp(k, 8)) << " + " << lit(-sp(k, 2)) << " * lnT + T * ("
      << horner(gs, "T") << ") + " << lit(sp(k, 7)) << " * invT;\n"
      << "    hRT[" << k << "] = hk;\n    gRT[" << k << "] = gk;\n"
      << "    sumYW += y[" << 1 + k << "] * " << lit(sp(k, 1)) << ";\n"
      << "    cpm += y[" << 1 + k << "] * cpw;\n  }\n";
  }
  o << "  cpm = cpm * RU;\n"
    << "  const double rho = pc * invT / (RU * sumYW);\n"
    << "  const double invrho = 1.0 / rho;\n  const double invcp = 1.0 / cpm;\n";
  for (int k = 0; k < N; ++k)
    o << "  C[" << k << "] = rho * y[" << 1 + k << "] * " << lit(sp(k, 1)) << ";\n  wdot[" << k << "] = 0.0;\n";
  // [M] = sum_l eps_l C_l of the third-body and falloff reactions as the sum of
  // all concentrations (once) plus (eps_l - 1) C_l where eps_l is not 1 (exact
  // literals: eps_l - 1 rounds to nothing for eps_l >= 1/2)
  bool any_collider = false;
  for (int j = 0; j < M; ++j) any_collider = any_collider || (meta_of(m, j).flags & 3) != 0;
  if (any_collider) {
    o << "  double ctot = C[0];\n";
    for (int k = 1; k < N; ++k) o << "  ctot += C[" << k << "];\n";
  }
  o
    << "  if (WITH_J) {\n#pragma unroll\n    for (int i = 0; i < n * n; ++i) Jv[i] = 0.0;\n";
  // the unit part of the collider efficiencies, sum over reactions of
  // nu_k d q / d[M], one value per row (sM, the stage vectors' storage, idle
  // while J is built); the conversion below adds it to every column
  if (any_collider) o << "#pragma unroll\n    for (int k = 0; k < NS; ++k) sM[k] = 0.0;\n";
  o << "  }\n"
    << "  const double lnP0RT = LOG_PSTD_RU - lnT;\n";
  for (int j = 0; j < M; ++j) {
    const RxMeta mt = meta_of(m, j);
    const RxSlots sl = slots_of(m, j);
    const int nr = mt.nrnp & 15, np = mt.nrnp >> 4, type = mt.flags & 3;
    const int r[3] = {mt.reac[0], mt.reac[1], mt.reac[2]};
    const int p[3] = {mt.prod[0], mt.prod[1], mt.prod[2]};
    o << "  {  // reaction " << j << "\n"
      << "    RxIn<double> g;\n    const double* r = mv.rx + RX_REC * " << j << ";\n"
      << "    g.lnA = r[0];\n    g.beta = " << lit(m->blob_host[m->dims.off_rx + RX_REC * j + 1])
      << ";\n    g.EaR = " << lit(m->blob_host[m->dims.off_rx + RX_REC * j + 2]) << ";\n";
    for (int i = 0; i < 3; ++i) o << "    g.mt.reac[" << i << "] = " << r[i] << ";\n";
    for (int i = 0; i < 3; ++i) o << "    g.mt.prod[" << i << "] = " << p[i] << ";\n";
    o << "    g.mt.nrnp = " << (int)mt.nrnp << ";\n    g.mt.flags = " << (int)mt.flags << ";\n"
      << "    g.sl.eff = " << sl.eff << ";\n    g.sl.troe = " << sl.troe << ";\n";
    for (int i = 0; i < 3; ++i)
      o << "    g.cr[" << i << "] = " << (i < nr ? "C[" + std::to_string(r[i]) + "]" : std::string("1.0")) << ";\n";
    for (int i = 0; i < 3; ++i)
      o << "    g.cp[" << i << "] = " << (i < np ? "C[" + std::to_string(p[i]) + "]" : std::string("1.0")) << ";\n";
    // sum nu g/RT and h/RT in rate_gather's order
    o << "    double sg = gRT[" << p[0] << "] - gRT[" << r[0] << "];\n"
      << "    double sh = 0.0;\n    if (WITH_J) sh = hRT[" << p[0] << "] - hRT[" << r[0] << "];\n";
    for (int i = 1; i < np; ++i) o << "    sg += gRT[" << p[i] << "];\n    if (WITH_J) sh += hRT[" << p[i] << "];\n";
    for (int i = 1; i < nr; ++i) o << "    sg -= gRT[" << r[i] << "];\n    if (WITH_J) sh -= hRT[" << r[i] << "];\n";
    o << "    g.sg = sg;\n    g.sh = sh;\n";
    auto eff = [&](int l) { return m->blob_host[m->dims.off_eff + N * sl.eff + l]; };
    if (type != 0) {
      o << "    {\n      double Mc = ctot;\n";
      for (int l = 0; l < N; ++l)
        if (eff(l) != 1.0) o << "      Mc += " << lit(eff(l) - 1.0) << " * C[" << l << "];\n";
      o << "      g.Mc = Mc;\n    }\n";
    } else {
      o << "    g.Mc = 0.0;\n";
    }
    if (type == 2) {  // the falloff parameters as literals too (a one-record table)
      const double* tr = &m->blob_host[m->dims.off_tr + TR_REC * sl.troe];
      o << "    const double trp[" << TR_REC << "] = {";
      for (int i = 0; i < TR_REC; ++i) o << (i ? ", " : "") << lit(tr[i]);
      o << "};\n    MechView mvt = mv;\n    mvt.tr = trp;\n    g.sl.troe = 0;\n"
        << "    RateOutT<double> ro;\n    rate_compute<NS, WITH_J>(mvt, g, T, lnT, invT, lnP0RT, ro);\n";
    } else {
      o << "    RateOutT<double> ro;\n    rate_compute<NS, WITH_J>(mv, g, T, lnT, invT, lnP0RT, ro);\n";
    }
    // The species of the reaction with their net stoichiometric coefficient
    // nu_k (products minus reactants): one update of wdot and of each Jacobian
    // row per species, scaled by nu_k, instead of one per reactant or product
    // entry (a species entered twice, or on both sides, is touched once or not
    // at all).  The columns d q / d C_l likewise sum the entries of species l.
    std::vector<int> spc;
    std::vector<int> nu(N, 0);
    for (int i = 0; i < nr; ++i) nu[r[i]] -= 1;
    for (int i = 0; i < np; ++i) nu[p[i]] += 1;
    for (int i = 0; i < nr; ++i)
      if (std::find(spc.begin(), spc.end(), r[i]) == spc.end()) spc.push_back(r[i]);
    for (int i = 0; i < np; ++i)
      if (std::find(spc.begin(), spc.end(), p[i]) == spc.end()) spc.push_back(p[i]);
    auto nu_times = [](int v, const std::string& x) {
      return v == 1 ? "(" + x + ")" : v == -1 ? "-(" + x + ")" : std::to_string(v) + ".0 * (" + x + ")";
    };
    o << "    if (ro.active) {\n      const double q = ro.q;\n";
    for (int k : spc)
      if (nu[k] != 0) o << "      wdot[" << k << "] += " << nu_times(nu[k], "q") << ";\n";
    o << "      if (WITH_J) {\n"
      << "        const double dr0 = ro.fk * ro.cr[1] * ro.cr[2];\n"
      << "        const double dr1 = ro.fk * ro.cr[0] * ro.cr[2];\n"
      << "        const double dr2 = ro.fk * ro.cr[0] * ro.cr[1];\n"
      << "        const double dp0 = -(ro.rk * ro.cp[1] * ro.cp[2]);\n"
      << "        const double dp1 = -(ro.rk * ro.cp[0] * ro.cp[2]);\n"
      << "        const double dp2 = -(ro.rk * ro.cp[0] * ro.cp[1]);\n"
      << "        (void)dr1; (void)dr2; (void)dp1; (void)dp2;\n";
    // d q / d C_l of each species of the reaction
    for (int l : spc) {
      std::string terms;
      for (int i = 0; i < nr; ++i)
        if (r[i] == l) terms += (terms.empty() ? "" : " + ") + std::string("dr") + std::to_string(i);
      for (int i = 0; i < np; ++i)
        if (p[i] == l) terms += (terms.empty() ? "" : " + ") + std::string("dp") + std::to_string(i);
      o << "        const double dq" << l << " = " << terms << ";\n";
    }
    // the concentration-space entries d wdot_k / d C_l enter row k scaled by
    // W_k / W_l (a literal), the column scaling of the conversion to mass
    // fractions below, so that the conversion adds only its rank-one part
    auto wk_over_wl = [&](int k, int l) { return sp(k, 0) * sp(l, 1); };  // W_k * (1 / W_l)
    for (int k : spc) {
      if (nu[k] == 0) continue;
      const int row = 1 + k;
      o << "        Jv[" << row * n << "] += " << nu_times(nu[k], "ro.dqdT") << ";\n";
      for (int l : spc) {
        if (l == k)
          o << "        Jv[" << row * n + 1 + l << "] += " << nu_times(nu[k], "dq" + std::to_string(l)) << ";\n";
        else
          o << "        Jv[" << row * n + 1 + l << "] += " << lit(nu[k] * wk_over_wl(k, l)) << " * dq" << l << ";\n";
      }
      if (type != 0) {
        o << "        {\n          const double cM = " << nu_times(nu[k], "ro.dqdM") << ";\n"
          << "          sM[" << k << "] += cM;\n";
        for (int l = 0; l < N; ++l) {
          if (eff(l) == 1.0) continue;
          const double c = l == k ? eff(l) - 1.0 : (eff(l) - 1.0) * wk_over_wl(k, l);
          o << "          Jv[" << row * n + 1 + l << "] += cM * " << lit(c) << ";\n";
        }
        o << "        }\n";
      }
    }
    o << "      }\n    }\n  }\n";
  }
  o << "  double Hw = 0.0;\n#pragma unroll\n  for (int k = 0; k < NS; ++k) Hw += hRT[k] * wdot[k];\n"
    << "  Hw = Hw * (RU * T);\n"
    ;
  for (int k = 0; k < N; ++k) o << "  f[" << 1 + k << "] = " << lit(sp(k, 0)) << " * wdot[" << k << "] * invrho;\n";
  o
    << "  f[0] = -(Hw * invrho * invcp);\n"
    << "  if (WITH_J) {\n"
    << "    const double Wbar = 1.0 / sumYW;\n"
    // row k holds S'_kl = (W_k / W_l) dwdot_k/dC_l; with s_k = sum_l S_kl C_l =
    // (1 / W_k) sum_l S'_kl rho Y_l and a_k = W_k Wbar (wdot_k - s_k) / rho:
    // dY_k/dY_l = S'_kl + a_k / W_l
    << "    double rY[NS];\n#pragma unroll\n    for (int l = 0; l < NS; ++l) rY[l] = rho * y[1 + l];\n"
    << "#pragma unroll 1\n"
    << "    for (int k = 0; k < NS; ++k) {\n"
    << "      const int row = (1 + k) * n;\n      const double Wk = mv.sp[SP_REC * k];\n"
    << "      double s = 0.0;\n#pragma unroll\n      for (int l = 0; l < NS; ++l) s += Jv[row + 1 + l] * rY[l];\n"
    << "      s = s * mv.sp[SP_REC * k + 1];\n"
    << (any_collider ? "      const double sMk = sM[k];\n      s = fma(sMk, ctot, s);\n" : "")
    << "      const double wk = wdot[k];\n      double a = Wk * Wbar * invrho * (wk - s);\n"
    << (any_collider ? "      a = fma(Wk, sMk, a);\n" : "")
    << "#pragma unroll\n      for (int i = 0; i < NS; ++i) Jv[row + 1 + i] = fma(a, mv.sp[SP_REC * i + 1], Jv[row + 1 + i]);\n"
    << "      Jv[row] = Wk * invrho * (Jv[row] + (wk - s) * invT);\n    }\n"
    << "    double dcp = 0.0, cpf = 0.0;\n";
  for (int k = 0; k < N; ++k) {
    const std::vector<double> d = {sp(k, 3), 2.0 * sp(k, 4), 3.0 * sp(k, 5), 4.0 * sp(k, 6)};
    o << "    dcp += y[" << 1 + k << "] * (" << horner(d, "T") << ") * " << lit(sp(k, 1)) << ";\n"
      << "    cpf += cpW[" << k << "] * f[" << 1 + k << "];\n";
  }
  o
    << "    dcp = dcp * RU;\n    cpf = cpf * RU;\n"
    // the temperature row's species weights (h_k/RT) / W_k, once
    << "    double hw[NS];\n";
  for (int k = 0; k < N; ++k) o << "    hw[" << k << "] = hRT[" << k << "] * " << lit(sp(k, 1)) << ";\n";
  o
    << "#pragma unroll 1\n    for (int jc = 0; jc < n; ++jc) {\n      double acc = 0.0;\n"
    << "#pragma unroll\n      for (int k = 0; k < NS; ++k) acc += hw[k] * Jv[(1 + k) * n + jc];\n"
    << "      acc = acc * (RU * T);\n"
    << "      if (jc == 0) {\n        Jv[0] = -(invcp * (acc + cpf)) - f[0] * dcp * invcp;\n      } else {\n"
    << "        const double cpj = RU * cpW[jc - 1];\n"
    << "        Jv[jc] = -(invcp * acc) - f[0] * cpj * invcp;\n      }\n    }\n  }\n"
    << "  return -Hw;\n}\n\n";
}

}  // namespace

std::string jit_thread_source(const df_mech* m) {
  std::ostringstream o;
  o << "// generated for a " << m->dims.N << "-species / " << m->dims.M << "-reaction mechanism\n"
    << "#include \"integrate_thread.cuh\"\n\nnamespace df {\n\n";
  emit_eval(o, m);
  o << "struct GenEval {\n"
    << "  static constexpr bool kSpeciesVectors = false;\n"
    << "  template <int NS, bool WITH_J, bool CONSTV, int ST>\n"
    << "  __device__ __forceinline__ static double run(const MechView& mv, double pc, const double (&y)[NS + 1],\n"
    << "                                               double (&f)[NS + 1], SVT<double, ST> scratch, SVT<double, ST>,\n"
    << "                                               SVT<double, ST>, SVT<double, ST>, SVT<double, ST>,\n"
    << "                                               SVT<double, ST> Jv) {\n"
    << "    static_assert(!CONSTV, \"generated evaluation: constant pressure\");\n"
    << "    return gen_eval<WITH_J, ST>(mv, pc, y, f, Jv, scratch);\n  }\n};\n\n}  // namespace df\n";
  return o.str();
}

std::string jit_kernel_name(int N, int threads, bool ign = false) {
  return "df::k_integrate_thread<" + std::to_string(N) + ", false, " + std::to_string(threads) + ", df::GenEval" +
         (ign ? ", true>" : ">");
}

namespace {

// ---------------------------------------------------------------------------
// NVRTC (opened at run time) and the driver entry points
// ---------------------------------------------------------------------------
typedef int (*nvrtcCreateProgram_t)(void**, const char*, const char*, int, const char* const*, const char* const*);
typedef int (*nvrtcCompileProgram_t)(void*, int, const char* const*);
typedef int (*nvrtcGetSize_t)(void*, size_t*);
typedef int (*nvrtcGetBuf_t)(void*, char*);
typedef int (*nvrtcDestroyProgram_t)(void**);
typedef int (*nvrtcAddNameExpression_t)(void*, const char*);
typedef int (*nvrtcGetLoweredName_t)(void*, const char*, const char**);
typedef int (*nvrtcVersion_t)(int*, int*);

struct Nvrtc {
  bool ok = false;
  std::string why;
  nvrtcCreateProgram_t create = nullptr;
  nvrtcCompileProgram_t compile = nullptr;
  nvrtcGetSize_t log_size = nullptr, cubin_size = nullptr;
  nvrtcGetBuf_t log = nullptr, cubin = nullptr;
  nvrtcDestroyProgram_t destroy = nullptr;
  nvrtcAddNameExpression_t add_name = nullptr;
  nvrtcGetLoweredName_t lowered = nullptr;
  int version = 0;  // major * 1000 + minor
};

const Nvrtc& nvrtc() {
  static Nvrtc r;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
      r.why = "NVRTC library not found";
      return;
    }
    r.create = (nvrtcCreateProgram_t)dlsym(h, "nvrtcCreateProgram");
    r.compile = (nvrtcCompileProgram_t)dlsym(h, "nvrtcCompileProgram");
    r.log_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetProgramLogSize");
    r.log = (nvrtcGetBuf_t)dlsym(h, "nvrtcGetProgramLog");
    r.cubin_size = (nvrtcGetSize_t)dlsym(h, "nvrtcGetCUBINSize");
    r.cubin = (nvrtcGetBuf_t)dlsym(h, "nvrtcGetCUBIN");
    r.destroy = (nvrtcDestroyProgram_t)dlsym(h, "nvrtcDestroyProgram");
    r.add_name = (nvrtcAddNameExpression_t)dlsym(h, "nvrtcAddNameExpression");
    r.lowered = (nvrtcGetLoweredName_t)dlsym(h, "nvrtcGetLoweredName");
    r.ok = r.create && r.compile && r.log_size && r.log && r.cubin_size && r.cubin && r.destroy && r.add_name &&
           r.lowered;
    if (auto ver = (nvrtcVersion_t)dlsym(h, "nvrtcVersion")) {
      int ma = 0, mi = 0;
      if (ver(&ma, &mi) == 0) r.version = ma * 1000 + mi;
    }
    if (!r.ok) r.why = "NVRTC library lacks an entry point";
  });
  return r;
}

typedef CUresult (*cuModuleLoadData_t)(CUmodule*, const void*);
typedef CUresult (*cuModuleGetFunction_t)(CUfunction*, CUmodule, const char*);
typedef CUresult (*cuModuleGetGlobal_t)(CUdeviceptr*, size_t*, CUmodule, const char*);
typedef CUresult (*cuLaunchKernel_t)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                                     unsigned, CUstream, void**, void**);
typedef CUresult (*cuFuncSetAttribute_t)(CUfunction, CUfunction_attribute, int);
typedef CUresult (*cuOccupancy_t)(int*, CUfunction, int, size_t);
typedef CUresult (*cuModuleUnload_t)(CUmodule);

struct Driver {
  bool ok = false;
  cuModuleLoadData_t load = nullptr;
  cuModuleUnload_t unload = nullptr;
  cuModuleGetFunction_t get_function = nullptr;
  cuModuleGetGlobal_t get_global = nullptr;
  cuLaunchKernel_t launch = nullptr;
  cuFuncSetAttribute_t set_attr = nullptr;
  cuOccupancy_t occupancy = nullptr;
};

void* entry(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return p;
}

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    d.load = (cuModuleLoadData_t)entry("cuModuleLoadData");
    d.unload = (cuModuleUnload_t)entry("cuModuleUnload");
    d.get_function = (cuModuleGetFunction_t)entry("cuModuleGetFunction");
    d.get_global = (cuModuleGetGlobal_t)entry("cuModuleGetGlobal");
    d.launch = (cuLaunchKernel_t)entry("cuLaunchKernel");
    d.set_attr = (cuFuncSetAttribute_t)entry("cuFuncSetAttribute");
    d.occupancy = (cuOccupancy_t)entry("cuOccupancyMaxActiveBlocksPerMultiprocessor");
    d.ok = d.load && d.unload && d.get_function && d.get_global && d.launch && d.set_attr && d.occupancy;
  });
  return d;
}

// directory of the library's device headers: next to the shared library
// (<package>/_build/lib*.so -> <package>/csrc)
std::string header_dir() {
  Dl_info info;
  if (!dladdr((void*)&header_dir, &info) || !info.dli_fname) return "";
  std::string so = info.dli_fname;
  const size_t cut = so.find_last_of('/');
  if (cut == std::string::npos) return "";
  std::string dir = so.substr(0, cut);
  const size_t up = dir.find_last_of('/');
  if (up == std::string::npos) return "";
  std::string cs = dir.substr(0, up) + "/csrc";
  std::string probe = cs + "/integrate_thread.cuh";
  if (FILE* f = fopen(probe.c_str(), "r")) {
    fclose(f);
    return cs;
  }
  return "";
}

// one compiled module per (device, generated source)
struct Module {
  bool ok = false;
  std::string why;
  CUmodule mod = nullptr;
  std::map<int, CUfunction> fn;  // threads per block -> kernel
  CUfunction fn_ign = nullptr;    // 32 threads, refining the ignition time (IntegArgs.t_ign)
  size_t compile_ms = 0;
  bool from_cache = false;
};

std::mutex g_mu;
std::map<std::pair<int, std::string>, Module> g_modules;

constexpr int kThreads[] = {32, 64};
constexpr int kIgnThreads = 32;  // the block size of the kernel that refines the ignition time
// the generated kernels' exp table: 256 entries (one FP64 operation fewer per
// exponential than the library's 64; 4 KB of shared memory per block)
constexpr int kGenExpTableBits = 8;

// ---------------------------------------------------------------------------
// on-disk cache of compiled modules: <dir>/<key>.cubin and <key>.names (the
// lowered names of the kernels and of the table), key = FNV-1a hash of the
// generated source, the device headers it includes, the target architecture
// and the NVRTC version.  Directory: $DF_JIT_CACHE ("0" disables), else
// $XDG_CACHE_HOME/df_chem_jit, else $HOME/.cache/df_chem_jit.
// ---------------------------------------------------------------------------
uint64_t fnv1a(const std::string& s, uint64_t h = 1469598103934665603ull) {
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

bool read_file(const std::string& path, std::string* out) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  std::string d;
  char buf[65536];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) d.append(buf, k);
  const bool ok = !ferror(f);
  fclose(f);
  if (ok) *out = std::move(d);
  return ok;
}

bool write_file_atomic(const std::string& path, const std::string& data) {
  const std::string tmp = path + ".tmp" + std::to_string((unsigned long long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
  if (fclose(f) != 0 || !ok) {
    remove(tmp.c_str());
    return false;
  }
  return rename(tmp.c_str(), path.c_str()) == 0;
}

std::string cache_dir() {
  const char* e = getenv("DF_JIT_CACHE");
  std::string d;
  if (e) {
    if (!*e || std::string(e) == "0") return "";
    d = e;
  } else if (const char* x = getenv("XDG_CACHE_HOME")) {
    d = std::string(x) + "/df_chem_jit";
  } else if (const char* hm = getenv("HOME")) {
    d = std::string(hm) + "/.cache/df_chem_jit";
  } else {
    return "";
  }
  // create the directory and its parents
  for (size_t pos = 1; pos <= d.size(); ++pos)
    if (pos == d.size() || d[pos] == '/') mkdir(d.substr(0, pos).c_str(), 0755);
  return d;
}

// the device headers' contents, hashed once per process
uint64_t headers_hash(const std::string& inc) {
  static uint64_t h = 0;
  static std::once_flag once;
  std::call_once(once, [&] {
    uint64_t acc = 1469598103934665603ull;
    const char* files[] = {"integrate_thread.cuh", "rosenbrock.cuh", "chem_thread.cuh", "dev_common.cuh",
                           "fastexp.cuh", "fastexp_table256.inc", "fastlog.cuh", "fastlog_table.inc", "dual.cuh"};
    for (const char* fn : files) {
      std::string d;
      read_file(inc + "/" + fn, &d);
      acc = fnv1a(std::string(fn) + d, acc);
    }
    h = acc;
  });
  return h;
}

// resolve the kernels and the table of a loaded cubin, upload the tables
bool finish_module(Module& r, const Driver& drv, const std::vector<char>& cubin,
                   const std::vector<std::string>& lowered) {
  if (drv.load(&r.mod, cubin.data()) != CUDA_SUCCESS) {
    r.why = "cuModuleLoadData failed";
    r.mod = nullptr;
    return false;
  }
  for (size_t i = 0; i < sizeof(kThreads) / sizeof(kThreads[0]); ++i) {
    CUfunction f = nullptr;
    if (i >= lowered.size() || lowered[i].empty() || drv.get_function(&f, r.mod, lowered[i].c_str()) != CUDA_SUCCESS) {
      r.why = "generated kernel not found in the module";
      drv.unload(r.mod);
      r.mod = nullptr;
      return false;
    }
    r.fn[kThreads[i]] = f;
  }
  {
    const size_t i = sizeof(kThreads) / sizeof(kThreads[0]);
    if (i >= lowered.size() || lowered[i].empty() ||
        drv.get_function(&r.fn_ign, r.mod, lowered[i].c_str()) != CUDA_SUCCESS) {
      r.why = "generated kernel (ignition time) not found in the module";
      drv.unload(r.mod);
      r.mod = nullptr;
      return false;
    }
  }
  CUdeviceptr tab = 0;
  size_t tab_bytes = 0;
  if (lowered.back().empty() || drv.get_global(&tab, &tab_bytes, r.mod, lowered.back().c_str()) != CUDA_SUCCESS ||
      tab_bytes != 2 * sizeof(RosTab)) {
    r.why = "Rosenbrock table not found in the module";
    drv.unload(r.mod);
    r.mod = nullptr;
    return false;
  }
  RosTab t[2] = {make_rodas4(), make_rodas3()};
  if (!t[0].stiff_acc || !t[1].stiff_acc) {  // ros_attempt relies on it
    r.why = "Rosenbrock table not stiffly accurate";
    drv.unload(r.mod);
    r.mod = nullptr;
    return false;
  }
  if (cudaMemcpy((void*)tab, t, sizeof(t), cudaMemcpyHostToDevice) != cudaSuccess) {
    r.why = "upload of the Rosenbrock tables failed";
    drv.unload(r.mod);
    r.mod = nullptr;
    return false;
  }
  r.ok = true;
  return true;
}

// Version of the cached entries (the cubin and its lowered-name list, and what
// finish_module expects of them); raised whenever either changes.
constexpr int kCacheFormat = 3;

Module build_module(int dev, const df_mech* m, const std::string& src) {
  Module r;
  const Driver& drv = driver();
  if (!drv.ok) {
    r.why = "driver entry points for module loading unavailable";
    return r;
  }
  const std::string inc = header_dir();
  if (inc.empty()) {
    r.why = "device headers (csrc) not found next to the library";
    return r;
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    r.why = "device attributes unavailable";
    return r;
  }
  const Nvrtc& nv = nvrtc();
  const std::string arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor) + "a";
  std::vector<std::string> names;
  for (int t : kThreads) names.push_back(jit_kernel_name(m->dims.N, t));
  names.push_back(jit_kernel_name(m->dims.N, kIgnThreads, true));
  names.push_back("&df::c_tab");
  const std::string incopt = "-I" + inc;
  const std::string expopt = "-DDF_EXP_TABLE_BITS=" + std::to_string(kGenExpTableBits);
  const char* opts[] = {arch.c_str(), "-std=c++17", incopt.c_str(), "-default-device", "-lineinfo",
                        "-diag-suppress=177", expopt.c_str()};
  // the on-disk cache: keyed by the generated source, the device headers, the
  // architecture, the NVRTC version, the compile options (the include path
  // left out: a moved tree keeps its entries) and the entry format
  const std::string dir = cache_dir();
  std::string keysrc = src + arch + std::to_string(nv.version) + "|format " + std::to_string(kCacheFormat);
  for (const char* o : opts)
    if (o != incopt.c_str()) keysrc += std::string("|") + o;
  char key[32] = {0};
  snprintf(key, sizeof key, "%016llx", (unsigned long long)fnv1a(keysrc, headers_hash(inc)));
  const std::string base = dir.empty() ? std::string() : dir + "/" + key;
  if (!base.empty()) {
    std::string bin, nm;
    if (read_file(base + ".cubin", &bin) && read_file(base + ".names", &nm) && !bin.empty()) {
      std::vector<std::string> lowered;
      std::istringstream in(nm);
      for (std::string line; std::getline(in, line);) lowered.push_back(line);
      if (lowered.size() == names.size()) {
        std::vector<char> cubin(bin.begin(), bin.end());
        if (finish_module(r, drv, cubin, lowered)) {
          r.from_cache = true;
          return r;
        }
        r = Module();  // unusable entry: compile afresh
      }
    }
  }
  if (!nv.ok) {
    r.why = nv.why;
    return r;
  }
  void* prog = nullptr;
  if (nv.create(&prog, src.c_str(), "df_generated.cu", 0, nullptr, nullptr) != 0) {
    r.why = "nvrtcCreateProgram failed";
    return r;
  }
  for (auto& s : names) nv.add_name(prog, s.c_str());
  const auto t0 = std::chrono::steady_clock::now();
  const int rc = nv.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
  r.compile_ms = (size_t)std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0)
                     .count();
  if (rc != 0) {
    size_t n = 0;
    nv.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) nv.log(prog, &log[0]);
    r.why = "NVRTC compilation failed: " + log.substr(0, 2000);
    nv.destroy(&prog);
    return r;
  }
  size_t nb = 0;
  nv.cubin_size(prog, &nb);
  std::vector<char> cubin(nb);
  nv.cubin(prog, cubin.data());
  std::vector<std::string> lowered;
  for (auto& s : names) {
    const char* l = nullptr;
    nv.lowered(prog, s.c_str(), &l);
    lowered.push_back(l ? std::string(l) : std::string());
  }
  nv.destroy(&prog);
  if (!finish_module(r, drv, cubin, lowered)) return r;
  if (!base.empty()) {  // best effort: a failed write only costs the next process a compile
    std::string nm;
    for (auto& l : lowered) nm += l + "\n";
    if (write_file_atomic(base + ".cubin", std::string(cubin.begin(), cubin.end())))
      write_file_atomic(base + ".names", nm);
  }
  return r;
}

}  // namespace

int jit_thread_launch(df_mech* m, int threads, int bps, const IntegArgs& a, cudaStream_t st, bool* launched) {
  *launched = false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DF_OK;
  Module* md = static_cast<Module*>(m->jit_module[dev]);
  if (!md) {  // first launch on this device: generate, and compile unless cached
    const std::string src = jit_thread_source(m);
    std::lock_guard<std::mutex> lock(g_mu);
    auto key = std::make_pair(dev, src);
    auto it = g_modules.find(key);
    if (it == g_modules.end()) it = g_modules.emplace(key, build_module(dev, m, src)).first;
    md = &it->second;
    m->jit_module[dev] = md;
    m->jit_note = !md->ok          ? md->why
                  : md->from_cache ? std::string("generated kernel loaded from the on-disk cache")
                                   : "generated kernel compiled in " + std::to_string(md->compile_ms) + " ms";
  }
  if (!md->ok) return DF_OK;
  CUfunction fk = nullptr;
  if (a.t_ign) {  // the variant that refines the ignition time, in its block size
    fk = md->fn_ign;
    threads = kIgnThreads;
  } else {
    auto f = md->fn.find(threads);
    if (f == md->fn.end()) return DF_OK;  // no generated kernel for this block size
    fk = f->second;
  }
  const Driver& drv = driver();
  const int N = m->dims.N;
  const int per_thread = (N + 1) * (N + 1) + 6 * (N + 1);  // J and the stage vectors
  IntegArgs args = a;
  // the exp table (2 doubles per entry), the mechanism if staging it leaves as
  // many blocks on an SM as reading it through L1, the per-thread workspace
  const size_t tab = 2 * ((size_t)1 << kGenExpTableBits);
  const size_t sm_staged = sizeof(double) * (tab + (size_t)blob_smem_doubles(m->dims) + (size_t)per_thread * threads);
  const size_t sm_plain = sizeof(double) * (tab + (size_t)per_thread * threads);
  auto blocks_per_sm = [m](size_t b) {
    return b > m->max_smem_optin ? (size_t)0 : m->smem_per_sm / (b + m->smem_reserved_per_block);
  };
  args.stage_blob = blocks_per_sm(sm_staged) >= blocks_per_sm(sm_plain) ? 1 : 0;
  const size_t sm = args.stage_blob ? sm_staged : sm_plain;
  if (sm > m->max_smem_optin) return DF_OK;
  if (drv.set_attr(fk, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)sm) != CUDA_SUCCESS)
    return set_error(DF_ECUDA, "generated integrator: shared-memory attribute");
  int occ = 0;
  if (drv.occupancy(&occ, fk, threads, sm) != CUDA_SUCCESS || occ < 1)
    return set_error(DF_ECUDA, "generated integrator: occupancy query");
  const int per_sm = bps > 0 ? std::min(bps, occ) : occ;
  int64_t blocks = (int64_t)m->num_sms * per_sm;
  const int64_t need = (args.nwork + threads - 1) / threads;
  if (blocks > need) blocks = std::max<int64_t>(1, need);
  int rc = cuda_check(cudaMemsetAsync(m->counters, 0, 4 * sizeof(unsigned long long), st), "reset work counter");
  if (rc) return rc;
  void* params[] = {&args};
  if (drv.launch(fk, (unsigned)blocks, 1, 1, (unsigned)threads, 1, 1, (unsigned)sm, (CUstream)st, params,
                 nullptr) != CUDA_SUCCESS)
    return set_error(DF_ECUDA, "generated integrator launch");
  *launched = true;
  m->jit_used = 1;
  return DF_OK;
}

}  // namespace df
