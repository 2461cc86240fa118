// Mechanism file -> blob.  A small JSON reader (objects, arrays, numbers,
// strings, true/false/null) and the packing of species and reactions into the
// fixed-size records of common.cuh.
//
// The mechanism describes the reaction system of Sec. 2.3 eq. (reaction):
// N species and M reversible reactions with molar stoichiometric coefficients
// nu'_{aj} (reactants) and nu''_{aj} (products); K_f by the Arrhenius law,
// optional third-body efficiencies and Troe falloff, and NASA-7 thermo from
// which the equilibrium constant K_c = K_f / K_r follows.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>

#include "common.cuh"

namespace df {
namespace {

struct JVal {
  enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
  bool b = false;
  double num = 0.0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;  // keeps file order

  const JVal* get(const std::string& k) const {
    for (auto& kv : obj)
      if (kv.first == k) return &kv.second;
    return nullptr;
  }
};

struct JParser {
  const char* s;
  const char* e;
  std::string err;

  void ws() {
    while (s < e && (*s == ' ' || *s == '\n' || *s == '\r' || *s == '\t')) ++s;
  }
  bool fail(const char* what) {
    if (err.empty()) err = what;
    return false;
  }
  bool parse(JVal& v, int depth = 0) {
    if (depth > 64) return fail("nesting too deep");
    ws();
    if (s >= e) return fail("unexpected end");
    char c = *s;
    if (c == '{') {
      ++s;
      v.kind = JVal::OBJ;
      ws();
      if (s < e && *s == '}') { ++s; return true; }
      while (true) {
        ws();
        JVal key;
        if (s >= e || *s != '"' || !parse_str(key.str)) return fail("expected key");
        ws();
        if (s >= e || *s != ':') return fail("expected ':'");
        ++s;
        JVal val;
        if (!parse(val, depth + 1)) return false;
        v.obj.emplace_back(key.str, std::move(val));
        ws();
        if (s < e && *s == ',') { ++s; continue; }
        if (s < e && *s == '}') { ++s; return true; }
        return fail("expected ',' or '}'");
      }
    }
    if (c == '[') {
      ++s;
      v.kind = JVal::ARR;
      ws();
      if (s < e && *s == ']') { ++s; return true; }
      while (true) {
        JVal val;
        if (!parse(val, depth + 1)) return false;
        v.arr.push_back(std::move(val));
        ws();
        if (s < e && *s == ',') { ++s; continue; }
        if (s < e && *s == ']') { ++s; return true; }
        return fail("expected ',' or ']'");
      }
    }
    if (c == '"') {
      v.kind = JVal::STR;
      return parse_str(v.str);
    }
    if (e - s >= 4 && !strncmp(s, "true", 4)) { s += 4; v.kind = JVal::BOOL; v.b = true; return true; }
    if (e - s >= 5 && !strncmp(s, "false", 5)) { s += 5; v.kind = JVal::BOOL; v.b = false; return true; }
    if (e - s >= 4 && !strncmp(s, "null", 4)) { s += 4; v.kind = JVal::NUL; return true; }
    // number
    char buf[64];
    int n = 0;
    while (s < e && n < 63 && (isdigit((unsigned char)*s) || *s == '-' || *s == '+' || *s == '.' ||
                               *s == 'e' || *s == 'E' || *s == 'I' || *s == 'n' || *s == 'f' ||
                               *s == 'i' || *s == 't' || *s == 'y' || *s == 'N' || *s == 'a'))
      buf[n++] = *s++;
    buf[n] = 0;
    if (n == 0) return fail("unexpected character");
    char* endp = nullptr;
    v.num = strtod(buf, &endp);
    if (endp != buf + n) return fail("bad number");
    v.kind = JVal::NUM;
    return true;
  }
  bool parse_str(std::string& out) {
    ++s;  // opening quote
    while (s < e && *s != '"') {
      if (*s == '\\') {
        ++s;
        if (s >= e) return fail("bad escape");
        char c = *s;
        if (c == 'n') out += '\n';
        else if (c == 't') out += '\t';
        else if (c == 'u') {
          if (e - s < 5) return fail("bad escape");
          out += '?';
          s += 4;
        } else out += c;
        ++s;
      } else {
        out += *s++;
      }
    }
    if (s >= e) return fail("unterminated string");
    ++s;
    return true;
  }
};

bool num_of(const JVal* v, double* out) {
  if (!v || v->kind != JVal::NUM) return false;
  *out = v->num;
  return true;
}

}  // namespace

int parse_mechanism(const char* path, df_mech* m) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return set_error(DF_EMECH, std::string("cannot open mechanism file ") + path);
  std::stringstream ss;
  ss << f.rdbuf();
  std::string txt = ss.str();
  JParser P{txt.data(), txt.data() + txt.size(), ""};
  JVal root;
  if (!P.parse(root) || root.kind != JVal::OBJ)
    return set_error(DF_EMECH, "mechanism JSON parse error: " + (P.err.empty() ? "not an object" : P.err));
  const JVal* sp = root.get("species");
  const JVal* rx = root.get("reactions");
  if (!sp || sp->kind != JVal::ARR || !rx || rx->kind != JVal::ARR)
    return set_error(DF_EMECH, "mechanism needs 'species' and 'reactions' arrays");
  const int N = (int)sp->arr.size();
  const int M = (int)rx->arr.size();
  if (N < 1 || N > MAX_SPECIES)
    return set_error(DF_EMECH, "species count must be in [1, 64], got " + std::to_string(N));
  if (M > MAX_REACTIONS)
    return set_error(DF_EMECH, "more than 4096 reactions");
  std::map<std::string, int> index;
  std::vector<double> spec(SP_REC * N);
  for (int k = 0; k < N; ++k) {
    const JVal& s = sp->arr[k];
    const JVal* name = s.get("name");
    const JVal* W = s.get("W");
    const JVal* nasa = s.get("nasa7");
    if (!name || name->kind != JVal::STR || !W || W->kind != JVal::NUM || !nasa ||
        nasa->kind != JVal::ARR || nasa->arr.size() != 7)
      return set_error(DF_EMECH, "species " + std::to_string(k) + ": needs name, W, nasa7[7]");
    if (index.count(name->str)) return set_error(DF_EMECH, "duplicate species " + name->str);
    index[name->str] = k;
    if (!(W->num > 0.0)) return set_error(DF_EMECH, "species " + name->str + ": W must be > 0");
    spec[SP_REC * k + 0] = W->num;
    spec[SP_REC * k + 1] = 1.0 / W->num;
    for (int i = 0; i < 7; ++i) {
      if (!num_of(&nasa->arr[i], &spec[SP_REC * k + 2 + i]))
        return set_error(DF_EMECH, "species " + name->str + ": nasa7 must hold numbers");
    }
    const double* a = &spec[SP_REC * k + 2];
    for (int i = 0; i < 4; ++i) spec[SP_REC * k + SP_H + i] = a[1 + i] / (2.0 + i);
    for (int i = 0; i < 3; ++i) spec[SP_REC * k + SP_S + i] = a[2 + i] / (2.0 + i);
  }
  // reactions
  std::vector<double> rec(RX_REC * M);
  std::vector<double> troe;
  std::vector<double> eff;
  std::vector<double> lnA(M);
  int n_eff = 0, n_troe = 0;
  for (int j = 0; j < M; ++j) {
    const JVal& r = rx->arr[j];
    const std::string tag = "reaction " + std::to_string(j) + ": ";
    RxMeta meta;
    memset(&meta, 0, sizeof(meta));
    RxSlots slots{-1, -1};
    int cnt[2] = {0, 0};
    const char* sides[2] = {"reactants", "products"};
    for (int sd = 0; sd < 2; ++sd) {
      const JVal* side = r.get(sides[sd]);
      if (!side || side->kind != JVal::OBJ) return set_error(DF_EMECH, tag + "needs " + sides[sd]);
      for (auto& kv : side->obj) {
        auto it = index.find(kv.first);
        if (it == index.end()) return set_error(DF_EMECH, tag + "unknown species " + kv.first);
        double nu;
        if (!num_of(&kv.second, &nu) || nu != std::floor(nu) || nu < 1 || nu > 3)
          return set_error(DF_EMECH, tag + "stoichiometric coefficients must be integers 1..3");
        for (int q = 0; q < (int)nu; ++q) {
          if (cnt[sd] >= 3) return set_error(DF_EMECH, tag + "more than 3 species entries on one side");
          (sd == 0 ? meta.reac : meta.prod)[cnt[sd]++] = (uint8_t)it->second;
        }
      }
      if (cnt[sd] == 0) return set_error(DF_EMECH, tag + "empty side");
    }
    meta.nrnp = (uint8_t)(cnt[0] | (cnt[1] << 4));
    const JVal* type = r.get("type");
    int t = 0;
    if (type) {
      if (type->kind != JVal::STR) return set_error(DF_EMECH, tag + "type must be a string");
      if (type->str == "elementary") t = 0;
      else if (type->str == "three-body") t = 1;
      else if (type->str == "falloff-troe") t = 2;
      else return set_error(DF_EMECH, tag + "unknown type " + type->str);
    }
    bool rev = true;
    if (const JVal* rv = r.get("reversible")) {
      if (rv->kind != JVal::BOOL) return set_error(DF_EMECH, tag + "reversible must be a bool");
      rev = rv->b;
    }
    meta.flags = (uint8_t)(t | (rev ? 4 : 0));
    double A, b, Ea;
    if (!num_of(r.get("A"), &A) || !num_of(r.get("b"), &b) || !num_of(r.get("Ea"), &Ea))
      return set_error(DF_EMECH, tag + "needs numeric A, b, Ea");
    if (A < 0.0) return set_error(DF_EMECH, tag + "A must be >= 0");
    lnA[j] = std::log(A);  // -inf for A = 0: K_f = 0
    rec[RX_REC * j + 0] = lnA[j];
    rec[RX_REC * j + 1] = b;
    rec[RX_REC * j + 2] = Ea * 1e3 / RU_SI;
    if (t != 0) {
      slots.eff = n_eff++;
      std::vector<double> e(N, 1.0);
      if (const JVal* ev = r.get("efficiencies")) {
        if (ev->kind != JVal::OBJ) return set_error(DF_EMECH, tag + "efficiencies must be an object");
        for (auto& kv : ev->obj) {
          auto it = index.find(kv.first);
          if (it == index.end()) return set_error(DF_EMECH, tag + "unknown species " + kv.first);
          if (!num_of(&kv.second, &e[it->second])) return set_error(DF_EMECH, tag + "bad efficiency");
        }
      }
      eff.insert(eff.end(), e.begin(), e.end());
    }
    if (t == 2) {
      const JVal* lo = r.get("low");
      const JVal* tr = r.get("troe");
      double A0, b0, Ea0, al, T3, T1, T2;
      if (!lo || !tr || !num_of(lo->get("A"), &A0) || !num_of(lo->get("b"), &b0) ||
          !num_of(lo->get("Ea"), &Ea0) || !num_of(tr->get("alpha"), &al) ||
          !num_of(tr->get("T3"), &T3) || !num_of(tr->get("T1"), &T1) || !num_of(tr->get("T2"), &T2))
        return set_error(DF_EMECH, tag + "falloff-troe needs low{A,b,Ea} and troe{alpha,T3,T1,T2}");
      if (A0 < 0.0 || !(T3 > 0.0) || !(T1 > 0.0))
        return set_error(DF_EMECH, tag + "bad Troe parameters");
      slots.troe = n_troe++;
      double d0 = (A == 0.0 || A0 == 0.0) ? -INFINITY : std::log(A0) - std::log(A);
      double trec[TR_REC] = {d0, b0, Ea0 * 1e3 / RU_SI, al, 1.0 / T3, 1.0 / T1, T2, 0.0};
      troe.insert(troe.end(), trec, trec + TR_REC);
    }
    memcpy(&rec[RX_REC * j + 3], &meta, 8);
    memcpy(&rec[RX_REC * j + 4], &slots, 8);
  }
  MechDims d = mech_dims(N, M, n_eff, n_troe);
  m->dims = d;
  m->blob_host.assign(d.total, 0.0);
  std::copy(spec.begin(), spec.end(), m->blob_host.begin() + d.off_sp);
  std::copy(rec.begin(), rec.end(), m->blob_host.begin() + d.off_rx);
  std::copy(troe.begin(), troe.end(), m->blob_host.begin() + d.off_tr);
  std::copy(eff.begin(), eff.end(), m->blob_host.begin() + d.off_eff);
  m->lnA_file = lnA;
  // species -> (reaction, net stoichiometric coefficient nu''_kj - nu'_kj) lists
  std::vector<std::vector<std::pair<int, int>>> lists(N);
  for (int j = 0; j < M; ++j) {
    RxMeta meta;
    memcpy(&meta, &rec[RX_REC * j + 3], 8);
    std::vector<int> nu(N, 0);
    for (int i = 0; i < (meta.nrnp & 15); ++i) nu[meta.reac[i]] -= 1;
    for (int i = 0; i < (meta.nrnp >> 4); ++i) nu[meta.prod[i]] += 1;
    for (int k = 0; k < N; ++k)
      if (nu[k] != 0) lists[k].emplace_back(j, nu[k]);
  }
  m->csr_host.assign(N + 1, 0);
  for (int k = 0; k < N; ++k) m->csr_host[k + 1] = m->csr_host[k] + (int)lists[k].size();
  for (int k = 0; k < N; ++k)
    for (auto& e : lists[k]) {
      m->csr_host.push_back(e.first);
      m->csr_host.push_back(e.second);
    }
  // Lane assignment of the warp path's species loops (production rates and
  // Jacobian rows): at most two species per lane, balanced by the cost of
  // their reaction lists (longest first, each to the least-loaded lane that
  // still has a free slot).  A third-body entry adds a full row of
  // efficiencies to the Jacobian row.  Table: 32 x (k0, k1), -1 = none.
  std::vector<std::pair<long, int>> cost(N);
  for (int k = 0; k < N; ++k) {
    long c = 0;
    for (auto& e : lists[k]) {
      RxMeta meta;
      memcpy(&meta, &rec[RX_REC * e.first + 3], 8);
      c += 13 + (((meta.flags & 3) != 0) ? N : 0);
    }
    cost[k] = {c, k};
  }
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<long, int>& a, const std::pair<long, int>& b) { return a.first > b.first; });
  std::vector<int> asg(64, -1);
  std::vector<long> load(32, 0);
  std::vector<int> used(32, 0);
  for (auto& ck : cost) {
    int best = -1;
    for (int l = 0; l < 32; ++l)
      if (used[l] < 2 && (best < 0 || load[l] < load[best])) best = l;
    if (best < 0) return set_error(DF_EMECH, "more than 64 species");  // excluded by the parser's limit
    asg[2 * best + used[best]] = ck.second;
    ++used[best];
    load[best] += ck.first;
  }
  m->csr_host.insert(m->csr_host.end(), asg.begin(), asg.end());
  // Sparse third-body efficiencies for the warp path: [n_eff], offsets
  // [n_eff + 1] (in triples), then per slot the (species, low word, high word)
  // triples of eps_l - 1 for every species whose efficiency is not 1.
  m->csr_host.push_back(n_eff);
  const size_t off0 = m->csr_host.size();
  m->csr_host.resize(off0 + n_eff + 1, 0);
  int ntrip = 0;
  for (int sl = 0; sl < n_eff; ++sl) {
    m->csr_host[off0 + sl] = ntrip;
    for (int l = 0; l < N; ++l) {
      const double e = eff[(size_t)sl * N + l];
      if (e == 1.0) continue;
      const double dlt = e - 1.0;
      unsigned long long bits;
      memcpy(&bits, &dlt, 8);
      m->csr_host.push_back(l);
      m->csr_host.push_back((int)(unsigned)(bits & 0xffffffffull));
      m->csr_host.push_back((int)(unsigned)(bits >> 32));
      ++ntrip;
    }
  }
  m->csr_host[off0 + n_eff] = ntrip;
  return DF_OK;
}

}  // namespace df
