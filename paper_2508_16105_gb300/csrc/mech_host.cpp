// Host-side reader, validator and packer for RDEMECH 1 mechanism text.
//
// Produces the packed byte image of mech_layout.h (SI units, ln A, E/R_u,
// NASA-7 fits regrouped per range for Horner evaluation).
#include <cmath>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "fastmath_tables.h"
#include "large_plan.h"
#include "mech_host.h"

namespace rde {

namespace {

constexpr double kRu = 8.31446261815324;  // J/(mol K)

struct Line {
  int no;
  std::vector<std::string> tok;
};

bool to_double(const std::string& s, double* v) {
  const char* b = s.c_str();
  char* e = nullptr;
  *v = std::strtod(b, &e);
  return e != b && *e == '\0';
}

bool to_int(const std::string& s, long* v) {
  const char* b = s.c_str();
  char* e = nullptr;
  *v = std::strtol(b, &e, 10);
  return e != b && *e == '\0';
}

struct Species {
  std::string name;
  double W_g, Tlow, Tmid, Thigh;
  std::vector<long> comp;
  double lo[7], hi[7];
};

struct Reaction {
  int type = RX_ELEM;
  bool rev = true;
  std::vector<std::pair<int, int>> reac, prod;  // (species, coefficient)
  double A = 0, b = 0, E = 0;
  bool has_low = false;
  double A0 = 0, b0 = 0, E0 = 0;
  int ntroe = 0;
  double troe[4] = {0, 0, 0, 0};
  std::vector<std::pair<int, double>> eff;
  int line = 0;
};

struct Parser {
  std::vector<Line> lines;
  size_t pos = 0;
  std::string err;

  bool fail(int line, const std::string& msg) {
    std::ostringstream o;
    o << "line " << line << ": " << msg;
    err = o.str();
    return false;
  }
};

}  // namespace

int pack_mechanism(const char* text, size_t len, std::vector<unsigned char>* image, std::string* err,
                   std::vector<double>* E_J) {
  Parser P;
  {
    std::string s(text, len);
    std::istringstream in(s);
    std::string ln;
    int no = 0;
    while (std::getline(in, ln)) {
      ++no;
      std::istringstream ls(ln);
      Line L;
      L.no = no;
      std::string t;
      while (ls >> t) L.tok.push_back(t);
      if (L.tok.empty() || L.tok[0][0] == '#') continue;
      P.lines.push_back(std::move(L));
    }
  }
  auto& Ls = P.lines;
  auto need = [&](size_t i, const char* kw, size_t ntok) -> bool {
    if (i >= Ls.size()) return P.fail(Ls.empty() ? 0 : Ls.back().no, std::string("missing ") + kw);
    if (Ls[i].tok[0] != kw) return P.fail(Ls[i].no, std::string("expected ") + kw + ", found " + Ls[i].tok[0]);
    if (Ls[i].tok.size() < ntok) return P.fail(Ls[i].no, std::string("too few fields in ") + kw);
    return true;
  };
  size_t i = 0;
  if (Ls.empty() || Ls[0].tok.size() != 2 || Ls[0].tok[0] != "RDEMECH" || Ls[0].tok[1] != "1") {
    *err = "not an RDEMECH 1 file";
    return -1;
  }
  ++i;
  if (!need(i, "ELEMENTS", 2)) { *err = P.err; return -1; }
  long ne = 0;
  if (!to_int(Ls[i].tok[1], &ne) || ne < 1 || (size_t)(ne + 2) != Ls[i].tok.size()) {
    *err = "line " + std::to_string(Ls[i].no) + ": bad ELEMENTS record";
    return -1;
  }
  ++i;
  if (!need(i, "SPECIES", 2)) { *err = P.err; return -1; }
  long K = 0;
  if (!to_int(Ls[i].tok[1], &K) || K < 1 || K > 4096) {
    *err = "line " + std::to_string(Ls[i].no) + ": bad species count";
    return -1;
  }
  ++i;
  std::vector<Species> sp;
  std::map<std::string, int> index;
  for (long k = 0; k < K; ++k) {
    if (!need(i, "SP", (size_t)(7 + ne - 1))) { *err = P.err; return -1; }
    const Line& L = Ls[i];
    if (L.tok.size() != (size_t)(6 + ne)) { *err = "line " + std::to_string(L.no) + ": bad SP record"; return -1; }
    Species s;
    s.name = L.tok[1];
    if (index.count(s.name)) { *err = "line " + std::to_string(L.no) + ": duplicate species " + s.name; return -2; }
    if (!to_double(L.tok[2], &s.W_g) || !to_double(L.tok[3], &s.Tlow) || !to_double(L.tok[4], &s.Tmid) ||
        !to_double(L.tok[5], &s.Thigh)) {
      *err = "line " + std::to_string(L.no) + ": bad number in SP record";
      return -1;
    }
    if (!(s.W_g > 0) || !std::isfinite(s.W_g)) { *err = "species " + s.name + ": molar mass must be > 0"; return -2; }
    if (!(s.Tlow > 0 && s.Tlow < s.Tmid && s.Tmid < s.Thigh) || !std::isfinite(s.Thigh)) {
      *err = "species " + s.name + ": need 0 < Tlow < Tmid < Thigh";
      return -2;
    }
    for (long e = 0; e < ne; ++e) {
      long c;
      if (!to_int(L.tok[6 + e], &c) || c < 0) { *err = "species " + s.name + ": bad element count"; return -1; }
      s.comp.push_back(c);
    }
    for (int r = 0; r < 2; ++r) {
      const char* kw = r == 0 ? "LO" : "HI";
      if (!need(i + 1 + r, kw, 8)) { *err = P.err; return -1; }
      double* a = r == 0 ? s.lo : s.hi;
      for (int j = 0; j < 7; ++j)
        if (!to_double(Ls[i + 1 + r].tok[1 + j], &a[j]) || !std::isfinite(a[j])) {
          *err = "species " + s.name + ": bad NASA coefficient";
          return -1;
        }
    }
    index[s.name] = (int)k;
    sp.push_back(s);
    i += 3;
  }
  if (!need(i, "REACTIONS", 2)) { *err = P.err; return -1; }
  long R = 0;
  if (!to_int(Ls[i].tok[1], &R) || R < 0 || R > 100000) {
    *err = "line " + std::to_string(Ls[i].no) + ": bad reaction count";
    return -1;
  }
  ++i;
  std::vector<Reaction> rx;
  while (i < Ls.size() && Ls[i].tok[0] != "END") {
    const Line& L = Ls[i];
    const std::string& kw = L.tok[0];
    if (kw == "RX") {
      Reaction r;
      r.line = L.no;
      if (L.tok.size() < 8) { *err = "line " + std::to_string(L.no) + ": short RX record"; return -1; }
      const std::string& ty = L.tok[1];
      if (ty == "ELEM") r.type = RX_ELEM;
      else if (ty == "THREEBODY") r.type = RX_THREEBODY;
      else if (ty == "LINDEMANN") r.type = RX_LINDEMANN;
      else if (ty == "TROE") r.type = RX_TROE;
      else { *err = "line " + std::to_string(L.no) + ": unknown reaction type " + ty; return -1; }
      if (L.tok[2] == "REV") r.rev = true;
      else if (L.tok[2] == "IRR") r.rev = false;
      else { *err = "line " + std::to_string(L.no) + ": expected REV or IRR"; return -1; }
      size_t q = 3;
      for (int side = 0; side < 2; ++side) {
        long ns;
        if (q >= L.tok.size() || !to_int(L.tok[q], &ns) || ns < 1 || ns > kMaxSide) {
          *err = "line " + std::to_string(L.no) + ": 1 to 3 species per side";
          return -2;
        }
        ++q;
        auto& lst = side == 0 ? r.reac : r.prod;
        int order = 0;
        for (long s = 0; s < ns; ++s) {
          if (q + 1 >= L.tok.size()) { *err = "line " + std::to_string(L.no) + ": short RX record"; return -1; }
          auto it = index.find(L.tok[q]);
          if (it == index.end()) { *err = "line " + std::to_string(L.no) + ": unknown species " + L.tok[q]; return -2; }
          long c;
          if (!to_int(L.tok[q + 1], &c) || c < 1 || c > kMaxOrder) {
            *err = "line " + std::to_string(L.no) + ": coefficients must be 1..3";
            return -2;
          }
          for (auto& pr : lst)
            if (pr.first == it->second) { *err = "line " + std::to_string(L.no) + ": species repeated on one side"; return -2; }
          lst.push_back({it->second, (int)c});
          order += (int)c;
          q += 2;
        }
        if (order > kMaxOrder) { *err = "line " + std::to_string(L.no) + ": total order above 3"; return -2; }
      }
      if (q + 3 != L.tok.size() || !to_double(L.tok[q], &r.A) || !to_double(L.tok[q + 1], &r.b) ||
          !to_double(L.tok[q + 2], &r.E)) {
        *err = "line " + std::to_string(L.no) + ": bad Arrhenius parameters";
        return -1;
      }
      if (!(r.A > 0) || !std::isfinite(r.A) || !std::isfinite(r.b) || !std::isfinite(r.E)) {
        *err = "line " + std::to_string(L.no) + ": A must be > 0 and finite";
        return -2;
      }
      rx.push_back(r);
    } else if (kw == "EFF" || kw == "LOW" || kw == "TROE") {
      if (rx.empty()) { *err = "line " + std::to_string(L.no) + ": " + kw + " before any reaction"; return -1; }
      Reaction& r = rx.back();
      if (kw == "EFF") {
        long n;
        if (r.type == RX_ELEM) { *err = "line " + std::to_string(L.no) + ": EFF on an elementary reaction"; return -2; }
        if (!to_int(L.tok[1], &n) || n < 0 || L.tok.size() != (size_t)(2 + 2 * n)) {
          *err = "line " + std::to_string(L.no) + ": bad EFF record";
          return -1;
        }
        for (long e = 0; e < n; ++e) {
          auto it = index.find(L.tok[2 + 2 * e]);
          double a;
          if (it == index.end()) { *err = "line " + std::to_string(L.no) + ": unknown species in EFF"; return -2; }
          if (!to_double(L.tok[3 + 2 * e], &a) || !(a >= 0) || !std::isfinite(a)) {
            *err = "line " + std::to_string(L.no) + ": efficiency must be >= 0";
            return -2;
          }
          r.eff.push_back({it->second, a});
        }
      } else if (kw == "LOW") {
        if (r.type != RX_LINDEMANN && r.type != RX_TROE) {
          *err = "line " + std::to_string(L.no) + ": LOW only for falloff reactions";
          return -2;
        }
        if (L.tok.size() != 4 || !to_double(L.tok[1], &r.A0) || !to_double(L.tok[2], &r.b0) ||
            !to_double(L.tok[3], &r.E0) || !(r.A0 > 0) || !std::isfinite(r.A0)) {
          *err = "line " + std::to_string(L.no) + ": bad LOW record";
          return -1;
        }
        r.has_low = true;
      } else {
        long n;
        if (r.type != RX_TROE) { *err = "line " + std::to_string(L.no) + ": TROE on a non-Troe reaction"; return -2; }
        if (!to_int(L.tok[1], &n) || (n != 3 && n != 4) || L.tok.size() != (size_t)(2 + n)) {
          *err = "line " + std::to_string(L.no) + ": TROE needs 3 or 4 parameters";
          return -1;
        }
        for (long j = 0; j < n; ++j)
          if (!to_double(L.tok[2 + j], &r.troe[j]) || !std::isfinite(r.troe[j])) {
            *err = "line " + std::to_string(L.no) + ": bad TROE parameter";
            return -1;
          }
        if (!(r.troe[1] > 0) || !(r.troe[2] > 0)) {
          *err = "line " + std::to_string(L.no) + ": TROE T*** and T* must be > 0";
          return -2;
        }
        r.ntroe = (int)n;
      }
    } else {
      *err = "line " + std::to_string(L.no) + ": unknown record " + kw;
      return -1;
    }
    ++i;
  }
  if (i >= Ls.size()) { *err = "missing END"; return -1; }
  if ((long)rx.size() != R) { *err = "reaction count does not match REACTIONS"; return -2; }

  // ---- validation that needs the whole file ----
  for (auto& r : rx) {
    const std::string where = "reaction at line " + std::to_string(r.line);
    if ((r.type == RX_LINDEMANN || r.type == RX_TROE) && !r.has_low) { *err = where + ": falloff without LOW"; return -2; }
    if (r.type == RX_TROE && r.ntroe == 0) { *err = where + ": TROE parameters missing"; return -2; }
    for (long e = 0; e < ne; ++e) {
      long bal = 0;
      for (auto& pr : r.reac) bal -= pr.second * sp[pr.first].comp[e];
      for (auto& pr : r.prod) bal += pr.second * sp[pr.first].comp[e];
      if (bal != 0) { *err = where + ": element " + Ls[1].tok[2 + e] + " not balanced"; return -2; }
    }
    std::vector<int> net(K, 0);
    for (auto& pr : r.reac) net[pr.first] -= pr.second;
    for (auto& pr : r.prod) net[pr.first] += pr.second;
    bool any = false;
    for (long k = 0; k < K; ++k) any |= net[k] != 0;
    if (!any) { *err = where + ": no net change"; return -2; }
  }

  // ---- pack ----
  std::vector<SpecPacked> S(K);
  for (long k = 0; k < K; ++k) {
    SpecPacked& s = S[k];
    std::memset(&s, 0, sizeof(s));
    s.W = sp[k].W_g * 1e-3;
    s.Winv = 1.0 / s.W;
    s.Tmid = sp[k].Tmid;
    for (int r = 0; r < 2; ++r) {
      const double* a = r == 0 ? sp[k].lo : sp[k].hi;
      for (int j = 0; j < 5; ++j) s.cp[r][j] = a[j];
      s.h[r][0] = a[0]; s.h[r][1] = a[1] / 2; s.h[r][2] = a[2] / 3; s.h[r][3] = a[3] / 4; s.h[r][4] = a[4] / 5;
      s.h[r][5] = a[5];
      // G/RT = H/RT - S/R
      s.g[r][0] = a[0] - a[6];
      s.g[r][1] = -a[0];
      s.g[r][2] = a[1] / 2 - a[1];
      s.g[r][3] = a[2] / 3 - a[2] / 2;
      s.g[r][4] = a[3] / 4 - a[3] / 3;
      s.g[r][5] = a[4] / 5 - a[4] / 4;
      s.g[r][6] = a[5];
      s.dcp[r][0] = a[1]; s.dcp[r][1] = 2 * a[2]; s.dcp[r][2] = 3 * a[3]; s.dcp[r][3] = 4 * a[4];
    }
  }
  std::vector<RxnPacked> X(R);
  std::vector<EffEntry> E;
  int n3 = 0, nfo = 0;
  for (long j = 0; j < R; ++j) {
    const Reaction& r = rx[j];
    RxnPacked& x = X[j];
    std::memset(&x, 0, sizeof(x));
    x.type = r.type;
    x.rev = r.rev ? 1 : 0;
    int order = 0;
    for (auto& pr : r.reac) order += pr.second;
    int m = order + (r.type == RX_THREEBODY ? 1 : 0);
    x.lnA = std::log(r.A) + (m - 1) * std::log(1e-6);
    x.b = r.b;
    x.EaR = r.E * 1e3 / kRu;
    if (E_J) E_J->push_back(r.E * 1e3);
    if (r.type == RX_LINDEMANN || r.type == RX_TROE) {
      x.lnA0 = std::log(r.A0) + order * std::log(1e-6);
      x.b0 = r.b0;
      x.EaR0 = r.E0 * 1e3 / kRu;
      ++nfo;
    }
    if (r.type == RX_THREEBODY) ++n3;
    if (r.type == RX_TROE) {
      x.troe_a = r.troe[0];
      x.troe_invT3 = 1.0 / r.troe[1];
      x.troe_invT1 = 1.0 / r.troe[2];
      x.troe_T2 = r.troe[3];
      x.has_T2 = r.ntroe == 4 ? 1 : 0;
    }
    x.nf = (int)r.reac.size();
    x.nb = (int)r.prod.size();
    for (int s = 0; s < x.nf; ++s) { x.fi[s] = r.reac[s].first; x.fo[s] = r.reac[s].second; x.fod[s] = r.reac[s].second; }
    for (int s = 0; s < x.nb; ++s) { x.bi[s] = r.prod[s].first; x.bo[s] = r.prod[s].second; x.bod[s] = r.prod[s].second; }
    std::vector<int> net(K, 0);
    for (auto& pr : r.reac) net[pr.first] -= pr.second;
    for (auto& pr : r.prod) net[pr.first] += pr.second;
    int dnu = 0;
    x.np = 0;
    // participants in first-appearance order: reactants then products
    std::vector<int> seen;
    for (auto& pr : r.reac) seen.push_back(pr.first);
    for (auto& pr : r.prod) seen.push_back(pr.first);
    for (int k : seen) {
      bool dup = false;
      for (int q = 0; q < x.np; ++q) dup |= x.pi[q] == k;
      if (dup || net[k] == 0) continue;
      x.pi[x.np] = k;
      x.pnu[x.np] = (double)net[k];
      ++x.np;
    }
    for (long k = 0; k < K; ++k) dnu += net[k];
    x.dnu = (double)dnu;
    x.eff_begin = (int)E.size();
    if (r.type != RX_ELEM) {
      for (auto& pe : r.eff) {
        if (pe.second == 1.0) continue;
        EffEntry e;
        std::memset(&e, 0, sizeof(e));
        e.alpha_minus_1 = pe.second - 1.0;
        e.k = pe.first;
        E.push_back(e);
      }
    }
    x.eff_end = (int)E.size();
  }
  MechHeader H;
  std::memset(&H, 0, sizeof(H));
  H.K = (int)K;
  H.R = (int)R;
  H.n_eff = (int)E.size();
  H.n_threebody = n3;
  H.n_falloff = nfo;
  const size_t tab_off = sizeof(MechHeader) + sizeof(SpecPacked) * K + sizeof(RxnPacked) * R + sizeof(EffEntry) * E.size();
  const size_t tab_bytes = sizeof(double) * (kExpTabSize + 2 * kLogTabSize);
  size_t bytes = tab_off + tab_bytes;
  H.bytes = (int)bytes;
  H.tab_offset = (int)tab_off;
  image->assign(bytes, 0);
  unsigned char* p = image->data();
  std::memcpy(p, &H, sizeof(H));
  p += sizeof(H);
  std::memcpy(p, S.data(), sizeof(SpecPacked) * K);
  p += sizeof(SpecPacked) * K;
  if (R) std::memcpy(p, X.data(), sizeof(RxnPacked) * R);
  p += sizeof(RxnPacked) * R;
  if (!E.empty()) std::memcpy(p, E.data(), sizeof(EffEntry) * E.size());
  p += sizeof(EffEntry) * E.size();
  std::memcpy(p, exp2_table_host(), sizeof(double) * kExpTabSize);
  p += sizeof(double) * kExpTabSize;
  std::memcpy(p, log_table_host(), sizeof(double) * 2 * kLogTabSize);
  return 0;
}

void build_large_plan(const unsigned char* image, std::vector<unsigned char>* plan) {
  const MechView v = mech_view(image);
  const int K = v.hdr->K, R = v.hdr->R;
  // omega_k: reactions with a non-zero net coefficient of k, ascending
  std::vector<std::vector<std::pair<int, double>>> spr(K), row(K);
  // D[k][j]: (reaction, slot, coefficient) in ascending reaction order
  std::vector<std::vector<std::vector<std::pair<int, std::pair<int, double>>>>> ent(K);
  for (int k = 0; k < K; ++k) ent[k].resize(K);
  for (int r = 0; r < R; ++r) {
    const RxnPacked& x = v.rx[r];
    for (int pp = 0; pp < x.np; ++pp) {
      const int k = x.pi[pp];
      const double nu = x.pnu[pp];
      spr[k].push_back({r, nu});
      for (int s = 0; s < x.nf; ++s) ent[k][x.fi[s]].push_back({r, {s, nu}});
      for (int s = 0; s < x.nb; ++s) ent[k][x.bi[s]].push_back({r, {3 + s, nu}});
      if (x.type != RX_ELEM) {
        row[k].push_back({r, nu});
        for (int e = x.eff_begin; e < x.eff_end; ++e)
          ent[k][v.eff[e].k].push_back({r, {6, nu * v.eff[e].alpha_minus_1}});
      }
    }
  }
  std::vector<int32_t> spr_ptr(K + 1, 0), spr_r, row_ptr(K + 1, 0), row_r, ent_index((size_t)K * K, -1), ent_ptr(1, 0),
      con_r, con_slot;
  std::vector<double> spr_nu, row_nu, con_coef;
  for (int k = 0; k < K; ++k) {
    for (auto& e : spr[k]) {
      spr_r.push_back(e.first);
      spr_nu.push_back(e.second);
    }
    spr_ptr[k + 1] = (int32_t)spr_r.size();
    for (auto& e : row[k]) {
      row_r.push_back(e.first);
      row_nu.push_back(e.second);
    }
    row_ptr[k + 1] = (int32_t)row_r.size();
    for (int j = 0; j < K; ++j) {
      if (ent[k][j].empty()) continue;
      ent_index[(size_t)k * K + j] = (int32_t)(ent_ptr.size() - 1);
      for (auto& c : ent[k][j]) {
        con_r.push_back(c.first);
        con_slot.push_back(c.second.first);
        con_coef.push_back(c.second.second);
      }
      ent_ptr.push_back((int32_t)con_r.size());
    }
  }
  PlanHeader H;
  std::memset(&H, 0, sizeof(H));
  H.K = K;
  H.R = R;
  H.n_spr = (int32_t)spr_r.size();
  H.n_ent = (int32_t)(ent_ptr.size() - 1);
  H.n_con = (int32_t)con_r.size();
  H.n_row = (int32_t)row_r.size();
  size_t off = sizeof(PlanHeader);
  auto place = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 15) & ~(size_t)15;
    return (int32_t)o;
  };
  H.o_spr_ptr = place(4 * spr_ptr.size());
  H.o_spr_r = place(4 * spr_r.size());
  H.o_spr_nu = place(8 * spr_nu.size());
  H.o_ent_index = place(4 * ent_index.size());
  H.o_ent_ptr = place(4 * ent_ptr.size());
  H.o_con_r = place(4 * con_r.size());
  H.o_con_slot = place(4 * con_slot.size());
  H.o_con_coef = place(8 * con_coef.size());
  H.o_row_ptr = place(4 * row_ptr.size());
  H.o_row_r = place(4 * row_r.size());
  H.o_row_nu = place(8 * row_nu.size());
  H.rx_stride = plan_rx_stride(R);
  H.rx_bytes = plan_rx_bytes(R);
  H.o_rx = place((size_t)H.rx_bytes);
  H.bytes = (int32_t)off;
  plan->assign(off, 0);
  unsigned char* b = plan->data();
  std::memcpy(b, &H, sizeof(H));
  auto put = [&](int32_t o, const void* src, size_t bytes) {
    if (bytes) std::memcpy(b + o, src, bytes);
  };
  put(H.o_spr_ptr, spr_ptr.data(), 4 * spr_ptr.size());
  put(H.o_spr_r, spr_r.data(), 4 * spr_r.size());
  put(H.o_spr_nu, spr_nu.data(), 8 * spr_nu.size());
  put(H.o_ent_index, ent_index.data(), 4 * ent_index.size());
  put(H.o_ent_ptr, ent_ptr.data(), 4 * ent_ptr.size());
  put(H.o_con_r, con_r.data(), 4 * con_r.size());
  put(H.o_con_slot, con_slot.data(), 4 * con_slot.size());
  put(H.o_con_coef, con_coef.data(), 8 * con_coef.size());
  put(H.o_row_ptr, row_ptr.data(), 4 * row_ptr.size());
  put(H.o_row_r, row_r.data(), 4 * row_r.size());
  put(H.o_row_nu, row_nu.data(), 8 * row_nu.size());
  // reaction table (structure of arrays)
  double* rxd = reinterpret_cast<double*>(b + H.o_rx);
  int32_t* meta = reinterpret_cast<int32_t*>(b + H.o_rx + 4 * 8 * H.rx_stride);
  for (int r = 0; r < R; ++r) {
    const RxnPacked& x = v.rx[r];
    rxd[0 * H.rx_stride + r] = x.lnA;
    rxd[1 * H.rx_stride + r] = x.b;
    rxd[2 * H.rx_stride + r] = x.EaR;
    rxd[3 * H.rx_stride + r] = x.dnu;
    int32_t w0 = (x.type & 3) | ((x.rev ? 1 : 0) << 2) | ((x.nf & 3) << 3) | ((x.nb & 3) << 5);
    int32_t w1 = 0, w2 = 0;
    for (int q = 0; q < kMaxSide; ++q) {
      if (q < x.nf) {
        w0 |= (x.fo[q] & 3) << (8 + 2 * q);
        w1 |= (x.fi[q] & 1023) << (10 * q);
      }
      if (q < x.nb) {
        w0 |= (x.bo[q] & 3) << (14 + 2 * q);
        w2 |= (x.bi[q] & 1023) << (10 * q);
      }
    }
    meta[4 * r + 0] = w0;
    meta[4 * r + 1] = w1;
    meta[4 * r + 2] = w2;
    meta[4 * r + 3] = 0;
  }
}

}  // namespace rde
