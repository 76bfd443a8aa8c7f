// MPO construction for H, H0 and U (Theory section, Eq. "part"; MPO form of
// Eq. mpo with bond dimension O(k^2), Implementation section).
//
// Every spin-orbital term of H is brought to a canonical operator string
// (stable sort by orbital then spin, with the fermionic sign of each swap).
// In the Jordan-Wigner matrix representation used for the MPS basis, a term
// is a Kronecker product of local 4x4 factors F(x) = (ops at site x) *
// P^(#ops right of x), P = (-1)^n.  At every bond a term is represented by a
// channel labelled either by its left ops (a "prefix": identity, one op, or
// two ops while the left block is the smaller side) or by its right ops (a
// "suffix": one op, two ops, or none = the finished left Hamiltonian).  A
// prefix channel is one product operator; a suffix channel is the sum of all
// left parts sharing that suffix (a complementary operator).  Each term
// switches from prefix to suffix labelling at exactly one site, where its
// coefficient enters the MPO; everywhere else channels pass through with a
// fixed local factor.  With at most two ops in any label the bond dimension
// is 2 + 4k + 8 min(n_left, n_right)^2, i.e. O(k^2).
#include "mpo.hpp"

#include <array>
#include <cmath>
#include <map>
#include <unordered_map>

namespace mpslcc {
namespace {

typedef std::array<double, 16> Mat4;  // [s_out * 4 + s_in]

// elementary kinds: 0 = a+ up, 1 = a+ dn, 2 = a up, 3 = a dn
inline int kspin(int kind) { return kind & 1; }
inline bool kcreate(int kind) { return kind < 2; }
inline QN kdq(int kind) {
  switch (kind) {
    case 0: return QN(1, 1);
    case 1: return QN(1, -1);
    case 2: return QN(-1, -1);
    default: return QN(-1, 1);
  }
}

Mat4 zero4() { Mat4 m; m.fill(0.0); return m; }
Mat4 ident4() { Mat4 m = zero4(); for (int i = 0; i < 4; ++i) m[i * 4 + i] = 1.0; return m; }
Mat4 parity4() { Mat4 m = zero4(); m[0] = 1; m[5] = -1; m[10] = -1; m[15] = 1; return m; }
Mat4 elem4(int kind) {
  // a+_up |0> = |up>, a+_up |dn> = |up dn>; a+_dn |0> = |dn>, a+_dn |up> = -|up dn>
  Mat4 m = zero4();
  auto set = [&](int so, int si, double v) { m[so * 4 + si] = v; };
  switch (kind) {
    case 0: set(1, 0, 1); set(3, 2, 1); break;
    case 1: set(2, 0, 1); set(3, 1, -1); break;
    case 2: set(0, 1, 1); set(2, 3, 1); break;
    case 3: set(0, 2, 1); set(1, 3, -1); break;
  }
  return m;
}
Mat4 mul4(const Mat4& a, const Mat4& b) {
  Mat4 c = zero4();
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      double v = a[i * 4 + k];
      if (v == 0.0) continue;
      for (int j = 0; j < 4; ++j) c[i * 4 + j] += v * b[k * 4 + j];
    }
  return c;
}

struct Op { int site, kind; };
struct Term { Op op[4]; int n; double c; };

uint64_t string_key(const Op* ops, int n) {
  uint64_t k = (uint64_t)n;
  for (int i = 0; i < n; ++i) k = (k << 14) | (uint64_t)((ops[i].site << 2) | ops[i].kind);
  return k;
}

// Stable sort by (site, spin) with fermionic signs; returns 0 if the string
// vanishes (same spin orbital created or annihilated twice).
int canonicalize(Op* ops, int n) {
  int sign = 1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j + 1 < n - i; ++j) {
      int ka = ops[j].site * 2 + kspin(ops[j].kind);
      int kb = ops[j + 1].site * 2 + kspin(ops[j + 1].kind);
      if (ka > kb) {
        std::swap(ops[j], ops[j + 1]);
        sign = -sign;
      }
    }
  for (int j = 0; j + 1 < n; ++j)
    if (ops[j].site == ops[j + 1].site && ops[j].kind == ops[j + 1].kind) return 0;
  return sign;
}

// channel labels
enum { T_I = 0, T_PRE1 = 1, T_PRE2 = 2, T_SUF2 = 3, T_SUF1 = 4, T_HL = 5 };

inline uint64_t mklabel(int type, int kinds, int major, int minor) {
  return ((uint64_t)type << 56) | ((uint64_t)kinds << 48) | ((uint64_t)major << 24) | (uint64_t)minor;
}
inline int label_type(uint64_t l) { return (int)(l >> 56); }
inline bool prefix_like(uint64_t l) { int t = label_type(l); return t == T_I || t == T_PRE1 || t == T_PRE2; }

struct Labeler {
  int k;
  bool small(int b) const { return b <= k - b; }
  uint64_t operator()(const Term& t, int b) const {
    int nL = 0;
    while (nL < t.n && t.op[nL].site < b) ++nL;
    int nR = t.n - nL;
    if (nR == 0) return mklabel(T_HL, 0, 0, 0);
    if (nL == 0) return mklabel(T_I, 0, 0, 0);
    if (nL == 1) return mklabel(T_PRE1, t.op[0].kind, t.op[0].site, 0);
    if (nR == 1) return mklabel(T_SUF1, t.op[t.n - 1].kind, t.op[t.n - 1].site, 0);
    // nL == 2 && nR == 2
    if (small(b))
      return mklabel(T_PRE2, t.op[0].kind * 4 + t.op[1].kind, t.op[1].site, t.op[0].site);
    return mklabel(T_SUF2, t.op[2].kind * 4 + t.op[3].kind, t.op[2].site, t.op[3].site);
  }
};

QN label_dq(uint64_t l) {
  int type = label_type(l);
  int kinds = (int)((l >> 48) & 0xff);
  switch (type) {
    case T_PRE1: return kdq(kinds);
    case T_PRE2: return kdq(kinds / 4) + kdq(kinds % 4);
    case T_SUF1: return -kdq(kinds);
    case T_SUF2: return -(kdq(kinds / 4) + kdq(kinds % 4));
    default: return QN(0, 0);
  }
}
int label_nops(uint64_t l) {
  int t = label_type(l);
  return (t == T_PRE1 || t == T_SUF1) ? 1 : ((t == T_PRE2 || t == T_SUF2) ? 2 : 0);
}

// local factor of a term at site x
Mat4 term_factor(const Term& t, int x) {
  Mat4 m = ident4();
  int nright = 0;
  for (int i = 0; i < t.n; ++i) {
    if (t.op[i].site == x) m = mul4(m, elem4(t.op[i].kind));
    else if (t.op[i].site > x) ++nright;
  }
  if (nright & 1) m = mul4(m, parity4());
  return m;
}

struct OpTable {
  std::vector<Mat4> mats;
  std::map<std::vector<int>, int> index;  // key: kinds at site + parity
  int get(const Term& t, int x) {
    std::vector<int> key;
    int nright = 0;
    for (int i = 0; i < t.n; ++i) {
      if (t.op[i].site == x) key.push_back(t.op[i].kind);
      else if (t.op[i].site > x) ++nright;
    }
    key.push_back(100 + (nright & 1));
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    int id = (int)mats.size();
    mats.push_back(term_factor(t, x));
    index[key] = id;
    return id;
  }
  int passive(int parity) {
    std::vector<int> key{200 + parity};
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    int id = (int)mats.size();
    mats.push_back(parity ? parity4() : ident4());
    index[key] = id;
    return id;
  }
};

void make_bond(MpoBond& B, const std::vector<uint64_t>& labels) {
  // order: class (dq ascending), then label key
  std::vector<std::pair<QN, uint64_t>> v;
  for (auto l : labels) v.push_back({label_dq(l), l});
  std::sort(v.begin(), v.end(), [](const std::pair<QN, uint64_t>& a, const std::pair<QN, uint64_t>& b) {
    if (!(a.first == b.first)) return a.first < b.first;
    return a.second < b.second;
  });
  B.n = (int)v.size();
  B.dq.resize(B.n);
  B.cls.resize(B.n);
  B.pos.resize(B.n);
  for (int i = 0; i < B.n; ++i) {
    B.dq[i] = v[i].first;
    if (B.class_dq.empty() || !(B.class_dq.back() == v[i].first)) {
      B.class_dq.push_back(v[i].first);
      B.class_start.push_back(i);
      B.class_n.push_back(0);
    }
    B.cls[i] = (int)B.class_dq.size() - 1;
    B.pos[i] = B.class_n.back()++;
  }
}

// Group the expanded entries of one site into fusion recipes.
std::vector<FuseGroup> make_groups(const std::vector<MpoEntry>& e, bool left_fuse, const MpoBond& tb,
                                   const MpoBond& sb) {
  // key (so, si, tcls) -> target -> list of (source, val)
  std::map<std::tuple<int, int, int>, std::map<int, std::vector<std::pair<int, double>>>> g;
  for (const auto& x : e) {
    int t = left_fuse ? x.w1 : x.w0;
    int s = left_fuse ? x.w0 : x.w1;
    g[std::make_tuple(x.so, x.si, tb.cls[t])][t].push_back({s, x.val});
  }
  std::vector<FuseGroup> out;
  for (auto& kv : g) {
    FuseGroup fg;
    fg.so = std::get<0>(kv.first);
    fg.si = std::get<1>(kv.first);
    fg.tcls = std::get<2>(kv.first);
    fg.scls = -1;
    std::vector<int> single, multi;
    for (auto& row : kv.second) {
      for (auto& sv : row.second) {
        int sc = sb.cls[sv.first];
        if (fg.scls < 0) fg.scls = sc;
        MPSLCC_REQUIRE(fg.scls == sc, ST_INTERNAL, "MPO fusion group mixes source classes");
      }
      (row.second.size() == 1 ? single : multi).push_back(row.first);
    }
    int t0 = tb.class_start[fg.tcls], s0 = sb.class_start[fg.scls];
    // pass runs
    for (size_t i = 0; i < single.size();) {
      int t = single[i];
      auto sv = kv.second[t][0];
      FuseGroup::Run r{t - t0, sv.first - s0, 1, sv.second};
      size_t j = i + 1;
      while (j < single.size()) {
        int tn = single[j];
        auto svn = kv.second[tn][0];
        if (tn == t + (int)(j - i) && svn.first == sv.first + (int)(j - i) && svn.second == sv.second) {
          ++r.n;
          ++j;
        } else
          break;
      }
      fg.runs.push_back(r);
      i = j;
    }
    // dense boxes over runs of consecutive multi-source rows
    for (size_t i = 0; i < multi.size();) {
      size_t j = i + 1;
      int lo = 1 << 30, hi = -1;
      for (auto& sv : kv.second[multi[i]]) { lo = std::min(lo, sv.first); hi = std::max(hi, sv.first); }
      while (j < multi.size() && multi[j] == multi[j - 1] + 1) {
        int l2 = 1 << 30, h2 = -1;
        for (auto& sv : kv.second[multi[j]]) { l2 = std::min(l2, sv.first); h2 = std::max(h2, sv.first); }
        // keep boxes reasonably tight
        int nlo = std::min(lo, l2), nhi = std::max(hi, h2);
        if ((nhi - nlo + 1) > 2 * std::max(hi - lo + 1, h2 - l2 + 1) + 8) break;
        lo = nlo;
        hi = nhi;
        ++j;
      }
      FuseGroup::Box b;
      b.t = multi[i] - t0;
      b.nt = (int)(j - i);
      b.s = lo - s0;
      b.ns = hi - lo + 1;
      b.C.assign((size_t)b.nt * b.ns, 0.0);
      for (size_t r = i; r < j; ++r)
        for (auto& sv : kv.second[multi[r]]) b.C[(r - i) * b.ns + (sv.first - lo)] += sv.second;
      fg.boxes.push_back(std::move(b));
      i = j;
    }
    out.push_back(std::move(fg));
  }
  return out;
}

}  // namespace

Mpo build_mpo(int k, const double* h, const double* V, int kind, int n_core, int n_active) {
  MPSLCC_REQUIRE(k >= 2 && k <= 60, ST_ARG, "n_orb must be in [2, 60]");
  Mpo mpo;
  mpo.k = k;
  mpo.bond.resize(k + 1);
  mpo.site.resize(k);

  std::vector<Term> terms;
  if (kind != MPO_ID) {
    auto set_of = [&](int p) { return p < n_core ? 0 : (p < n_core + n_active ? 1 : 2); };
    std::unordered_map<uint64_t, Term> merged;
    merged.reserve(1 << 20);
    auto add = [&](Op* ops, int n, double c) {
      if (kind != MPO_H) {
        int cnt[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) cnt[set_of(ops[i].site)] += kcreate(ops[i].kind) ? 1 : -1;
        bool keep0 = cnt[0] == 0 && cnt[1] == 0 && cnt[2] == 0;
        if ((kind == MPO_H0) != keep0) return;
      }
      int sg = canonicalize(ops, n);
      if (sg == 0) return;
      uint64_t key = string_key(ops, n);
      auto it = merged.find(key);
      if (it == merged.end()) {
        Term t;
        t.n = n;
        t.c = sg * c;
        for (int i = 0; i < n; ++i) t.op[i] = ops[i];
        merged.emplace(key, t);
      } else
        it->second.c += sg * c;
    };
    const double tol = 1e-14;
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q) {
        double v = h[p * k + q];
        if (std::fabs(v) <= tol) continue;
        for (int s = 0; s < 2; ++s) {
          Op ops[2] = {{p, s}, {q, 2 + s}};
          add(ops, 2, v);
        }
      }
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q)
        for (int r = 0; r < k; ++r)
          for (int s = 0; s < k; ++s) {
            double v = V[(((size_t)p * k + q) * k + r) * k + s];
            if (std::fabs(v) <= tol) continue;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) {
                if (p == r && a == b) continue;
                if (s == q && a == b) continue;
                // 1/2 (pq|rs) a+_{p a} a+_{r b} a_{s b} a_{q a}
                Op ops[4] = {{p, a}, {r, b}, {s, 2 + b}, {q, 2 + a}};
                add(ops, 4, 0.5 * v);
              }
          }
    for (auto& kv : merged)
      if (std::fabs(kv.second.c) > 1e-13) terms.push_back(kv.second);
    std::sort(terms.begin(), terms.end(), [](const Term& a, const Term& b) {
      return string_key(a.op, a.n) < string_key(b.op, b.n);
    });
  }
  mpo.n_terms = (long)terms.size();

  if (kind == MPO_ID || terms.empty()) {
    // identity MPO (kind ID) or the zero operator (identity with a zero site)
    for (int b = 0; b <= k; ++b) make_bond(mpo.bond[b], {mklabel(T_I, 0, 0, 0)});
    for (int x = 0; x < k; ++x) {
      double v = (kind == MPO_ID || x > 0) ? 1.0 : 0.0;
      if (v != 0.0)
        for (int s = 0; s < 4; ++s) mpo.site[x].e.push_back({0, 0, s, s, v});
    }
  } else {
    Labeler lab{k};
    // channel discovery: label -> bitmask of bonds where it is used
    std::unordered_map<uint64_t, std::vector<uint8_t>> used;
    auto mark = [&](uint64_t l, int b) {
      auto& v = used[l];
      if (v.empty()) v.assign(k + 1, 0);
      v[b] = 1;
    };
    for (const auto& t : terms)
      for (int b = 0; b <= k; ++b) mark(lab(t, b), b);
    std::vector<std::vector<uint64_t>> blabels(k + 1);
    for (auto& kv : used)
      for (int b = 0; b <= k; ++b)
        if (kv.second[b]) blabels[b].push_back(kv.first);
    for (int b = 0; b <= k; ++b) make_bond(mpo.bond[b], blabels[b]);
    // label -> channel index per bond
    std::vector<std::unordered_map<uint64_t, int>> chan(k + 1);
    for (int b = 0; b <= k; ++b) {
      std::vector<std::pair<QN, uint64_t>> v;
      for (auto l : blabels[b]) v.push_back({label_dq(l), l});
      std::sort(v.begin(), v.end(), [](const std::pair<QN, uint64_t>& a, const std::pair<QN, uint64_t>& c) {
        if (!(a.first == c.first)) return a.first < c.first;
        return a.second < c.second;
      });
      for (int i = 0; i < (int)v.size(); ++i) chan[b][v[i].second] = i;
    }
    OpTable ops;
    for (int x = 0; x < k; ++x) {
      std::map<std::pair<int, int>, int> pass;                 // (w0, w1) -> op id
      std::map<std::tuple<int, int, int>, double> sw;          // (w0, w1, op) -> coef
      // passive pass-throughs: labels present on both sides of site x
      for (auto& kv : chan[x + 1]) {
        auto it = chan[x].find(kv.first);
        if (it == chan[x].end()) continue;
        pass[{it->second, kv.second}] = ops.passive(label_nops(kv.first) & 1);
      }
      for (const auto& t : terms) {
        bool has = false;
        for (int i = 0; i < t.n; ++i) has |= (t.op[i].site == x);
        uint64_t l0 = lab(t, x), l1 = lab(t, x + 1);
        if (!has && l0 == l1) continue;
        int w0 = chan[x].at(l0), w1 = chan[x + 1].at(l1);
        bool p0 = prefix_like(l0), p1 = prefix_like(l1);
        MPSLCC_REQUIRE(!(!p0 && p1), ST_INTERNAL, "MPO labelling not monotone");
        int id = ops.get(t, x);
        if (p0 == p1) {
          auto key = std::make_pair(w0, w1);
          auto it = pass.find(key);
          if (it == pass.end()) pass[key] = id;
          else MPSLCC_REQUIRE(ops.mats[it->second] == ops.mats[id], ST_INTERNAL, "inconsistent MPO pass factor");
        } else {
          sw[std::make_tuple(w0, w1, id)] += t.c;
        }
      }
      std::map<std::tuple<int, int, int, int>, double> acc;
      for (auto& kv : pass) {
        const Mat4& m = ops.mats[kv.second];
        for (int so = 0; so < 4; ++so)
          for (int si = 0; si < 4; ++si)
            if (m[so * 4 + si] != 0.0)
              acc[std::make_tuple(kv.first.first, kv.first.second, so, si)] += m[so * 4 + si];
      }
      for (auto& kv : sw) {
        const Mat4& m = ops.mats[std::get<2>(kv.first)];
        for (int so = 0; so < 4; ++so)
          for (int si = 0; si < 4; ++si)
            if (m[so * 4 + si] != 0.0)
              acc[std::make_tuple(std::get<0>(kv.first), std::get<1>(kv.first), so, si)] +=
                  kv.second * m[so * 4 + si];
      }
      for (auto& kv : acc)
        if (kv.second != 0.0)
          mpo.site[x].e.push_back({std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                                   std::get<3>(kv.first), kv.second});
    }
  }
  for (int x = 0; x < k; ++x) {
    mpo.site[x].lfuse = make_groups(mpo.site[x].e, true, mpo.bond[x + 1], mpo.bond[x]);
    mpo.site[x].rfuse = make_groups(mpo.site[x].e, false, mpo.bond[x], mpo.bond[x + 1]);
  }
  return mpo;
}

}  // namespace mpslcc
