// Shared host-side types of the MPS-LCC library.
#pragma once
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>
#include <algorithm>

namespace mpslcc {

// U(1)xU(1) quantum number: electrons and 2*S_z.
struct QN {
  int n = 0, s = 0;
  QN() = default;
  QN(int n_, int s_) : n(n_), s(s_) {}
};
inline bool operator<(const QN& a, const QN& b) { return a.n < b.n || (a.n == b.n && a.s < b.s); }
inline bool operator==(const QN& a, const QN& b) { return a.n == b.n && a.s == b.s; }
inline bool operator!=(const QN& a, const QN& b) { return !(a == b); }
inline QN operator+(const QN& a, const QN& b) { return QN(a.n + b.n, a.s + b.s); }
inline QN operator-(const QN& a, const QN& b) { return QN(a.n - b.n, a.s - b.s); }
inline QN operator-(const QN& a) { return QN(-a.n, -a.s); }
inline uint64_t qkey(const QN& q) { return ((uint64_t)(uint32_t)(q.n + 4096) << 32) | (uint32_t)(q.s + 4096); }

// Local basis of one spatial orbital: 0=|0>, 1=|up>, 2=|dn>, 3=|up dn>.
static const QN LOCAL_Q[4] = {QN(0, 0), QN(1, 1), QN(1, -1), QN(2, 0)};

struct Error : std::runtime_error {
  int status;
  Error(int st, const std::string& m) : std::runtime_error(m), status(st) {}
};

#define MPSLCC_REQUIRE(cond, st, msg)                                  \
  do {                                                                 \
    if (!(cond)) throw ::mpslcc::Error((st), std::string(msg));        \
  } while (0)

enum { ST_OK = 0, ST_ARG = 1, ST_STATE = 2, ST_CUDA = 3, ST_NOMEM = 4, ST_NOCONV = 5,
       ST_TIMEOUT = 6, ST_INTERNAL = 7, ST_NUMERIC = 8 };

// A list of sectors, sorted ascending by (N, 2Sz).
struct Sectors {
  std::vector<QN> q;
  std::vector<int> d;
  int size() const { return (int)q.size(); }
  int find(const QN& x) const {
    auto it = std::lower_bound(q.begin(), q.end(), x);
    if (it == q.end() || !(*it == x)) return -1;
    return (int)(it - q.begin());
  }
  long total() const {
    long t = 0;
    for (int v : d) t += v;
    return t;
  }
};

}  // namespace mpslcc
