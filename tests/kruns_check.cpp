// Randomised check of the K-run merging of the sigma tasks (kruns.hpp): for
// ranges [a, b) of non-zero columns in any order, overlapping, touching or
// empty, every column of a range must be read by exactly one run, runs must
// start on 8-column boundaries and read whole steps, and the exact merge must
// return the union of the ranges as sorted, disjoint, non-touching ranges.
// Exits 0 when every case holds.
#include <cstdio>
#include <random>
#include <set>
#include <vector>

#include "kruns.hpp"

using mpslcc::KRun;

static int fail(const char* what, int trial) {
  std::printf("FAIL trial %d: %s\n", trial, what);
  return 1;
}

int main() {
  std::mt19937_64 rng(20260);
  int bad = 0;
  for (int trial = 0; trial < 4000; ++trial) {
    const int KT = trial % 2 ? 32 : 64;
    const int nr = 1 + (int)(rng() % 40);
    const long span = 64 + (long)(rng() % 4000);
    std::vector<std::pair<long, long>> r;
    for (int i = 0; i < nr; ++i) {
      const long a = (long)(rng() % span);
      long len = (long)(rng() % 300);
      if (rng() % 7 == 0) len = 0;                     // empty range
      r.push_back({a, a + len});
      if (rng() % 5 == 0 && len > 0) r.push_back({a + len, a + len + 1 + (long)(rng() % 20)});  // touching
    }
    std::set<long> cols;
    for (const auto& x : r)
      for (long c = x.first; c < x.second; ++c) cols.insert(c);
    std::vector<std::pair<long, long>> r2 = r;
    const std::vector<KRun> runs = mpslcc::merge_runs(r, KT);
    long prev_end = -1;
    for (const KRun& k : runs) {
      if (k.kx % 8 != 0) bad += fail("run start not on an 8-column boundary", trial);
      if (k.steps < 1) bad += fail("empty run", trial);
      if (k.kx < prev_end) bad += fail("read windows overlap (a column read twice)", trial);
      prev_end = k.kx + k.steps * KT;
      bool any = false;
      for (long c = k.kx; c < k.kx + k.steps * KT && !any; ++c) any = cols.count(c) > 0;
      if (!any) bad += fail("run reads no column of any range", trial);
    }
    for (long c : cols) {
      int hits = 0;
      for (const KRun& k : runs) hits += (c >= k.kx && c < k.kx + k.steps * KT);
      if (hits != 1) {
        bad += fail("a column of a range is not read exactly once", trial);
        break;
      }
    }
    const std::vector<std::pair<long, long>> m = mpslcc::merge_exact(r2);
    std::set<long> mc;
    for (size_t i = 0; i < m.size(); ++i) {
      if (m[i].second <= m[i].first) bad += fail("empty exact range", trial);
      if (i > 0 && m[i].first <= m[i - 1].second) bad += fail("exact ranges overlap or touch", trial);
      for (long c = m[i].first; c < m[i].second; ++c) mc.insert(c);
    }
    if (mc != cols) bad += fail("exact merge is not the union of the ranges", trial);
    if (bad > 20) break;
  }
  if (bad) return 1;
  std::printf("ok\n");
  return 0;
}
