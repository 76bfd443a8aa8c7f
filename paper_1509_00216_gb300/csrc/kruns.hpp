// K runs of the sigma tasks (host side): the column ranges of an operand that
// hold a task's non-zero local pieces, merged into the runs a kernel reads.
// Header-only and free of CUDA, so that the host logic is tested on its own.
#pragma once
#include <algorithm>
#include <utility>
#include <vector>

namespace mpslcc {

// One run of a tensor-core task: `steps` K steps of KT columns from column kx.
struct KRun {
  long kx, steps;
};

// Runs of a tensor-core task whose non-zero columns come as ranges [a, b) of
// the operands' K extent (any order; empty ranges are dropped).  Each run
// starts on an 8-element boundary (a 16-byte TMA coordinate for 16-bit types)
// and is read in whole steps of KT columns.  A range that starts (rounded
// down to 8) before the open run's last step ends joins that run, so no
// column is read by two runs; the columns a run reads outside the ranges must
// be zero in one operand, so that they add nothing.
inline std::vector<KRun> merge_runs(std::vector<std::pair<long, long>>& r, int KT) {
  std::sort(r.begin(), r.end());
  std::vector<KRun> out;
  long de = 0;   // end of the data the open run must cover
  for (const auto& x : r) {
    if (x.second <= x.first) continue;
    const long a8 = x.first & ~7L;
    if (!out.empty() && a8 < out.back().kx + out.back().steps * KT) {
      de = std::max(de, x.second);
      out.back().steps = (de - out.back().kx + KT - 1) / KT;
    } else {
      out.push_back({a8, (x.second - a8 + KT - 1) / KT});
      de = x.second;
    }
  }
  return out;
}

// The same ranges merged exactly (sorted, disjoint, neither overlapping nor
// touching), for kernels that read element by element (the FP64 path).
inline std::vector<std::pair<long, long>> merge_exact(std::vector<std::pair<long, long>>& r) {
  std::sort(r.begin(), r.end());
  std::vector<std::pair<long, long>> m;
  for (const auto& x : r) {
    if (x.second <= x.first) continue;
    if (!m.empty() && x.first <= m.back().second) m.back().second = std::max(m.back().second, x.second);
    else m.push_back(x);
  }
  return m;
}

}  // namespace mpslcc
