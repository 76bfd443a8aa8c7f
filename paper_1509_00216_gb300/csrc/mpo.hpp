// Matrix product operators of H, H0 and U (Theory section, Eq. "part" and
// the Fink partition; Implementation section, Eq. mpo).
#pragma once
#include "common.hpp"

namespace mpslcc {

// One nonzero of a site tensor: W[w_left, w_right](s_out, s_in) = val.
struct MpoEntry {
  int w0, w1;
  int so, si;
  double val;
};

// Channels of one MPO bond, ordered by quantum-number change (class).
struct MpoBond {
  int n = 0;
  std::vector<QN> dq;         // per channel: change of the left block's QN
  std::vector<int> cls;       // per channel: class id
  std::vector<int> pos;       // per channel: position inside its class
  std::vector<QN> class_dq;   // per class
  std::vector<int> class_start, class_n;
  int find_class(const QN& d) const {
    for (size_t c = 0; c < class_dq.size(); ++c)
      if (class_dq[c] == d) return (int)c;
    return -1;
  }
};

// Fusion recipe of one site tensor with an environment, for one local
// matrix element (so, si) and one target class.  Targets are channels of the
// bond being produced, sources channels of the environment's bond; positions
// are relative to the class starts.
struct FuseGroup {
  int so, si;
  int tcls, scls;
  struct Run { int t, s, n; double v; };          // t+j <- v * s+j
  struct Box { int t, nt, s, ns; std::vector<double> C; long doff = 0; };  // [nt x ns] dense
  std::vector<Run> runs;
  std::vector<Box> boxes;
};

struct MpoSite {
  std::vector<MpoEntry> e;
  std::vector<FuseGroup> lfuse;  // targets = right bond (building L')
  std::vector<FuseGroup> rfuse;  // targets = left bond (building R')
};

struct Mpo {
  int k = 0;
  std::vector<MpoBond> bond;  // k+1 bonds; bond b sits left of site b
  std::vector<MpoSite> site;
  long n_terms = 0;
  int max_bond() const {
    int m = 0;
    for (auto& b : bond) m = std::max(m, b.n);
    return m;
  }
};

enum MpoKind { MPO_H = 0, MPO_H0 = 1, MPO_U = 2, MPO_ID = 3 };

// Build the MPO of H (kind 0), H0 (1), U = H - H0 (2) or the identity (3)
// for integrals h (k x k) and V (k^4, chemists' order).  Orbitals
// [0, n_core) are core, [n_core, n_core + n_active) active, the rest virtual.
Mpo build_mpo(int k, const double* h, const double* V, int kind, int n_core, int n_active);

}  // namespace mpslcc
