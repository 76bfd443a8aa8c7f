// Block-sparse MPS machinery on the GPU: fused spaces, environments, sigma
// plans, truncation and the DMRG / LCC sweeps.
#pragma once
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <map>
#include <memory>
#include <string>

#include "common.hpp"
#include "kernels.hpp"
#include "mpo.hpp"
#include "mpslcc.h"

namespace mpslcc {

struct Ctx;

double wall_seconds();  // monotonic host clock
void cuda_check(cudaError_t e, const char* what);

// Device buffer owned by a context (stream-ordered allocation).
struct DBuf {
  Ctx* c = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { swap(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); swap(o); }
    return *this;
  }
  ~DBuf() { release(); }
  void swap(DBuf& o) noexcept {
    std::swap(c, o.c);
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
  }
  void alloc(Ctx* ctx, size_t nbytes);
  void ensure(Ctx* ctx, size_t nbytes) {
    if (bytes < nbytes) { release(); alloc(ctx, nbytes); }
  }
  void release();
  double* d() const { return (double*)p; }
};

// A fused (bond x site) or (site x bond) space: sectors and their pieces.
struct Piece { int sec, s, dim, off; };
struct Fused {
  std::vector<QN> q;
  std::vector<int> d;
  std::vector<std::vector<Piece>> pc;
  int find(const QN& x) const {
    auto it = std::lower_bound(q.begin(), q.end(), x);
    if (it == q.end() || !(*it == x)) return -1;
    return (int)(it - q.begin());
  }
  const Piece* piece(int f, int sec, int s) const {
    for (const auto& p : pc[f])
      if (p.sec == sec && p.s == s) return &p;
    return nullptr;
  }
  long total() const {
    long t = 0;
    for (int v : d) t += v;
    return t;
  }
};
Fused fuse_left(const Sectors& b, const std::vector<int>& mask);   // key = q_bond + q_s
Fused fuse_right(const std::vector<int>& mask, const Sectors& b);  // key = q_bond - q_s

// Site tensor, kept in the left-fused layout (blocks per right-bond sector,
// [dimFL x d_b] row-major) and/or the right-fused layout (blocks per
// left-bond sector, [d_a x dimFR] row-major).
struct SiteT {
  DBuf lf, rf;
  bool has_lf = false, has_rf = false;
  std::vector<long> lf_off, rf_off;
};

struct MPS {
  bool present = false;
  int k = 0;
  QN target;
  std::vector<Sectors> bond;             // k+1
  std::vector<std::vector<int>> mask;    // allowed local states per site
  std::vector<SiteT> site;
};

struct EnvPair { int ib, ik, cls, nw; long off; };
struct Env {
  bool valid = false;
  std::vector<EnvPair> pairs;
  DBuf data;
  long size = 0;
};

struct Family {
  MPS* bra = nullptr;
  MPS* ket = nullptr;
  const Mpo* mpo = nullptr;
  const DBuf* boxes = nullptr;   // device copy of the MPO's dense fusion boxes
  std::vector<Env> L, R;         // per bond (k+1)
  void reset(int k) {
    L.clear();
    R.clear();
    L.resize(k + 1);
    R.resize(k + 1);
  }
};

// L'[w] of site p (w on MPO bond p+1), on the fused spaces FL_p.
struct LeftFused {
  int p = -1;
  Fused FLb, FLk;
  std::vector<int> kb, kk;            // key sectors (indices into FLb / FLk)
  std::vector<int> kb_of, kk_of;      // FL index -> key index or -1
  struct Seg { int cls, kidx, width, nw; long koff; };
  std::vector<std::vector<Seg>> seg;  // per bra key
  std::vector<long> K, off;           // per bra key
  DBuf data;
  long size = 0;
  const Seg* find_seg(int bkey, int cls) const {
    for (const auto& s : seg[bkey])
      if (s.cls == cls) return &s;
    return nullptr;
  }
};

// R'[w] of site p (w on MPO bond p), on the fused spaces FR_p.  For a
// one-site position the right side is the environment R[p+1] itself (spaces
// = the bond's sectors, one piece each): `ext` then points at the
// environment's data, which the plan does not own.
struct RightFused {
  int p = -1;
  Fused FRb, FRk;
  std::vector<int> kb, kk, kb_of, kk_of;
  struct Stk { int kidx, cls, bidx, nw; long off; };
  std::vector<Stk> stk;
  std::map<std::pair<int, int>, int> sidx;  // (ket key, class) -> stack
  DBuf data;
  const double* ext = nullptr;
  long size = 0;
  const double* base() const { return ext ? ext : data.d(); }
};

// Fused operator of one side of two-site position l, built ahead of time
// (while the truncation at the neighbouring position runs): the right side
// R' of site l+1 during a left-to-right sweep, the left side L' of site l
// during a right-to-left sweep.  Neither depends on the sites that
// truncation changes, but both are keyed by the middle sectors of position
// l, which can change with the truncated bond: the plan uses it only when
// they did not.
struct FusedAhead {
  int l = -1;
  bool right = false;              // holds rf (else lf)
  std::vector<QN> mid_b, mid_k;    // middle sectors it was built for
  LeftFused lf;
  RightFused rf;
};

// Sigma plan at two-site position l (sites l, l+1) or, with one_site, at
// site l alone.
struct SigmaPlan {
  int l = -1;
  bool one_site = false;
  Family* fam = nullptr;
  LeftFused lf;
  RightFused rf;
  std::vector<QN> mid_b, mid_k;        // middle sectors (bra / ket)
  std::vector<long> off_b, off_k;      // local-vector offsets
  long nb = 0, nk = 0;
  std::vector<long> tt_off;            // per bra middle
  DBuf tt;
  DBuf xin;
  DBuf tasks1, tasks2;
  int n1 = 0, n2 = 0;
  long long tiles1 = 0, tiles2 = 0;
  // FP64 phase 2: per-split partial products and the segments of their
  // fixed-order sum into sigma
  DBuf ypart, segs;
  DBuf kruns;                          // K-run tables of the FP64 tasks
  int nseg = 0;
  long long seg_tiles = 0;
  double flops = 0.0;                  // algorithmic flops of one application
  // low-precision operand copies and task lists of the tensor-core path:
  // tc for TF32 / BF16, tc6 for the three-piece layout (BF16X3 and BF16X6)
  struct TcState* tc = nullptr;
  struct TcState* tc6 = nullptr;
  SigmaPlan() = default;
  SigmaPlan(const SigmaPlan&) = delete;
  SigmaPlan& operator=(const SigmaPlan&) = delete;
  ~SigmaPlan();
};

struct Stats {
  double sigma_flops = 0, sigma_seconds = 0, env_flops = 0;
  long long sigma_calls = 0, gemm_launches = 0, kernel_launches = 0;
  double last_sweep_seconds = 0, last_sweep_sigma_seconds = 0, last_sweep_sigma_flops = 0;
  long long last_sweep_sigma_calls = 0, last_sweep_kernel_launches = 0;
  int max_bond_dim = 0;
  // per-phase device time / algorithmic bytes of the sigma kernels
  double tc_phase1_s = 0, tc_phase2_s = 0, tc_phase1_bytes = 0, tc_phase2_bytes = 0;
  double f64_phase1_s = 0, f64_phase2_s = 0;
  long long tc_launches = 0;
  double tc_gemm_flops = 0;
  // host wall time per sweep stage (stream-synchronised)
  double t_plan = 0, t_trunc = 0, t_env = 0, t_solve = 0, t_rhs = 0;
  double t_fuse_left = 0, t_fuse_right = 0, t_tc_prepare = 0;
  long long ahead_used = 0, ahead_missed = 0;
  long long n_noconv = 0, n_indefinite = 0, n_j_rise = 0;
  double max_rel_residual = 0;
  long long tune_trials = 0;
  long long tc_cap_launches[4] = {0, 0, 0, 0};   // sigma launches per tile shape: cap 256 / 128 / 64, 64 on 2 CTAs/SM
};

// Solver outcome counters of the current sweep call (reset per call).
struct CallFlags {
  long long noconv = 0, indefinite = 0, j_rise = 0;
  double max_rel_residual = 0;
  void reset() { *this = CallFlags(); }
};

// Adds the wall time of a scope (after synchronising the stream) to *acc.
struct StageTimer {
  Ctx& c;
  double* acc;
  double t0;
  StageTimer(Ctx& c_, double* a);
  ~StageTimer();
};

struct Ctx {
  // live device allocations (start -> bytes), used to validate every task's
  // address range on the host before a launch
  std::map<uintptr_t, size_t> allocs;
  void check_range(const void* p, long long first, long long last, const char* what) const;
  void check_bytes(const void* p, long long nbytes, const char* what) const;

  int device = 0;
  bool host_only = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  mpslcc_opts opts{};
  std::string err;
  cusolverDnHandle_t solver = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_p0 = nullptr, ev_p1 = nullptr, ev_p2 = nullptr;

  // problem
  int k = 0, n_elec = 0, two_sz = 0;
  std::vector<double> h, V;
  int n_core = 0, n_active = 0;
  bool have_mpo = false;
  Mpo mpo[4];              // H, H0, U, identity
  DBuf boxes[4];
  MPS phi0, phi1;
  double E0 = 0, E2 = 0, E3 = 0, J = 0, ovl01 = 0, norm1 = 0, max_disc = 0;
  bool have_E0 = false, have_E2 = false, e3_valid = false, e_valid = false;
  int sweeps_done = 0;
  Stats st;
  CallFlags cf;        // of the last dmrg_reference / lcc_sweep call
  int flags = 0;       // MPSLCC_FLAG_* reported with the energies

  // families
  Family f00;   // <Phi0|H0|Phi0>
  Family f11;   // <Phi1|H0|Phi1>
  Family f10;   // <Phi1|H|Phi0>
  Family s10;   // <Phi1|Phi0>
  Family u11;   // <Phi1|U|Phi1>
  Family h11;   // <Phi1|H|Phi1>

  // higher orders (Eq. 1 for n >= 2): Phi(n) and, per order, the families of
  // its sweeps: <Phi(n)|H0|Phi(n)>, <Phi(n)|U|Phi(n-1)>, <Phi(n)|Phi0> and
  // <Phi(n)|Phi(j)> for j = 1 .. n-2
  static constexpr int MAX_ORDER = 8;
  struct OrderFamilies {
    Family a, t, s0;
    std::vector<Family> s;   // index j (1 .. n-2)
  };
  std::vector<std::unique_ptr<MPS>> phin;              // index n >= 2
  std::vector<std::unique_ptr<OrderFamilies>> ofam;     // index n >= 2
  std::vector<double> Eseries;                          // E(0 .. 2N+1), Eq. 2
  bool series_valid = false;
  MPS* phi_of(int n) {
    if (n == 0) return &phi0;
    if (n == 1) return &phi1;
    if ((int)phin.size() <= n) phin.resize(n + 1);
    if (!phin[n]) phin[n].reset(new MPS());
    return phin[n].get();
  }
  int highest_order() {
    int n = phi1.present ? 1 : 0;
    while (n >= 1 && n + 1 < (int)phin.size() && phin[n + 1] && phin[n + 1]->present) ++n;
    return n;
  }
  void clear_orders_above(int n) {   // Phi(m) for m > n and their families
    for (int m = std::max(n + 1, 2); m < (int)phin.size(); ++m) phin[m].reset();
    for (int m = std::max(n + 1, 2); m < (int)ofam.size(); ++m) ofam[m].reset();
    series_valid = false;
  }

  // scratch
  DBuf red, red_out, red_ticket, gtask, ctask;
  DBuf eig_work, eig_w, eig_info;
  static constexpr int NEIG = 8;   // concurrent eigensolver streams
  cudaStream_t eig_stream[NEIG] = {};
  cusolverDnHandle_t eig_solver[NEIG] = {};
  cudaEvent_t eig_ev[NEIG] = {}, eig_fork = nullptr;
  DBuf eig_ws[NEIG];
  DBuf scratch_a, scratch_b;
  DBuf scratch_tc, tc_conv_tasks, tc_gemm_tasks, tc_err;
  // precision of the per-site FP64 GEMM tasks (fusion, renormalisation,
  // truncation): MPSLCC_FP64, or MPSLCC_BF16X3 inside mixed-precision sweeps
  int gemm_prec = MPSLCC_FP64;
  // SMs the persistent tensor-core launches leave free (set while a
  // truncation's eigensolvers run on their side streams)
  int tc_sm_reserve = 0;

  // tile-shape autotuner of the sigma phases (tc_gemm.cu): best N-tile cap
  // per (bra, ket, operator, position, phase, sigma precision)
  struct TuneKey {
    const void *bra, *ket, *mpo;
    int l, phase, v;
    bool operator<(const TuneKey& o) const {
      if (bra != o.bra) return bra < o.bra;
      if (ket != o.ket) return ket < o.ket;
      if (mpo != o.mpo) return mpo < o.mpo;
      if (l != o.l) return l < o.l;
      if (phase != o.phase) return phase < o.phase;
      return v < o.v;
    }
  };
  struct TuneEntry {
    double bytes = 0;
    double ms[4] = {0, 0, 0, 0};
    int tried = 0, best = -1;
  };
  std::map<TuneKey, TuneEntry> tune;

  cudaStream_t s() const { return stream; }
};

// ---- engine entry points (engine.cpp / sweep.cpp) ----
void upload_boxes(Ctx& c, int which);
void run_gemms(Ctx& c, std::vector<GemmTask>& t);
void run_gemms_tc(Ctx& c, std::vector<GemmTask>& t);
// FP64 DFMA kernel or split-BF16 tensor cores, by c.gemm_prec
void run_gemm_tasks(Ctx& c, std::vector<GemmTask>& t);
void validate_gemm(const Ctx& c, const GemmTask& t);
void validate_copy(const Ctx& c, const CopyTask& t);
void run_copies(Ctx& c, std::vector<CopyTask>& t);
double dev_dot(Ctx& c, const double* x, const double* y, long n);
// x1.y1 and x2.y2 in one pass (one launch, one host round trip)
void dev_dot2(Ctx& c, const double* x1, const double* y1, const double* x2, const double* y2, long n, double* r1,
              double* r2);
// v -= (u.v) u with the coefficient kept on the device (no host round trip)
void dev_project(Ctx& c, const double* u, double* v, long n);

void ensure_lf(Ctx& c, MPS& m, int p);
void ensure_rf(Ctx& c, MPS& m, int p);
void set_site_lf(Ctx& c, MPS& m, int p, DBuf&& data);
void set_site_rf(Ctx& c, MPS& m, int p, DBuf&& data);
std::vector<long> layout_offsets(const MPS& m, int p, int layout, long* total);

void boundary_envs(Ctx& c, Family& F);
void build_left_env(Ctx& c, Family& F, int p);    // L[p+1] from L[p] and site p
void build_right_env(Ctx& c, Family& F, int p);   // R[p] from R[p+1] and site p
void make_left_fused(Ctx& c, Family& F, int p, const std::vector<QN>& kb, const std::vector<QN>& kk,
                     LeftFused& lf);
void make_right_fused(Ctx& c, Family& F, int p, const std::vector<QN>& kb, const std::vector<QN>& kk,
                      RightFused& rf);
void env_update_left(Ctx& c, Family& F, int p, const LeftFused& lf);
void env_update_right(Ctx& c, Family& F, int p, const RightFused& rf);

// Local pieces (s_out, s_in) of the fused operators of site p that can be
// non-zero, per target channel: bit 4 s_out + s_in of entry w, w a channel of
// MPO bond p+1 for the left side (L'), of bond p for the right side (R').
std::vector<uint16_t> fused_piece_masks(const Mpo& W, int p, bool left);
// Dimension of the piece of local state s in sector f of a fused space (0 if
// the sector has none); a piece of state -1 (a bare bond sector) matches any s.
int piece_dim(const Fused& F, int f, int s);
int piece_off(const Fused& F, int f, int s);

void two_site_middle(const MPS& m, int l, std::vector<QN>& mid, std::vector<long>& off, long& n);
void one_site_middle(const MPS& m, int l, std::vector<QN>& mid, std::vector<long>& off, long& n);
void make_sigma_plan(Ctx& c, Family& F, int l, SigmaPlan& P, FusedAhead* ahead = nullptr);
void make_sigma_plan1(Ctx& c, Family& F, int l, SigmaPlan& P);   // one-site plan at site l
void form_one_site(Ctx& c, MPS& m, int l, double* psi);            // site l in the one-site layout
void ensure_envs_at(Ctx& c, Family& F, int lb, int rb);             // L up to bond lb, R down to bond rb
void build_fused_ahead(Ctx& c, Family& F, int l, bool right_side, FusedAhead& A);
void sigma_apply(Ctx& c, SigmaPlan& P, const double* x, double* y, int prec);
void sigma_diag(Ctx& c, SigmaPlan& P, double* diag);
void form_two_site(Ctx& c, MPS& m, int l, double* psi);   // psi in m's middle layout
void ensure_envs(Ctx& c, Family& F, int l);

// tensor-core path (tc_gemm.cu)
void tc_prepare(Ctx& c, SigmaPlan& P, int prec);
void tc_sigma(Ctx& c, SigmaPlan& P, const double* x, double* y, int prec);
void tc_selftest(Ctx& c, int prec, int m, int n, int k, const double* A, const double* B, double* C, int mode,
                 int ksplit);
size_t tc_gemm_noalloc_max_bytes();
void tc_gemm_noalloc(int device, cudaStream_t stream, int prec, int m, int n, int k, const double* dA,
                     const double* dB, double* dC);

// sweeps (sweep.cpp)
void init_random_mps(Ctx& c, MPS& m, int M, bool frozen, unsigned long long seed);
double dmrg_reference(Ctx& c, int M0, int n_sweeps);
double lcc_sweeps(Ctx& c, int M1, int n_sweeps, int order = 1);
double lcc_window(Ctx& c, int M1, int first, int count, int dir, int order = 1);
double lcc_sweeps1(Ctx& c, int n_sweeps, int order = 1);
void compute_series(Ctx& c);
void compute_e3(Ctx& c);
void compute_energies(Ctx& c);
double reference_energy_fp64(Ctx& c);

}  // namespace mpslcc
