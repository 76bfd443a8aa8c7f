// Environments, fused operators and the sigma vector (Implementation
// section: transition elements contracted site by site, Fig. 2; the partial
// derivative of the functional with respect to the local tensor, Fig. 3).
//
// For a two-site position (l, l+1) the effective Hamiltonian is
//   H_eff = sum_w L'_w (x) R'_w ,
//   L'_w = sum_w0 L_w0 (x) W_l[w0, w],     R'_w = sum_w2 W_l+1[w, w2] (x) R_w2 ,
// with L / R the left / right environments.  sigma = sum_w L'_w psi R'_w^T is
// evaluated per middle quantum-number sector as two stacked GEMMs:
//   phase 1:  T_w^T = R'_w psi^T           (one tall product per ket sector)
//   phase 2:  sigma = [L'_w1 | L'_w2 | ...] [T_w1 ; T_w2 ; ...]
// so the sum over operator channels sits in the K dimension of one GEMM.
#include "engine.hpp"
#include "kruns.hpp"

#include <cmath>
#include <cstring>
#include <ctime>

namespace mpslcc {

double wall_seconds() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + 1e-9 * ts.tv_nsec;
}
StageTimer::StageTimer(Ctx& c_, double* a) : c(c_), acc(a) {
  cudaStreamSynchronize(c.s());
  t0 = wall_seconds();
}
StageTimer::~StageTimer() {
  cudaStreamSynchronize(c.s());
  *acc += wall_seconds() - t0;
}

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw Error(e == cudaErrorMemoryAllocation ? ST_NOMEM : ST_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

void DBuf::alloc(Ctx* ctx, size_t nbytes) {
  c = ctx;
  bytes = nbytes;
  p = nullptr;
  if (nbytes == 0) return;
  if (ctx->opts.alloc) {
    p = ctx->opts.alloc(nbytes, ctx->opts.alloc_user);
    if (!p) throw Error(ST_NOMEM, "device allocation failed (" + std::to_string(nbytes) + " bytes)");
  } else {
    cudaError_t e = cudaMallocAsync(&p, nbytes, ctx->stream);
    if (e != cudaSuccess) {
      p = nullptr;
      bytes = 0;
      cudaGetLastError();
      throw Error(ST_NOMEM, "cudaMallocAsync of " + std::to_string(nbytes) + " bytes failed");
    }
  }
  ctx->allocs[(uintptr_t)p] = nbytes;
}

void Ctx::check_range(const void* ptr, long long first, long long last, const char* what) const {
  if (last < first) return;
  uintptr_t a = (uintptr_t)ptr + (uintptr_t)(first * 8), b = (uintptr_t)ptr + (uintptr_t)(last * 8 + 8);
  if (first < 0) a = (uintptr_t)ptr - (uintptr_t)(-first * 8);
  auto it = allocs.upper_bound(a);
  bool ok = false;
  if (it != allocs.begin()) {
    --it;
    ok = a >= it->first && b <= it->first + it->second;
  }
  if (!ok) throw Error(ST_INTERNAL, std::string("device access out of bounds in ") + what);
}

void Ctx::check_bytes(const void* ptr, long long nbytes, const char* what) const {
  if (nbytes <= 0) return;
  uintptr_t a = (uintptr_t)ptr, b = a + (uintptr_t)nbytes;
  auto it = allocs.upper_bound(a);
  bool ok = false;
  if (it != allocs.begin()) {
    --it;
    ok = a >= it->first && b <= it->first + it->second;
  }
  if (!ok) throw Error(ST_INTERNAL, std::string("device access out of bounds in ") + what);
}

void DBuf::release() {
  if (p && c) c->allocs.erase((uintptr_t)p);
  if (p && c) {
    if (c->opts.free) c->opts.free(p, bytes, c->opts.alloc_user);
    else if (c->stream || !c->own_stream) cudaFreeAsync(p, c->stream);
    else cudaFree(p);   // the context's own stream is gone (teardown): a synchronous free
  }
  p = nullptr;
  bytes = 0;
}

Fused fuse_left(const Sectors& b, const std::vector<int>& mask) {
  std::map<QN, std::vector<Piece>> m;
  for (int s : mask)
    for (int i = 0; i < b.size(); ++i) m[b.q[i] + LOCAL_Q[s]].push_back({i, s, b.d[i], 0});
  Fused f;
  for (auto& kv : m) {
    int off = 0;
    for (auto& p : kv.second) { p.off = off; off += p.dim; }
    f.q.push_back(kv.first);
    f.d.push_back(off);
    f.pc.push_back(kv.second);
  }
  return f;
}

Fused fuse_right(const std::vector<int>& mask, const Sectors& b) {
  std::map<QN, std::vector<Piece>> m;
  for (int s : mask)
    for (int i = 0; i < b.size(); ++i) m[b.q[i] - LOCAL_Q[s]].push_back({i, s, b.d[i], 0});
  Fused f;
  for (auto& kv : m) {
    int off = 0;
    for (auto& p : kv.second) { p.off = off; off += p.dim; }
    f.q.push_back(kv.first);
    f.d.push_back(off);
    f.pc.push_back(kv.second);
  }
  return f;
}

// ---------------------------------------------------------------------------
// task launch helpers
// ---------------------------------------------------------------------------
static long long span(int rows, int cols, long long ld) {
  return (rows <= 0 || cols <= 0) ? -1 : (long long)(rows - 1) * ld + (cols - 1);
}

void validate_gemm(const Ctx& c, const GemmTask& t) {
  if (t.m <= 0 || t.n <= 0 || t.batch <= 0) return;
  bool ta = t.flags & GEMM_TA, tb = t.flags & GEMM_TB;
  long long ea = ta ? span(t.k, t.m, t.lda) : span(t.m, t.k, t.lda);
  long long eb = tb ? span(t.n, t.k, t.ldb) : span(t.k, t.n, t.ldb);
  long long ec = span(t.m, t.n, t.ldc);
  if (t.k > 0) {
    c.check_range(t.A, 0, ea + (long long)(t.batch - 1) * t.sA, "gemm A");
    c.check_range(t.B, 0, eb + (long long)(t.batch - 1) * t.sB, "gemm B");
  }
  const long long ek = (t.ksplit > 1 && t.sK > 0) ? (long long)(t.ksplit - 1) * t.sK : 0;
  c.check_range(t.C, 0, ec + (long long)(t.batch - 1) * t.sC + ek, "gemm C");
  if ((!ta && t.lda < t.k) || (ta && t.lda < t.m) || (!tb && t.ldb < t.n) || (tb && t.ldb < t.k) || t.ldc < t.n)
    throw Error(ST_INTERNAL, "gemm leading dimension too small");
}

void validate_copy(const Ctx& c, const CopyTask& t) {
  if (t.rows <= 0 || t.cols <= 0 || t.batch <= 0) return;
  c.check_range(t.src, 0, span(t.rows, t.cols, t.src_ld) + (long long)(t.batch - 1) * t.s_src, "copy src");
  c.check_range(t.dst, 0, span(t.rows, t.cols, t.dst_ld) + (long long)(t.batch - 1) * t.s_dst, "copy dst");
}

void run_gemms(Ctx& c, std::vector<GemmTask>& t) {
  if (t.empty()) return;
  for (const auto& x : t) validate_gemm(c, x);
  long long tiles = plan_gemm_tiles(t.data(), (int)t.size());
  if (tiles == 0) return;
  size_t bytes = t.size() * sizeof(GemmTask);
  c.gtask.ensure(&c, bytes);
  cuda_check(cudaMemcpyAsync(c.gtask.p, t.data(), bytes, cudaMemcpyHostToDevice, c.s()), "upload gemm tasks");
  launch_gemm_f64((const GemmTask*)c.gtask.p, (int)t.size(), tiles, c.s());
  cuda_check(cudaGetLastError(), "gemm_f64 launch");
  c.st.gemm_launches++;
  c.st.kernel_launches++;
}

void run_gemm_tasks(Ctx& c, std::vector<GemmTask>& t) {
  if (c.gemm_prec == MPSLCC_FP64) run_gemms(c, t);
  else run_gemms_tc(c, t);
}

void run_copies(Ctx& c, std::vector<CopyTask>& t) {
  if (t.empty()) return;
  for (const auto& x : t) validate_copy(c, x);
  long long tiles = plan_copy_tiles(t.data(), (int)t.size());
  if (tiles == 0) return;
  size_t bytes = t.size() * sizeof(CopyTask);
  c.ctask.ensure(&c, bytes);
  cuda_check(cudaMemcpyAsync(c.ctask.p, t.data(), bytes, cudaMemcpyHostToDevice, c.s()), "upload copy tasks");
  launch_copy_f64((const CopyTask*)c.ctask.p, (int)t.size(), tiles, c.s());
  cuda_check(cudaGetLastError(), "copy launch");
  c.st.kernel_launches++;
}

static unsigned int* dot_ticket(Ctx& c) {
  if (!c.red_ticket.p) {
    c.red_ticket.alloc(&c, 256);
    cuda_check(cudaMemsetAsync(c.red_ticket.p, 0, 256, c.s()), "dot ticket");
  }
  c.red.ensure(&c, 4096 * sizeof(double));
  c.red_out.ensure(&c, 256 * sizeof(double));
  return (unsigned int*)c.red_ticket.p;
}

double dev_dot(Ctx& c, const double* x, const double* y, long n) {
  if (n <= 0) return 0.0;
  unsigned int* tk = dot_ticket(c);
  launch_dot_fused(x, y, nullptr, nullptr, n, c.red_out.d(), c.red.d(), tk, c.s());
  c.st.kernel_launches++;
  double r = 0;
  cuda_check(cudaMemcpyAsync(&r, c.red_out.p, sizeof(double), cudaMemcpyDeviceToHost, c.s()), "dot d2h");
  cuda_check(cudaStreamSynchronize(c.s()), "dot sync");
  return r;
}

void dev_dot2(Ctx& c, const double* x1, const double* y1, const double* x2, const double* y2, long n, double* r1,
              double* r2) {
  *r1 = *r2 = 0.0;
  if (n <= 0) return;
  unsigned int* tk = dot_ticket(c);
  launch_dot_fused(x1, y1, x2, y2, n, c.red_out.d(), c.red.d(), tk, c.s());
  c.st.kernel_launches++;
  double r[2] = {0, 0};
  cuda_check(cudaMemcpyAsync(r, c.red_out.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.s()), "dot d2h");
  cuda_check(cudaStreamSynchronize(c.s()), "dot sync");
  *r1 = r[0];
  *r2 = r[1];
}

void dev_project(Ctx& c, const double* u, double* v, long n) {
  if (n <= 0) return;
  unsigned int* tk = dot_ticket(c);
  double* a = c.red_out.d() + 8;   // consumed by the next launch on the stream
  launch_dot_fused(u, v, nullptr, nullptr, n, a, c.red.d(), tk, c.s());
  launch_axpy_dev(n, a, -1.0, u, v, c.s());
  c.st.kernel_launches += 2;
}

static GemmTask gemm(const double* A, const double* B, double* C, int m, int n, int k, int lda, int ldb, int ldc,
                     int flags = 0, int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0,
                     double alpha = 1.0, double beta = 0.0) {
  GemmTask t;
  std::memset(&t, 0, sizeof(t));
  t.A = A; t.B = B; t.C = C;
  t.m = m; t.n = n; t.k = k;
  t.lda = lda; t.ldb = ldb; t.ldc = ldc;
  t.flags = flags;
  t.batch = batch;
  t.sA = sA; t.sB = sB; t.sC = sC;
  t.alpha = alpha; t.beta = beta;
  t.ksplit = 1;
  return t;
}

static CopyTask copyt(const double* src, double* dst, int rows, int cols, int src_ld, int dst_ld, int batch = 1,
                      long long ss = 0, long long sd = 0, double alpha = 1.0, int acc = 0) {
  CopyTask t;
  std::memset(&t, 0, sizeof(t));
  t.src = src; t.dst = dst;
  t.rows = rows; t.cols = cols; t.src_ld = src_ld; t.dst_ld = dst_ld;
  t.batch = batch; t.s_src = ss; t.s_dst = sd;
  t.alpha = alpha; t.accumulate = acc;
  return t;
}

void upload_boxes(Ctx& c, int which) {
  Mpo& W = c.mpo[which];
  long tot = 0;
  for (auto& st : W.site) {
    for (auto& g : st.lfuse) for (auto& b : g.boxes) tot += (long)b.C.size();
    for (auto& g : st.rfuse) for (auto& b : g.boxes) tot += (long)b.C.size();
  }
  std::vector<double> host((size_t)std::max(tot, 1L));
  long off = 0;
  for (auto& st : W.site) {
    for (auto* grp : {&st.lfuse, &st.rfuse})
      for (auto& g : *grp)
        for (auto& b : g.boxes) {
          b.doff = off;
          std::copy(b.C.begin(), b.C.end(), host.begin() + off);
          off += (long)b.C.size();
        }
  }
  c.boxes[which].release();
  c.boxes[which].alloc(&c, host.size() * sizeof(double));
  cuda_check(cudaMemcpyAsync(c.boxes[which].p, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice,
                             c.s()),
             "upload MPO boxes");
  cuda_check(cudaStreamSynchronize(c.s()), "upload MPO boxes sync");
}

// ---------------------------------------------------------------------------
// site tensors
// ---------------------------------------------------------------------------
std::vector<long> layout_offsets(const MPS& m, int p, int layout, long* total) {
  std::vector<long> off;
  long tot = 0;
  if (layout == 0) {
    Fused FL = fuse_left(m.bond[p], m.mask[p]);
    const Sectors& b = m.bond[p + 1];
    for (int j = 0; j < b.size(); ++j) {
      int f = FL.find(b.q[j]);
      off.push_back(tot);
      tot += (long)(f < 0 ? 0 : FL.d[f]) * b.d[j];
    }
  } else {
    Fused FR = fuse_right(m.mask[p], m.bond[p + 1]);
    const Sectors& a = m.bond[p];
    for (int i = 0; i < a.size(); ++i) {
      int f = FR.find(a.q[i]);
      off.push_back(tot);
      tot += (long)a.d[i] * (f < 0 ? 0 : FR.d[f]);
    }
  }
  if (total) *total = tot;
  return off;
}

static void convert_site(Ctx& c, MPS& m, int p, bool to_rf) {
  SiteT& S = m.site[p];
  Fused FL = fuse_left(m.bond[p], m.mask[p]);
  Fused FR = fuse_right(m.mask[p], m.bond[p + 1]);
  long tl = 0, tr = 0;
  std::vector<long> lo = layout_offsets(m, p, 0, &tl), ro = layout_offsets(m, p, 1, &tr);
  DBuf& dst = to_rf ? S.rf : S.lf;
  dst.release();
  dst.alloc(&c, std::max(to_rf ? tr : tl, 1L) * sizeof(double));
  cuda_check(cudaMemsetAsync(dst.p, 0, std::max(to_rf ? tr : tl, 1L) * sizeof(double), c.s()), "memset site");
  std::vector<CopyTask> t;
  const Sectors& a = m.bond[p];
  const Sectors& b = m.bond[p + 1];
  for (int ia = 0; ia < a.size(); ++ia)
    for (int s : m.mask[p]) {
      int ib = b.find(a.q[ia] + LOCAL_Q[s]);
      if (ib < 0) continue;
      int fl = FL.find(b.q[ib]);
      int fr = FR.find(a.q[ia]);
      const Piece* pl = FL.piece(fl, ia, s);
      const Piece* pr = FR.piece(fr, ib, s);
      if (!pl || !pr) continue;
      const double* lptr = S.lf.d() + lo[ib] + (long)pl->off * b.d[ib];
      const double* rptr = S.rf.d() + ro[ia] + pr->off;
      int ldl = b.d[ib], ldr = FR.d[fr];
      if (to_rf) t.push_back(copyt(lptr, (double*)rptr, a.d[ia], b.d[ib], ldl, ldr));
      else t.push_back(copyt(rptr, (double*)lptr, a.d[ia], b.d[ib], ldr, ldl));
    }
  run_copies(c, t);
  if (to_rf) { S.rf_off = ro; S.has_rf = true; }
  else { S.lf_off = lo; S.has_lf = true; }
}

void ensure_lf(Ctx& c, MPS& m, int p) {
  if (m.site[p].has_lf) return;
  MPSLCC_REQUIRE(m.site[p].has_rf, ST_STATE, "site tensor missing");
  convert_site(c, m, p, false);
}
void ensure_rf(Ctx& c, MPS& m, int p) {
  if (m.site[p].has_rf) return;
  MPSLCC_REQUIRE(m.site[p].has_lf, ST_STATE, "site tensor missing");
  convert_site(c, m, p, true);
}
void set_site_lf(Ctx& c, MPS& m, int p, DBuf&& data) {
  SiteT& S = m.site[p];
  S.lf = std::move(data);
  S.lf_off = layout_offsets(m, p, 0, nullptr);
  S.has_lf = true;
  S.rf.release();
  S.has_rf = false;
}
void set_site_rf(Ctx& c, MPS& m, int p, DBuf&& data) {
  SiteT& S = m.site[p];
  S.rf = std::move(data);
  S.rf_off = layout_offsets(m, p, 1, nullptr);
  S.has_rf = true;
  S.lf.release();
  S.has_lf = false;
}

// ---------------------------------------------------------------------------
// environments
// ---------------------------------------------------------------------------
void boundary_envs(Ctx& c, Family& F) {
  int k = F.bra->k;
  F.reset(k);
  const Mpo& W = *F.mpo;
  MPSLCC_REQUIRE(W.bond[0].n == 1 && W.bond[k].n == 1, ST_INTERNAL, "MPO boundary bonds must have one channel");
  double one = 1.0;
  for (int side = 0; side < 2; ++side) {
    Env& E = side == 0 ? F.L[0] : F.R[k];
    E.pairs = {EnvPair{0, 0, 0, 1, 0}};
    E.size = 1;
    E.data.alloc(&c, sizeof(double));
    cuda_check(cudaMemcpyAsync(E.data.p, &one, sizeof(double), cudaMemcpyHostToDevice, c.s()), "boundary env");
    cuda_check(cudaStreamSynchronize(c.s()), "boundary env sync");
    E.valid = true;
  }
}

std::vector<uint16_t> fused_piece_masks(const Mpo& W, int p, bool left) {
  const MpoBond& b = W.bond[left ? p + 1 : p];
  std::vector<uint16_t> m((size_t)b.n, 0);
  for (const auto& e : W.site[p].e) m[left ? e.w1 : e.w0] |= (uint16_t)(1u << (4 * e.so + e.si));
  return m;
}

int piece_dim(const Fused& F, int f, int s) {
  for (const auto& p : F.pc[f])
    if (p.s == s || p.s < 0) return p.dim;
  return 0;
}

int piece_off(const Fused& F, int f, int s) {
  for (const auto& p : F.pc[f])
    if (p.s == s || p.s < 0) return p.off;
  return 0;
}

static std::vector<int> class_list(const MpoBond& b) {
  std::vector<int> v(b.class_dq.size());
  for (size_t i = 0; i < v.size(); ++i) v[i] = (int)i;
  return v;
}

static void set_keys(const Fused& F, const std::vector<QN>& keys, std::vector<int>& kv, std::vector<int>& of) {
  kv.clear();
  of.assign(F.q.size(), -1);
  for (const QN& q : keys) {
    int f = F.find(q);
    MPSLCC_REQUIRE(f >= 0, ST_INTERNAL, "key sector missing from fused space");
    of[f] = (int)kv.size();
    kv.push_back(f);
  }
}

static bool has_state(const std::vector<int>& mask, int s) {
  return std::find(mask.begin(), mask.end(), s) != mask.end();
}

void make_left_fused(Ctx& c, Family& F, int p, const std::vector<QN>& kbq, const std::vector<QN>& kkq,
                     LeftFused& lf) {
  MPS& B = *F.bra;
  MPS& Kt = *F.ket;
  const Mpo& W = *F.mpo;
  const Env& E = F.L[p];
  MPSLCC_REQUIRE(E.valid, ST_INTERNAL, "left environment missing");
  lf.p = p;
  lf.FLb = fuse_left(B.bond[p], B.mask[p]);
  lf.FLk = fuse_left(Kt.bond[p], Kt.mask[p]);
  set_keys(lf.FLb, kbq, lf.kb, lf.kb_of);
  set_keys(lf.FLk, kkq, lf.kk, lf.kk_of);
  const MpoBond& mb = W.bond[p + 1];
  lf.seg.assign(lf.kb.size(), {});
  lf.K.assign(lf.kb.size(), 0);
  lf.off.assign(lf.kb.size(), 0);
  lf.size = 0;
  for (size_t bi = 0; bi < lf.kb.size(); ++bi) {
    QN qb = lf.FLb.q[lf.kb[bi]];
    long K = 0;
    for (int cl : class_list(mb)) {
      int fk = lf.FLk.find(qb - mb.class_dq[cl]);
      if (fk < 0 || lf.kk_of[fk] < 0) continue;
      LeftFused::Seg sg{cl, lf.kk_of[fk], lf.FLk.d[fk], mb.class_n[cl], K};
      lf.seg[bi].push_back(sg);
      K += (long)sg.nw * sg.width;
    }
    lf.K[bi] = K;
    lf.off[bi] = lf.size;
    lf.size += (long)lf.FLb.d[lf.kb[bi]] * K;
  }
  lf.data.release();
  lf.data.alloc(&c, std::max(lf.size, 1L) * sizeof(double));
  cuda_check(cudaMemsetAsync(lf.data.p, 0, std::max(lf.size, 1L) * sizeof(double), c.s()), "memset L'");
  std::vector<GemmTask> gt;
  std::vector<CopyTask> ct;
  const double* boxes = F.boxes->d();
  for (const auto& g : W.site[p].lfuse) {
    if (!has_state(B.mask[p], g.so) || !has_state(Kt.mask[p], g.si)) continue;
    for (const auto& e : E.pairs) {
      if (e.cls != g.scls) continue;
      int fb = lf.FLb.find(B.bond[p].q[e.ib] + LOCAL_Q[g.so]);
      int fk = lf.FLk.find(Kt.bond[p].q[e.ik] + LOCAL_Q[g.si]);
      if (fb < 0 || fk < 0) continue;
      int bk = lf.kb_of[fb], kk = lf.kk_of[fk];
      if (bk < 0 || kk < 0) continue;
      const LeftFused::Seg* sg = lf.find_seg(bk, g.tcls);
      if (!sg) continue;
      MPSLCC_REQUIRE(sg->kidx == kk, ST_INTERNAL, "L' segment mismatch");
      const Piece* pb = lf.FLb.piece(fb, e.ib, g.so);
      const Piece* pk = lf.FLk.piece(fk, e.ik, g.si);
      int drow = B.bond[p].d[e.ib], dcol = Kt.bond[p].d[e.ik];
      long blk = (long)drow * dcol;
      long K = lf.K[bk];
      double* base = lf.data.d() + lf.off[bk] + (long)pb->off * K + sg->koff + pk->off;
      const double* src = E.data.d() + e.off;
      for (const auto& r : g.runs)
        ct.push_back(copyt(src + (long)r.s * blk, base + (long)r.t * sg->width, drow, dcol, dcol, (int)K, r.n, blk,
                           sg->width, r.v));
      for (const auto& bx : g.boxes)
        gt.push_back(gemm(boxes + bx.doff, src + (long)bx.s * blk, base + (long)bx.t * sg->width, bx.nt, dcol, bx.ns,
                          bx.ns, (int)blk, sg->width, 0, drow, 0, dcol, K));
    }
  }
  run_copies(c, ct);
  run_gemm_tasks(c, gt);
}

void make_right_fused(Ctx& c, Family& F, int p, const std::vector<QN>& kbq, const std::vector<QN>& kkq,
                      RightFused& rf) {
  MPS& B = *F.bra;
  MPS& Kt = *F.ket;
  const Mpo& W = *F.mpo;
  const Env& E = F.R[p + 1];
  MPSLCC_REQUIRE(E.valid, ST_INTERNAL, "right environment missing");
  rf.p = p;
  rf.FRb = fuse_right(B.mask[p], B.bond[p + 1]);
  rf.FRk = fuse_right(Kt.mask[p], Kt.bond[p + 1]);
  set_keys(rf.FRb, kbq, rf.kb, rf.kb_of);
  set_keys(rf.FRk, kkq, rf.kk, rf.kk_of);
  const MpoBond& mb = W.bond[p];
  rf.stk.clear();
  rf.sidx.clear();
  rf.size = 0;
  for (size_t ki = 0; ki < rf.kk.size(); ++ki) {
    int fk = rf.kk[ki];
    QN q = rf.FRk.q[fk];
    for (int cl : class_list(mb)) {
      int fb = rf.FRb.find(q + mb.class_dq[cl]);
      if (fb < 0 || rf.kb_of[fb] < 0) continue;
      RightFused::Stk s{(int)ki, cl, rf.kb_of[fb], mb.class_n[cl], rf.size};
      rf.sidx[{(int)ki, cl}] = (int)rf.stk.size();
      rf.stk.push_back(s);
      rf.size += (long)s.nw * rf.FRb.d[fb] * rf.FRk.d[fk];
    }
  }
  rf.data.release();
  rf.data.alloc(&c, std::max(rf.size, 1L) * sizeof(double));
  cuda_check(cudaMemsetAsync(rf.data.p, 0, std::max(rf.size, 1L) * sizeof(double), c.s()), "memset R'");
  std::vector<GemmTask> gt;
  std::vector<CopyTask> ct;
  const double* boxes = F.boxes->d();
  for (const auto& g : W.site[p].rfuse) {
    if (!has_state(B.mask[p], g.so) || !has_state(Kt.mask[p], g.si)) continue;
    for (const auto& e : E.pairs) {
      if (e.cls != g.scls) continue;
      int fb = rf.FRb.find(B.bond[p + 1].q[e.ib] - LOCAL_Q[g.so]);
      int fk = rf.FRk.find(Kt.bond[p + 1].q[e.ik] - LOCAL_Q[g.si]);
      if (fb < 0 || fk < 0) continue;
      int bk = rf.kb_of[fb], kk = rf.kk_of[fk];
      if (bk < 0 || kk < 0) continue;
      auto it = rf.sidx.find({kk, g.tcls});
      if (it == rf.sidx.end()) continue;
      const RightFused::Stk& S = rf.stk[it->second];
      MPSLCC_REQUIRE(S.bidx == bk, ST_INTERNAL, "R' stack mismatch");
      const Piece* pb = rf.FRb.piece(fb, e.ib, g.so);
      const Piece* pk = rf.FRk.piece(fk, e.ik, g.si);
      int drow = B.bond[p + 1].d[e.ib], dcol = Kt.bond[p + 1].d[e.ik];
      long blk = (long)drow * dcol;
      int Wd = rf.FRk.d[fk];
      long blkS = (long)rf.FRb.d[fb] * Wd;
      double* base = rf.data.d() + S.off + (long)pb->off * Wd + pk->off;
      const double* src = E.data.d() + e.off;
      for (const auto& r : g.runs)
        ct.push_back(copyt(src + (long)r.s * blk, base + (long)r.t * blkS, drow, dcol, dcol, Wd, r.n, blk, blkS, r.v));
      for (const auto& bx : g.boxes)
        gt.push_back(gemm(boxes + bx.doff, src + (long)bx.s * blk, base + (long)bx.t * blkS, bx.nt, dcol, bx.ns,
                          bx.ns, (int)blk, (int)blkS, 0, drow, 0, dcol, Wd));
    }
  }
  run_copies(c, ct);
  run_gemm_tasks(c, gt);
}

void env_update_left(Ctx& c, Family& F, int p, const LeftFused& lf) {
  MPS& B = *F.bra;
  MPS& Kt = *F.ket;
  ensure_lf(c, B, p);
  ensure_lf(c, Kt, p);
  const MpoBond& mb = F.mpo->bond[p + 1];
  Env ne;
  const Sectors& bb = B.bond[p + 1];
  const Sectors& bk = Kt.bond[p + 1];
  struct Job { int ib, ik, fb, fk, bkey; const LeftFused::Seg* sg; long xoff, eoff; };
  std::vector<Job> jobs;
  long xsize = 0;
  for (int ib = 0; ib < bb.size(); ++ib) {
    int fb = lf.FLb.find(bb.q[ib]);
    if (fb < 0 || lf.kb_of[fb] < 0) continue;
    for (int ik = 0; ik < bk.size(); ++ik) {
      int fk = lf.FLk.find(bk.q[ik]);
      if (fk < 0 || lf.kk_of[fk] < 0) continue;
      int cl = mb.find_class(bb.q[ib] - bk.q[ik]);
      if (cl < 0) continue;
      const LeftFused::Seg* sg = lf.find_seg(lf.kb_of[fb], cl);
      if (!sg || sg->kidx != lf.kk_of[fk]) continue;
      EnvPair pr{ib, ik, cl, sg->nw, ne.size};
      ne.pairs.push_back(pr);
      jobs.push_back({ib, ik, fb, fk, lf.kb_of[fb], sg, xsize, ne.size});
      ne.size += (long)sg->nw * bb.d[ib] * bk.d[ik];
      xsize += (long)sg->nw * lf.FLb.d[fb] * bk.d[ik];
    }
  }
  ne.data.alloc(&c, std::max(ne.size, 1L) * sizeof(double));
  c.scratch_a.ensure(&c, std::max(xsize, 1L) * sizeof(double));
  double* X = c.scratch_a.d();
  // X_w = L'_w A_k over the non-zero local pieces of L'_w only: per run of
  // channels with equal piece masks and per bra local state so, one product
  // per ket state si the pieces reach.  The k-th si of a row block adds
  // (beta = 1) in launch k, so no two tasks of one launch write the same
  // rows; rows that no piece reaches stay zero.
  cuda_check(cudaMemsetAsync(X, 0, std::max(xsize, 1L) * sizeof(double), c.s()), "env X zero");
  const std::vector<uint16_t> mL = fused_piece_masks(*F.mpo, p, true);
  std::vector<std::vector<GemmTask>> tx(4);
  std::vector<GemmTask> ty;
  for (const auto& j : jobs) {
    const int rows = lf.FLb.d[j.fb];
    const int dk = bk.d[j.ik], db = bb.d[j.ib];
    const long K = lf.K[j.bkey];
    const int width = j.sg->width, c0 = mb.class_start[j.sg->cls];
    const double* Lp = lf.data.d() + lf.off[j.bkey] + j.sg->koff;
    const double* Ak = Kt.site[p].lf.d() + Kt.site[p].lf_off[j.ik];
    const double* Ab = B.site[p].lf.d() + B.site[p].lf_off[j.ib];
    for (int w = 0; w < j.sg->nw;) {
      const uint16_t m = mL[c0 + w];
      int w1 = w + 1;
      while (w1 < j.sg->nw && mL[c0 + w1] == m) ++w1;
      for (int so = 0; so < 4; ++so) {
        const int dso = piece_dim(lf.FLb, j.fb, so);
        if (dso == 0) continue;
        const long ro = piece_off(lf.FLb, j.fb, so);
        int k = 0;
        for (int si = 0; si < 4; ++si) {
          if (!((m >> (4 * so + si)) & 1)) continue;
          const int dsi = piece_dim(lf.FLk, j.fk, si);
          if (dsi == 0) continue;
          const long co = piece_off(lf.FLk, j.fk, si);
          tx[k].push_back(gemm(Lp + ro * K + (long)w * width + co, Ak + co * dk, X + j.xoff + (long)w * rows * dk + ro * dk,
                               dso, dk, dsi, (int)K, dk, dk, 0, w1 - w, width, 0, (long long)rows * dk, 1.0,
                               k > 0 ? 1.0 : 0.0));
          c.st.env_flops += 2.0 * (w1 - w) * (double)dso * dk * dsi;
          ++k;
        }
      }
      w = w1;
    }
    ty.push_back(gemm(Ab, X + j.xoff, ne.data.d() + j.eoff, db, dk, rows, db, dk, dk, GEMM_TA, j.sg->nw, 0,
                      (long long)rows * dk, (long long)db * dk));
    c.st.env_flops += 2.0 * j.sg->nw * (double)db * dk * rows;
  }
  for (auto& t : tx) run_gemm_tasks(c, t);
  run_gemm_tasks(c, ty);
  ne.valid = true;
  F.L[p + 1] = std::move(ne);
}

void env_update_right(Ctx& c, Family& F, int p, const RightFused& rf) {
  MPS& B = *F.bra;
  MPS& Kt = *F.ket;
  ensure_rf(c, B, p);
  ensure_rf(c, Kt, p);
  const MpoBond& mb = F.mpo->bond[p];
  Env ne;
  const Sectors& bb = B.bond[p];
  const Sectors& bk = Kt.bond[p];
  struct Job { int ib, ik, fb, fk; const RightFused::Stk* S; long yoff, eoff; };
  std::vector<Job> jobs;
  long ysize = 0;
  for (int ib = 0; ib < bb.size(); ++ib) {
    int fb = rf.FRb.find(bb.q[ib]);
    if (fb < 0 || rf.kb_of[fb] < 0) continue;
    for (int ik = 0; ik < bk.size(); ++ik) {
      int fk = rf.FRk.find(bk.q[ik]);
      if (fk < 0 || rf.kk_of[fk] < 0) continue;
      int cl = mb.find_class(bb.q[ib] - bk.q[ik]);
      if (cl < 0) continue;
      auto it = rf.sidx.find({rf.kk_of[fk], cl});
      if (it == rf.sidx.end()) continue;
      const RightFused::Stk* S = &rf.stk[it->second];
      if (S->bidx != rf.kb_of[fb]) continue;
      ne.pairs.push_back(EnvPair{ib, ik, cl, S->nw, ne.size});
      jobs.push_back({ib, ik, fb, fk, S, ysize, ne.size});
      ne.size += (long)S->nw * bb.d[ib] * bk.d[ik];
      ysize += (long)S->nw * rf.FRb.d[fb] * bk.d[ik];
    }
  }
  ne.data.alloc(&c, std::max(ne.size, 1L) * sizeof(double));
  c.scratch_a.ensure(&c, std::max(ysize, 1L) * sizeof(double));
  double* Y = c.scratch_a.d();
  // Y_w = R'_w B_k^T over the non-zero local pieces of R'_w only (as for the
  // left side); a one-site position's right side (the environment itself,
  // one piece per sector) keeps the dense product
  const bool pieces = !rf.ext;
  if (pieces) cuda_check(cudaMemsetAsync(Y, 0, std::max(ysize, 1L) * sizeof(double), c.s()), "env Y zero");
  const std::vector<uint16_t> mR = pieces ? fused_piece_masks(*F.mpo, p, false) : std::vector<uint16_t>();
  std::vector<std::vector<GemmTask>> ty(4);
  std::vector<GemmTask> tz;
  for (const auto& j : jobs) {
    const int rb = rf.FRb.d[j.fb], rk = rf.FRk.d[j.fk];
    const int dk = bk.d[j.ik], db = bb.d[j.ib];
    const long blkS = (long)rb * rk;
    const double* Rp = rf.base() + j.S->off;
    const double* Bk = Kt.site[p].rf.d() + Kt.site[p].rf_off[j.ik];
    const double* Bb = B.site[p].rf.d() + B.site[p].rf_off[j.ib];
    if (!pieces) {
      ty[0].push_back(gemm(Rp, Bk, Y + j.yoff, rb, dk, rk, rk, rk, dk, GEMM_TB, j.S->nw, blkS, 0, (long long)rb * dk));
      c.st.env_flops += 2.0 * j.S->nw * (double)rb * dk * rk;
    } else {
      const int c0 = mb.class_start[j.S->cls];
      for (int w = 0; w < j.S->nw;) {
        const uint16_t m = mR[c0 + w];
        int w1 = w + 1;
        while (w1 < j.S->nw && mR[c0 + w1] == m) ++w1;
        for (int so = 0; so < 4; ++so) {
          const int dso = piece_dim(rf.FRb, j.fb, so);
          if (dso == 0) continue;
          const long ro = piece_off(rf.FRb, j.fb, so);
          int k = 0;
          for (int si = 0; si < 4; ++si) {
            if (!((m >> (4 * so + si)) & 1)) continue;
            const int dsi = piece_dim(rf.FRk, j.fk, si);
            if (dsi == 0) continue;
            const long co = piece_off(rf.FRk, j.fk, si);
            ty[k].push_back(gemm(Rp + ((long)w * rb + ro) * rk + co, Bk + co, Y + j.yoff + (long)w * rb * dk + ro * dk,
                                 dso, dk, dsi, rk, rk, dk, GEMM_TB, w1 - w, blkS, 0, (long long)rb * dk, 1.0,
                                 k > 0 ? 1.0 : 0.0));
            c.st.env_flops += 2.0 * (w1 - w) * (double)dso * dk * dsi;
            ++k;
          }
        }
        w = w1;
      }
    }
    tz.push_back(gemm(Bb, Y + j.yoff, ne.data.d() + j.eoff, db, dk, rb, rb, dk, dk, 0, j.S->nw, 0,
                      (long long)rb * dk, (long long)db * dk));
    c.st.env_flops += 2.0 * j.S->nw * (double)db * dk * rb;
  }
  for (auto& t : ty) run_gemm_tasks(c, t);
  run_gemm_tasks(c, tz);
  ne.valid = true;
  F.R[p] = std::move(ne);
}

void build_left_env(Ctx& c, Family& F, int p) {
  ensure_lf(c, *F.bra, p);
  ensure_lf(c, *F.ket, p);
  LeftFused lf;
  Fused FLb = fuse_left(F.bra->bond[p], F.bra->mask[p]);
  Fused FLk = fuse_left(F.ket->bond[p], F.ket->mask[p]);
  std::vector<QN> kb, kk;
  for (const QN& q : F.bra->bond[p + 1].q)
    if (FLb.find(q) >= 0) kb.push_back(q);
  for (const QN& q : F.ket->bond[p + 1].q)
    if (FLk.find(q) >= 0) kk.push_back(q);
  make_left_fused(c, F, p, kb, kk, lf);
  env_update_left(c, F, p, lf);
}

void build_right_env(Ctx& c, Family& F, int p) {
  ensure_rf(c, *F.bra, p);
  ensure_rf(c, *F.ket, p);
  RightFused rf;
  Fused FRb = fuse_right(F.bra->mask[p], F.bra->bond[p + 1]);
  Fused FRk = fuse_right(F.ket->mask[p], F.ket->bond[p + 1]);
  std::vector<QN> kb, kk;
  for (const QN& q : F.bra->bond[p].q)
    if (FRb.find(q) >= 0) kb.push_back(q);
  for (const QN& q : F.ket->bond[p].q)
    if (FRk.find(q) >= 0) kk.push_back(q);
  make_right_fused(c, F, p, kb, kk, rf);
  env_update_right(c, F, p, rf);
}

void ensure_envs_at(Ctx& c, Family& F, int lb, int rb) {
  int k = F.bra->k;
  if (F.L.empty() || !F.L[0].valid || !F.R[k].valid) boundary_envs(c, F);
  int b = lb;
  while (b > 0 && !F.L[b].valid) --b;
  for (int p = b; p < lb; ++p) build_left_env(c, F, p);
  int e = rb;
  while (e < k && !F.R[e].valid) ++e;
  for (int p = e - 1; p >= rb; --p) build_right_env(c, F, p);
}

void ensure_envs(Ctx& c, Family& F, int l) { ensure_envs_at(c, F, l, l + 2); }

// ---------------------------------------------------------------------------
// two-site sigma
// ---------------------------------------------------------------------------
void two_site_middle(const MPS& m, int l, std::vector<QN>& mid, std::vector<long>& off, long& n) {
  Fused FL = fuse_left(m.bond[l], m.mask[l]);
  Fused FR = fuse_right(m.mask[l + 1], m.bond[l + 2]);
  mid.clear();
  off.clear();
  n = 0;
  for (size_t i = 0; i < FL.q.size(); ++i) {
    int j = FR.find(FL.q[i]);
    if (j < 0 || FL.d[i] == 0 || FR.d[j] == 0) continue;
    mid.push_back(FL.q[i]);
    off.push_back(n);
    n += (long)FL.d[i] * FR.d[j];
  }
}

// One-site middle sectors of site l: the sectors q of bond l+1 reachable
// from bond l; the local vector is site l in its left-fused layout, one
// row-major block [dimFL(q) x d(q)] per sector.
void one_site_middle(const MPS& m, int l, std::vector<QN>& mid, std::vector<long>& off, long& n) {
  Fused FL = fuse_left(m.bond[l], m.mask[l]);
  const Sectors& b = m.bond[l + 1];
  mid.clear();
  off.clear();
  n = 0;
  for (int j = 0; j < b.size(); ++j) {
    int f = FL.find(b.q[j]);
    if (f < 0 || FL.d[f] == 0 || b.d[j] == 0) continue;
    mid.push_back(b.q[j]);
    off.push_back(n);
    n += (long)FL.d[f] * b.d[j];
  }
}

void form_one_site(Ctx& c, MPS& m, int l, double* psi) {
  ensure_lf(c, m, l);
  std::vector<QN> mid;
  std::vector<long> off;
  long n;
  one_site_middle(m, l, mid, off, n);
  long tot = 0;
  layout_offsets(m, l, 0, &tot);
  MPSLCC_REQUIRE(tot == n, ST_INTERNAL, "one-site layout differs from the left-fused site layout");
  if (n > 0)
    cuda_check(cudaMemcpyAsync(psi, m.site[l].lf.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.s()),
               "one-site vector");
}

// The right side of a one-site position l: the environment R[l+1] on the
// bond's sectors, its blocks used in place as the phase-1 stacks.
static void make_right_env(Ctx& c, Family& F, int l, const std::vector<QN>& kbq, const std::vector<QN>& kkq,
                           RightFused& rf) {
  MPS& B = *F.bra;
  MPS& Kt = *F.ket;
  const Env& E = F.R[l + 1];
  MPSLCC_REQUIRE(E.valid, ST_INTERNAL, "right environment missing");
  auto bond_space = [](const Sectors& s) {
    Fused f;
    for (int i = 0; i < s.size(); ++i) {
      f.q.push_back(s.q[i]);
      f.d.push_back(s.d[i]);
      f.pc.push_back({Piece{i, -1, s.d[i], 0}});
    }
    return f;
  };
  rf.p = l;
  rf.FRb = bond_space(B.bond[l + 1]);
  rf.FRk = bond_space(Kt.bond[l + 1]);
  set_keys(rf.FRb, kbq, rf.kb, rf.kb_of);
  set_keys(rf.FRk, kkq, rf.kk, rf.kk_of);
  std::map<std::pair<int, int>, const EnvPair*> pairs;
  for (const auto& e : E.pairs) pairs[{e.ib, e.ik}] = &e;
  const MpoBond& mb = F.mpo->bond[l + 1];
  rf.stk.clear();
  rf.sidx.clear();
  for (size_t ki = 0; ki < rf.kk.size(); ++ki) {
    const int ik = rf.kk[ki];
    for (size_t cl = 0; cl < mb.class_dq.size(); ++cl) {
      const int ib = rf.FRb.find(rf.FRk.q[ik] + mb.class_dq[cl]);
      if (ib < 0 || rf.kb_of[ib] < 0) continue;
      auto it = pairs.find({ib, ik});
      if (it == pairs.end()) continue;
      MPSLCC_REQUIRE(it->second->cls == (int)cl && it->second->nw == mb.class_n[cl], ST_INTERNAL,
                     "environment pair class mismatch");
      RightFused::Stk st{(int)ki, (int)cl, rf.kb_of[ib], it->second->nw, it->second->off};
      rf.sidx[{(int)ki, (int)cl}] = (int)rf.stk.size();
      rf.stk.push_back(st);
    }
  }
  rf.data.release();
  rf.ext = E.data.d();
  rf.size = E.size;
}

void build_fused_ahead(Ctx& c, Family& F, int l, bool right_side, FusedAhead& A) {
  std::vector<long> ob, ok;
  long nb = 0, nk = 0;
  A.l = -1;
  two_site_middle(*F.bra, l, A.mid_b, ob, nb);
  two_site_middle(*F.ket, l, A.mid_k, ok, nk);
  if (right_side) make_right_fused(c, F, l + 1, A.mid_b, A.mid_k, A.rf);
  else make_left_fused(c, F, l, A.mid_b, A.mid_k, A.lf);
  A.l = l;
  A.right = right_side;
}

static void finish_sigma_plan(Ctx& c, SigmaPlan& P);

void make_sigma_plan(Ctx& c, Family& F, int l, SigmaPlan& P, FusedAhead* ahead) {
  ensure_envs(c, F, l);
  P.l = l;
  P.fam = &F;
  two_site_middle(*F.bra, l, P.mid_b, P.off_b, P.nb);
  two_site_middle(*F.ket, l, P.mid_k, P.off_k, P.nk);
  const bool match = ahead && ahead->l == l && ahead->mid_b == P.mid_b && ahead->mid_k == P.mid_k;
  const bool have_l = match && !ahead->right;
  const bool have_r = match && ahead->right;
  if (ahead && ahead->l == l) (match ? c.st.ahead_used : c.st.ahead_missed)++;
  if (have_l) {
    P.lf = std::move(ahead->lf);
  } else {
    StageTimer tm(c, &c.st.t_fuse_left);
    make_left_fused(c, F, l, P.mid_b, P.mid_k, P.lf);
  }
  if (have_r) {
    P.rf = std::move(ahead->rf);
  } else {
    StageTimer tm(c, &c.st.t_fuse_right);
    make_right_fused(c, F, l + 1, P.mid_b, P.mid_k, P.rf);
  }
  if (ahead) ahead->l = -1;
  finish_sigma_plan(c, P);
}

void make_sigma_plan1(Ctx& c, Family& F, int l, SigmaPlan& P) {
  ensure_envs_at(c, F, l, l + 1);
  P.l = l;
  P.fam = &F;
  P.one_site = true;
  one_site_middle(*F.bra, l, P.mid_b, P.off_b, P.nb);
  one_site_middle(*F.ket, l, P.mid_k, P.off_k, P.nk);
  {
    StageTimer tm(c, &c.st.t_fuse_left);
    make_left_fused(c, F, l, P.mid_b, P.mid_k, P.lf);
  }
  make_right_env(c, F, l, P.mid_b, P.mid_k, P.rf);
  finish_sigma_plan(c, P);
}

// Intermediate buffers and the task lists of both sigma phases of a plan
// whose fused left operator and right operator are in place.
static void finish_sigma_plan(Ctx& c, SigmaPlan& P) {
  const LeftFused& lf = P.lf;
  const RightFused& rf = P.rf;
  P.tt_off.assign(P.mid_b.size(), 0);
  long tts = 0;
  for (size_t bi = 0; bi < P.mid_b.size(); ++bi) {
    P.tt_off[bi] = tts;
    tts += (long)rf.FRb.d[rf.kb[bi]] * lf.K[bi];
  }
  P.tt.release();
  P.tt.alloc(&c, std::max(tts, 1L) * sizeof(double));
  // phase 1 writes only the rows of T that a channel's R' reaches; the rest
  // stay zero for every product of the plan
  cuda_check(cudaMemsetAsync(P.tt.p, 0, std::max(tts, 1L) * sizeof(double), c.s()), "T zero");
  P.xin.release();
  P.xin.alloc(&c, std::max(P.nk, 1L) * sizeof(double));
  std::vector<GemmTask> t1, t2;
  // Algorithmic flops: a channel's fused block is non-zero only on the local
  // pieces (s_out, s_in) its site tensor reaches, so both phases count the
  // block products piece by piece (and both the FP64 and the tensor-core
  // tasks multiply only those pieces).
  const Mpo& W = *P.fam->mpo;
  const std::vector<uint16_t> mL = fused_piece_masks(W, lf.p, true);
  const std::vector<uint16_t> mR = rf.ext ? std::vector<uint16_t>() : fused_piece_masks(W, rf.p, false);
  auto piece_flops = [](const Fused& Fb, int fb, const Fused& Fk, int fk, uint16_t mask, double other) {
    double f = 0;
    for (int b = 0; b < 16; ++b)
      if (mask >> b & 1) f += 2.0 * piece_dim(Fb, fb, b >> 2) * piece_dim(Fk, fk, b & 3) * other;
    return f;
  };
  double fl = 0;
  for (const auto& S : rf.stk) {
    const int fb = rf.kb[S.bidx], fk = rf.kk[S.kidx];
    const double dl = lf.FLk.d[lf.kk[S.kidx]];
    if (rf.ext) {
      fl += 2.0 * S.nw * (double)rf.FRb.d[fb] * rf.FRk.d[fk] * dl;
      continue;
    }
    const int c0 = W.bond[rf.p].class_start[S.cls];
    for (int w = 0; w < S.nw; ++w) fl += piece_flops(rf.FRb, fb, rf.FRk, fk, mR[c0 + w], dl);
  }
  for (size_t bi = 0; bi < P.mid_b.size(); ++bi) {
    const int fb = lf.kb[bi];
    const double dr = rf.FRb.d[rf.kb[bi]];
    for (const auto& sg : lf.seg[bi]) {
      const int c0 = W.bond[lf.p + 1].class_start[sg.cls], fk = lf.kk[sg.kidx];
      for (int w = 0; w < sg.nw; ++w) fl += piece_flops(lf.FLb, fb, lf.FLk, fk, mL[c0 + w], dr);
    }
  }
  // Phase 1: T_w^T = R'_w psi^T per unit — the rows of one R' stack with bra
  // local state so for a run of channels whose pieces (so, .) agree, batched
  // over those channels — summing only over the ket pieces the unit reaches
  // (K runs).  A one-site position's right side is one piece per sector.
  // Every task's run table is {operand column, virtual start} pairs and a
  // sentinel; a task whose runs cover its K extent densely has none.
  std::vector<std::vector<int>> rt1, rt2;
  auto add_runs = [](std::vector<std::pair<long, long>>& rg, int kext, std::vector<int>& tab) {
    const std::vector<std::pair<long, long>> m = merge_exact(rg);   // sorted, disjoint [start, end)
    tab.clear();
    int v = 0;
    for (const auto& x : m) {
      MPSLCC_REQUIRE(x.first >= 0 && x.second <= kext, ST_INTERNAL, "K run outside the operand");
      tab.push_back((int)x.first);
      tab.push_back(v);
      v += (int)(x.second - x.first);
    }
    tab.push_back(0);
    tab.push_back(v);
    return v;
  };
  const int nso = rf.ext ? 1 : 4;
  for (const auto& S : rf.stk) {
    const int ki = S.kidx, bi = S.bidx;
    const LeftFused::Seg* sg = lf.find_seg(bi, S.cls);
    MPSLCC_REQUIRE(sg && sg->kidx == ki, ST_INTERNAL, "sigma plan: segment/stack mismatch");
    const int fb = rf.kb[bi], fk = rf.kk[ki];
    const int dFRk = rf.FRk.d[fk], dFRb = rf.FRb.d[fb], dFLk = lf.FLk.d[lf.kk[ki]];
    const long K = lf.K[bi];
    const int c0 = rf.ext ? 0 : W.bond[rf.p].class_start[S.cls];
    for (int so = 0; so < nso; ++so) {
      const int d = piece_dim(rf.FRb, fb, so);
      if (d == 0) continue;
      const int boff = piece_off(rf.FRb, fb, so);
      for (int w = 0; w < S.nw;) {
        const int in = rf.ext ? 1 : (mR[c0 + w] >> (4 * so)) & 15;
        int w1 = w + 1;
        while (w1 < S.nw && (rf.ext ? 1 : (mR[c0 + w1] >> (4 * so)) & 15) == in) ++w1;
        if (in) {
          std::vector<std::pair<long, long>> rg;
          for (int sn = 0; sn < 4; ++sn)
            if (in >> sn & 1) {
              const int o = piece_off(rf.FRk, fk, sn);
              rg.push_back({o, o + piece_dim(rf.FRk, fk, sn)});
            }
          std::vector<int> tab;
          const int kv = add_runs(rg, dFRk, tab);
          if (kv > 0) {
            GemmTask t = gemm(rf.base() + S.off + ((long)w * dFRb + boff) * dFRk, P.xin.d() + P.off_k[ki],
                              P.tt.d() + P.tt_off[bi] + (long)boff * K + sg->koff + (long)w * sg->width, d, dFLk, dFRk,
                              dFRk, dFRk, (int)K, GEMM_TB, w1 - w, (long long)dFRb * dFRk, 0, sg->width);
            if (!(tab.size() == 4 && tab[0] == 0 && kv == dFRk)) {
              t.kv = kv;
              t.nkr = (int)tab.size() / 2 - 1;
              rt1.push_back(std::move(tab));
            } else {
              rt1.push_back({});
            }
            t1.push_back(t);
          }
        }
        w = w1;
      }
    }
  }
  // phase 2: sigma rows of one (middle sector, bra local state) = Lcat Tt^T
  // over the K runs of the L' pieces those rows reach, split over K when the
  // row blocks alone give too few tiles.  Every split stores its partial at
  // its own offset of `ypart`; sigma_apply sums them in a fixed order (no
  // atomics: results are reproducible bit for bit)
  struct U2 { int bi, so, d, boff, kv; std::vector<int> tab; };
  std::vector<U2> u2;
  long long base_tiles = 0;
  for (size_t bi = 0; bi < P.mid_b.size(); ++bi) {
    const int fb = lf.kb[bi], dFRb = rf.FRb.d[rf.kb[bi]];
    for (int so = 0; so < 4; ++so) {
      const int d = piece_dim(lf.FLb, fb, so);
      if (d == 0) continue;
      std::vector<std::pair<long, long>> rg;
      for (const auto& sg : lf.seg[bi]) {
        const int c0 = W.bond[lf.p + 1].class_start[sg.cls], fk = lf.kk[sg.kidx];
        for (int w = 0; w < sg.nw; ++w)
          for (int sn = 0; sn < 4; ++sn)
            if ((mL[c0 + w] >> (4 * so + sn)) & 1) {
              const int o = (int)(sg.koff + (long)w * sg.width + piece_off(lf.FLk, fk, sn));
              rg.push_back({o, o + piece_dim(lf.FLk, fk, sn)});
            }
      }
      U2 u{(int)bi, so, d, piece_off(lf.FLb, fb, so), 0, {}};
      u.kv = add_runs(rg, (int)lf.K[bi], u.tab);
      base_tiles += (long long)((d + 63) / 64) * ((dFRb + 63) / 64);
      u2.push_back(std::move(u));
    }
  }
  const long long target = 152LL * 6;
  std::vector<SplitSeg> segs;
  std::vector<int> ksv(u2.size(), 0);
  long poff = 0;
  for (size_t i = 0; i < u2.size(); ++i) {
    const U2& u = u2[i];
    const int dFRb = rf.FRb.d[rf.kb[u.bi]];
    SplitSeg sg;
    std::memset(&sg, 0, sizeof(sg));
    sg.out_off = P.off_b[u.bi] + (long long)u.boff * dFRb;
    sg.m = u.d;
    sg.n = dFRb;
    sg.ldp = dFRb;
    sg.sstride = (long long)u.d * dFRb;
    if (u.kv > 0) {  // no run: no operator channel reaches these rows, they stay zero
      int ks = 1;
      if (base_tiles < target) {
        long long f = (target + base_tiles - 1) / std::max(1LL, base_tiles);
        ks = (int)std::max(1LL, std::min(f, (long long)(u.kv / 256)));
      }
      ksv[i] = ks;
      sg.nsplit = ks;
      sg.part_off = poff;
      poff += (long)ks * sg.sstride;
    }
    segs.push_back(sg);
  }
  P.ypart.release();
  P.ypart.alloc(&c, std::max(poff, 1L) * sizeof(double));
  for (size_t i = 0; i < u2.size(); ++i) {
    if (ksv[i] == 0) continue;
    U2& u = u2[i];
    const long K = lf.K[u.bi];
    const int dFRb = rf.FRb.d[rf.kb[u.bi]];
    GemmTask t = gemm(lf.data.d() + lf.off[u.bi] + (long)u.boff * K, P.tt.d() + P.tt_off[u.bi],
                      P.ypart.d() + segs[i].part_off, u.d, dFRb, (int)K, (int)K, (int)K, dFRb, GEMM_TB);
    t.ksplit = ksv[i];
    t.sK = segs[i].sstride;
    t.kv = u.kv;
    t.nkr = (int)u.tab.size() / 2 - 1;
    rt2.push_back(std::move(u.tab));
    t2.push_back(t);
  }
  // run tables of both phases in one device buffer
  std::vector<int> tab;
  std::vector<long> at1(t1.size(), -1), at2(t2.size(), -1);
  for (size_t i = 0; i < t1.size(); ++i)
    if (!rt1[i].empty()) { at1[i] = (long)tab.size(); tab.insert(tab.end(), rt1[i].begin(), rt1[i].end()); }
  for (size_t i = 0; i < t2.size(); ++i) { at2[i] = (long)tab.size(); tab.insert(tab.end(), rt2[i].begin(), rt2[i].end()); }
  P.kruns.release();
  P.kruns.alloc(&c, std::max<size_t>(tab.size(), 4) * sizeof(int));
  if (!tab.empty())
    cuda_check(cudaMemcpyAsync(P.kruns.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, c.s()),
               "upload K runs");
  for (size_t i = 0; i < t1.size(); ++i)
    if (at1[i] >= 0) t1[i].kr = (const int*)P.kruns.p + at1[i];
  for (size_t i = 0; i < t2.size(); ++i) t2[i].kr = (const int*)P.kruns.p + at2[i];
  P.nseg = (int)segs.size();
  P.seg_tiles = plan_split_tiles(segs.data(), P.nseg);
  P.segs.release();
  P.segs.alloc(&c, std::max<size_t>(segs.size(), 1) * sizeof(SplitSeg));
  if (!segs.empty())
    cuda_check(cudaMemcpyAsync(P.segs.p, segs.data(), segs.size() * sizeof(SplitSeg), cudaMemcpyHostToDevice, c.s()),
               "upload split segments");
  for (const auto& x : t1) validate_gemm(c, x);
  for (const auto& x : t2) validate_gemm(c, x);
  P.flops = fl;
  P.n1 = (int)t1.size();
  P.n2 = (int)t2.size();
  P.tiles1 = t1.empty() ? 0 : plan_gemm_tiles(t1.data(), P.n1);
  P.tiles2 = t2.empty() ? 0 : plan_gemm_tiles(t2.data(), P.n2);
  P.tasks1.release();
  P.tasks2.release();
  P.tasks1.alloc(&c, std::max<size_t>(t1.size(), 1) * sizeof(GemmTask));
  P.tasks2.alloc(&c, std::max<size_t>(t2.size(), 1) * sizeof(GemmTask));
  if (!t1.empty())
    cuda_check(cudaMemcpyAsync(P.tasks1.p, t1.data(), t1.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, c.s()),
               "upload sigma tasks");
  if (!t2.empty())
    cuda_check(cudaMemcpyAsync(P.tasks2.p, t2.data(), t2.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, c.s()),
               "upload sigma tasks");
  cuda_check(cudaStreamSynchronize(c.s()), "sigma plan sync");
}

void sigma_apply(Ctx& c, SigmaPlan& P, const double* x, double* y, int prec) {
  if (prec != MPSLCC_FP64) {
    tc_sigma(c, P, x, y, prec);
    return;
  }
  if (P.nk > 0)
    cuda_check(cudaMemcpyAsync(P.xin.p, x, P.nk * sizeof(double), cudaMemcpyDeviceToDevice, c.s()), "sigma in");
  cudaEventRecord(c.ev_p0, c.s());
  launch_gemm_f64((const GemmTask*)P.tasks1.p, P.n1, P.tiles1, c.s());
  cudaEventRecord(c.ev_p1, c.s());
  launch_gemm_f64((const GemmTask*)P.tasks2.p, P.n2, P.tiles2, c.s());
  cudaEventRecord(c.ev_p2, c.s());
  launch_splitk_reduce_f64((const SplitSeg*)P.segs.p, P.nseg, P.seg_tiles, P.ypart.d(), y, c.s());
  cuda_check(cudaGetLastError(), "sigma launch");
  c.st.kernel_launches += 3;
  c.st.gemm_launches += 2;
  c.st.sigma_calls++;
  c.st.sigma_flops += P.flops;
  cuda_check(cudaEventSynchronize(c.ev_p2), "sigma phase sync");
  float m1 = 0, m2 = 0;
  cudaEventElapsedTime(&m1, c.ev_p0, c.ev_p1);
  cudaEventElapsedTime(&m2, c.ev_p1, c.ev_p2);
  c.st.f64_phase1_s += m1 * 1e-3;
  c.st.f64_phase2_s += m2 * 1e-3;
}

void sigma_diag(Ctx& c, SigmaPlan& P, double* diag) {
  MPSLCC_REQUIRE(P.fam->bra == P.fam->ket, ST_INTERNAL, "diagonal needs bra == ket");
  cuda_check(cudaMemsetAsync(diag, 0, std::max(P.nb, 1L) * sizeof(double), c.s()), "diag zero");
  const LeftFused& lf = P.lf;
  const RightFused& rf = P.rf;
  const MpoBond& mb = P.fam->mpo->bond[P.l + 1];
  int c0 = mb.find_class(QN(0, 0));
  if (c0 < 0) return;
  int nw = mb.class_n[c0];
  long need = 0;
  for (size_t bi = 0; bi < P.mid_b.size(); ++bi)
    need += (long)nw * (lf.FLb.d[lf.kb[bi]] + rf.FRb.d[rf.kb[bi]]);
  c.scratch_b.ensure(&c, std::max(need, 1L) * sizeof(double));
  std::vector<GatherTask> gt;
  std::vector<GemmTask> mt;
  long off = 0;
  int maxe = 0;
  for (size_t bi = 0; bi < P.mid_b.size(); ++bi) {
    const LeftFused::Seg* sg = lf.find_seg((int)bi, c0);
    auto it = rf.sidx.find({(int)bi, c0});
    if (!sg || it == rf.sidx.end()) continue;
    const RightFused::Stk& S = rf.stk[it->second];
    int dl = lf.FLb.d[lf.kb[bi]], dr = rf.FRb.d[rf.kb[bi]];
    long K = lf.K[bi];
    double* DL = c.scratch_b.d() + off;
    double* DR = DL + (long)nw * dl;
    off += (long)nw * (dl + dr);
    gt.push_back({lf.data.d() + lf.off[bi] + sg->koff, DL, nw, dl, (long long)sg->width, (long long)K + 1});
    gt.push_back({rf.base() + S.off, DR, nw, dr, (long long)dr * rf.FRk.d[rf.kk[bi]],
                  (long long)rf.FRk.d[rf.kk[bi]] + 1});
    maxe = std::max(maxe, nw * std::max(dl, dr));
    mt.push_back(gemm(DL, DR, diag + P.off_b[bi], dl, dr, nw, dl, dr, dr, GEMM_TA));
  }
  for (const auto& g : gt) {
    c.check_range(g.src, 0, (long long)(g.nw - 1) * g.sw + (long long)(g.n - 1) * g.sr, "gather src");
    c.check_range(g.dst, 0, (long long)g.nw * g.n - 1, "gather dst");
  }
  if (!gt.empty()) {
    c.scratch_a.ensure(&c, gt.size() * sizeof(GatherTask));
    cuda_check(cudaMemcpyAsync(c.scratch_a.p, gt.data(), gt.size() * sizeof(GatherTask), cudaMemcpyHostToDevice,
                               c.s()),
               "upload gather");
    launch_gather((const GatherTask*)c.scratch_a.p, (int)gt.size(), maxe, c.s());
    cuda_check(cudaGetLastError(), "gather launch");
    cuda_check(cudaStreamSynchronize(c.s()), "gather sync");
  }
  run_gemm_tasks(c, mt);
}

void form_two_site(Ctx& c, MPS& m, int l, double* psi) {
  ensure_lf(c, m, l);
  ensure_rf(c, m, l + 1);
  std::vector<QN> mid;
  std::vector<long> off;
  long n;
  two_site_middle(m, l, mid, off, n);
  cuda_check(cudaMemsetAsync(psi, 0, std::max(n, 1L) * sizeof(double), c.s()), "psi zero");
  Fused FL = fuse_left(m.bond[l], m.mask[l]);
  Fused FR = fuse_right(m.mask[l + 1], m.bond[l + 2]);
  std::vector<GemmTask> t;
  for (size_t i = 0; i < mid.size(); ++i) {
    int j = m.bond[l + 1].find(mid[i]);
    if (j < 0) continue;
    int dl = FL.d[FL.find(mid[i])], dr = FR.d[FR.find(mid[i])], dj = m.bond[l + 1].d[j];
    t.push_back(gemm(m.site[l].lf.d() + m.site[l].lf_off[j], m.site[l + 1].rf.d() + m.site[l + 1].rf_off[j],
                     psi + off[i], dl, dr, dj, dj, dr, dr));
  }
  run_gemm_tasks(c, t);
}

}  // namespace mpslcc
