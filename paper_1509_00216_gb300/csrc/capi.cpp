// C ABI of the MPS-LCC library (declared in include/mpslcc.h).  No exception
// crosses this boundary: every entry point catches, records the message and
// returns a status code.
#include <cmath>
#include <cstring>

#include "engine.hpp"

using namespace mpslcc;

struct mpslcc_ctx {
  Ctx c;
};

namespace {

template <class F>
mpslcc_status guard(mpslcc_ctx* ctx, F&& f) {
  if (!ctx) return MPSLCC_E_ARG;
  try {
    f(ctx->c);
    ctx->c.err.clear();
    return MPSLCC_OK;
  } catch (const Error& e) {
    ctx->c.err = e.what();
    if (!ctx->c.host_only) cudaGetLastError();
    return (mpslcc_status)e.status;
  } catch (const std::bad_alloc&) {
    ctx->c.err = "host allocation failed";
    return MPSLCC_E_NOMEM;
  } catch (const std::exception& e) {
    ctx->c.err = e.what();
    return MPSLCC_E_INTERNAL;
  }
}

void need_device(Ctx& c) { MPSLCC_REQUIRE(!c.host_only, ST_STATE, "host-only context cannot run kernels"); }

void require_finite(const double* x, size_t n, const char* what) {
  for (size_t i = 0; i < n; ++i)
    MPSLCC_REQUIRE(std::isfinite(x[i]), ST_ARG, std::string(what) + " contains a non-finite value");
}

// A sweep call whose local solves stopped at max_iter above their tolerance
// still completes and keeps its results; it reports MPSLCC_E_NOCONV.
mpslcc_status noconv_status(mpslcc_ctx* ctx, mpslcc_status st) {
  if (st != MPSLCC_OK || ctx->c.cf.noconv == 0) return st;
  ctx->c.err = std::to_string(ctx->c.cf.noconv) +
               " local solve(s) stopped at max_iter above their tolerance; the states and energies were kept";
  return MPSLCC_E_NOCONV;
}

void reset_families(Ctx& c) {
  for (Family* F : {&c.f00, &c.f11, &c.f10, &c.s10, &c.u11, &c.h11}) {
    F->L.clear();
    F->R.clear();
    F->bra = F->ket = nullptr;
  }
  c.ofam.clear();
  c.series_valid = false;
}

void build_partition_mpos(Ctx& c) {
  c.mpo[MPO_H0] = build_mpo(c.k, c.h.data(), c.V.data(), MPO_H0, c.n_core, c.n_active);
  c.mpo[MPO_U] = build_mpo(c.k, c.h.data(), c.V.data(), MPO_U, c.n_core, c.n_active);
  if (!c.host_only) {
    upload_boxes(c, MPO_H0);
    upload_boxes(c, MPO_U);
  }
}

Family& family_for(Ctx& c, int op) {
  MPS* bra = nullptr;
  MPS* ket = nullptr;
  int mpo = 0;
  Family* F = nullptr;
  switch (op) {
    case MPSLCC_OP_H0_11: F = &c.f11; bra = ket = &c.phi1; mpo = MPO_H0; break;
    case MPSLCC_OP_H0_00: F = &c.f00; bra = ket = &c.phi0; mpo = MPO_H0; break;
    case MPSLCC_OP_H_10: F = &c.f10; bra = &c.phi1; ket = &c.phi0; mpo = MPO_H; break;
    case MPSLCC_OP_U_11: F = &c.u11; bra = ket = &c.phi1; mpo = MPO_U; break;
    case MPSLCC_OP_S_10: F = &c.s10; bra = &c.phi1; ket = &c.phi0; mpo = MPO_ID; break;
    case MPSLCC_OP_H_11: F = &c.h11; bra = ket = &c.phi1; mpo = MPO_H; break;
    default: throw Error(ST_ARG, "unknown operator");
  }
  MPSLCC_REQUIRE(bra->present && ket->present, ST_STATE, "MPS for this operator not present");
  if (F->bra != bra || F->ket != ket || F->mpo != &c.mpo[mpo] || F->L.empty()) {
    F->bra = bra;
    F->ket = ket;
    F->mpo = &c.mpo[mpo];
    F->boxes = &c.boxes[mpo];
    boundary_envs(c, *F);
  }
  return *F;
}

}  // namespace

extern "C" {

void mpslcc_default_opts(mpslcc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->stream = nullptr;
  o->prec = MPSLCC_FP64;
  o->tol = 1e-10;
  o->max_iter = 200;
  o->solver = 2;
  o->davidson_max_subspace = 24;
  o->refine_steps = 4;
  o->init_guess = 0;
  o->seed = 7;
  o->verbose = 0;
  o->autotune = 1;
}

mpslcc_status mpslcc_create(mpslcc_ctx** out, const mpslcc_opts* opts) {
  if (!out) return MPSLCC_E_ARG;
  *out = nullptr;
  mpslcc_ctx* ctx = new (std::nothrow) mpslcc_ctx();
  if (!ctx) return MPSLCC_E_NOMEM;
  if (opts) ctx->c.opts = *opts;
  else mpslcc_default_opts(&ctx->c.opts);
  mpslcc_status st = guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(c.opts.prec >= MPSLCC_FP64 && c.opts.prec <= MPSLCC_BF16X6, ST_ARG, "opts.prec out of range");
    MPSLCC_REQUIRE(c.opts.init_guess == 0 || c.opts.init_guess == 1, ST_ARG, "opts.init_guess must be 0 or 1");
    c.device = c.opts.device;
    c.host_only = c.device < 0;
    if (c.host_only) return;
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    if (c.opts.stream) {
      c.stream = (cudaStream_t)c.opts.stream;
      c.own_stream = false;
    } else {
      cuda_check(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "stream create");
      c.own_stream = true;
    }
    MPSLCC_REQUIRE(cusolverDnCreate(&c.solver) == CUSOLVER_STATUS_SUCCESS, ST_CUDA, "cusolverDnCreate failed");
    cusolverDnSetStream(c.solver, c.stream);
    for (cudaEvent_t* e : {&c.ev0, &c.ev1, &c.ev_p0, &c.ev_p1, &c.ev_p2}) cuda_check(cudaEventCreate(e), "event");
  });
  if (st != MPSLCC_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return MPSLCC_OK;
}

mpslcc_status mpslcc_destroy(mpslcc_ctx* ctx) {
  if (!ctx) return MPSLCC_E_ARG;
  Ctx& c = ctx->c;
  if (!c.host_only) {
    cudaSetDevice(c.device);
    // every member that owns device memory is released here, while the
    // stream its frees are ordered on still exists
    reset_families(c);
    c.phi0 = MPS();
    c.phi1 = MPS();
    c.phin.clear();
    c.ofam.clear();
    for (auto& b : c.boxes) b.release();
    for (DBuf* b : {&c.red, &c.red_out, &c.red_ticket, &c.gtask, &c.ctask, &c.eig_work, &c.eig_w, &c.eig_info, &c.scratch_a,
                    &c.scratch_b, &c.scratch_tc, &c.tc_conv_tasks, &c.tc_gemm_tasks, &c.tc_err})
      b->release();
    for (int s = 0; s < Ctx::NEIG; ++s) c.eig_ws[s].release();
    cudaStreamSynchronize(c.stream);
    for (int s = 0; s < Ctx::NEIG; ++s) {
      if (c.eig_solver[s]) cusolverDnDestroy(c.eig_solver[s]);
      if (c.eig_stream[s]) cudaStreamDestroy(c.eig_stream[s]);
      if (c.eig_ev[s]) cudaEventDestroy(c.eig_ev[s]);
    }
    if (c.eig_fork) cudaEventDestroy(c.eig_fork);
    if (c.solver) cusolverDnDestroy(c.solver);
    for (cudaEvent_t e : {c.ev0, c.ev1, c.ev_p0, c.ev_p1, c.ev_p2})
      if (e) cudaEventDestroy(e);
    if (c.own_stream && c.stream) {
      cudaStreamDestroy(c.stream);
      c.stream = nullptr;   // a buffer released after this point is freed synchronously
    }
  }
  delete ctx;
  return MPSLCC_OK;
}

const char* mpslcc_last_error(const mpslcc_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

mpslcc_status mpslcc_build_mpo(mpslcc_ctx* ctx, const double* h, const double* V, int n_orb, int n_elec,
                               int two_sz) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(h && V, ST_ARG, "null integrals");
    MPSLCC_REQUIRE(n_orb >= 2 && n_orb <= 60, ST_ARG, "n_orb must be in [2, 60]");
    MPSLCC_REQUIRE(n_elec >= 0 && n_elec <= 2 * n_orb, ST_ARG, "n_elec out of range");
    MPSLCC_REQUIRE(((n_elec + two_sz) % 2 == 0) && std::abs(two_sz) <= n_elec &&
                       std::abs(two_sz) <= 2 * n_orb - n_elec,
                   ST_ARG, "n_elec +- two_sz must be even and in range");
    int k = n_orb;
    require_finite(h, (size_t)k * k, "h");
    require_finite(V, (size_t)k * k * k * k, "V");
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q)
        MPSLCC_REQUIRE(std::fabs(h[p * k + q] - h[q * k + p]) <= 1e-10, ST_ARG, "h is not symmetric");
    auto Vat = [&](int a, int b, int cc, int d) { return V[(((size_t)a * k + b) * k + cc) * k + d]; };
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q)
        for (int r = 0; r < k; ++r)
          for (int s = 0; s < k; ++s) {
            double v = Vat(p, q, r, s);
            MPSLCC_REQUIRE(std::fabs(v - Vat(q, p, r, s)) <= 1e-10 && std::fabs(v - Vat(r, s, p, q)) <= 1e-10 &&
                               std::fabs(v - Vat(p, q, s, r)) <= 1e-10,
                           ST_ARG, "V lacks the 8-fold permutational symmetry");
          }
    if (!c.host_only) cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    reset_families(c);
    c.phi0 = MPS();
    c.phi1 = MPS();
    c.phin.clear();
    c.have_E0 = c.have_E2 = c.e3_valid = false;
    c.k = k;
    c.n_elec = n_elec;
    c.two_sz = two_sz;
    c.h.assign(h, h + (size_t)k * k);
    c.V.assign(V, V + (size_t)k * k * k * k);
    c.n_core = 0;
    c.n_active = k;
    c.mpo[MPO_H] = build_mpo(k, h, V, MPO_H, 0, k);
    c.mpo[MPO_ID] = build_mpo(k, h, V, MPO_ID, 0, k);
    if (!c.host_only) {
      upload_boxes(c, MPO_H);
      upload_boxes(c, MPO_ID);
    }
    build_partition_mpos(c);
    c.have_mpo = true;
  });
}

mpslcc_status mpslcc_set_spaces(mpslcc_ctx* ctx, int n_core, int n_active) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(c.have_mpo, ST_STATE, "build_mpo first");
    MPSLCC_REQUIRE(n_core >= 0 && n_active >= 0 && n_core + n_active <= c.k, ST_ARG, "bad partition");
    MPSLCC_REQUIRE(2 * n_core <= c.n_elec && c.n_elec - 2 * n_core <= 2 * n_active, ST_ARG,
                   "electrons do not fit the partition");
    if (!c.host_only) cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    reset_families(c);
    c.phi0 = MPS();
    c.phi1 = MPS();
    c.phin.clear();
    c.have_E0 = c.have_E2 = c.e3_valid = false;
    c.n_core = n_core;
    c.n_active = n_active;
    build_partition_mpos(c);
  });
}

mpslcc_status mpslcc_dmrg_reference(mpslcc_ctx* ctx, int M0, int n_sweeps, double* E0_out) {
  if (ctx) ctx->c.cf.reset();
  return noconv_status(ctx, guard(ctx, [&](Ctx& c) {
    need_device(c);
    MPSLCC_REQUIRE(c.have_mpo, ST_STATE, "build_mpo first");
    MPSLCC_REQUIRE(M0 >= 1 && n_sweeps >= 0, ST_ARG, "M0 must be positive and n_sweeps non-negative");
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    double E;
    if (n_sweeps == 0) {
      MPSLCC_REQUIRE(c.phi0.present, ST_STATE, "n_sweeps = 0 evaluates a loaded reference: load_mps(0) first");
      E = reference_energy_fp64(c);
    } else {
      reset_families(c);
      c.phi1 = MPS();
      c.phin.clear();
      c.have_E2 = c.e3_valid = false;
      E = dmrg_reference(c, M0, n_sweeps);
    }
    if (E0_out) *E0_out = E;
  }));
}

mpslcc_status mpslcc_lcc_sweep(mpslcc_ctx* ctx, int M1, int order, int n_sweeps, double* E2_out) {
  if (ctx) ctx->c.cf.reset();
  return noconv_status(ctx, guard(ctx, [&](Ctx& c) {
    need_device(c);
    MPSLCC_REQUIRE(order >= 1 && order <= Ctx::MAX_ORDER, ST_ARG, "order must be in [1, 8]");
    MPSLCC_REQUIRE(M1 >= 1 && n_sweeps >= 1, ST_ARG, "M1 and n_sweeps must be positive");
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    double E2 = lcc_sweeps(c, M1, n_sweeps, order);
    if (E2_out) *E2_out = E2;
  }));
}

mpslcc_status mpslcc_lcc_sweep_onesite(mpslcc_ctx* ctx, int order, int n_sweeps, double* J_out) {
  if (ctx) ctx->c.cf.reset();
  return noconv_status(ctx, guard(ctx, [&](Ctx& c) {
    need_device(c);
    MPSLCC_REQUIRE(order >= 1 && order <= Ctx::MAX_ORDER, ST_ARG, "order must be in [1, 8]");
    MPSLCC_REQUIRE(n_sweeps >= 1, ST_ARG, "n_sweeps must be positive");
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    double J = lcc_sweeps1(c, n_sweeps, order);
    if (J_out) *J_out = J;
  }));
}

mpslcc_status mpslcc_lcc_sweep_window(mpslcc_ctx* ctx, int M1, int order, int first, int count, int dir,
                                      double* J_out) {
  if (ctx) ctx->c.cf.reset();
  return noconv_status(ctx, guard(ctx, [&](Ctx& c) {
    need_device(c);
    MPSLCC_REQUIRE(order >= 1 && order <= Ctx::MAX_ORDER, ST_ARG, "order must be in [1, 8]");
    MPSLCC_REQUIRE(M1 >= 1, ST_ARG, "M1 must be positive");
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    double J = lcc_window(c, M1, first, count, dir, order);
    if (J_out) *J_out = J;
  }));
}

mpslcc_status mpslcc_energy_series(mpslcc_ctx* ctx, double* E, int max_terms, int* n_terms) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(c.have_E0 && c.phi1.present, ST_STATE, "the energy series needs E0 and Phi1");
    MPSLCC_REQUIRE(max_terms >= 0 && (E || max_terms == 0), ST_ARG, "bad output buffer");
    if (!c.series_valid) {
      need_device(c);
      cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
      compute_series(c);
    }
    const int n = (int)c.Eseries.size();
    for (int i = 0; i < std::min(n, max_terms); ++i) E[i] = c.Eseries[i];
    if (n_terms) *n_terms = n;
  });
}

mpslcc_status mpslcc_energy(mpslcc_ctx* ctx, mpslcc_energies* out) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(out, ST_ARG, "null output");
    MPSLCC_REQUIRE(c.have_E0, ST_STATE, "no reference energy yet");
    if (c.phi1.present && c.phi0.present && !c.e_valid) {
      // FP64 evaluation of the current states (optimised or loaded)
      need_device(c);
      cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
      compute_energies(c);
      c.have_E2 = true;
    }
    std::memset(out, 0, sizeof(*out));
    out->E0 = c.E0;
    out->E2 = c.have_E2 ? c.E2 : 0.0;
    out->E3 = c.have_E2 ? c.E3 : 0.0;
    out->E_lcc2 = out->E0 + out->E2;
    out->E_lcc3 = out->E_lcc2 + out->E3;
    out->hylleraas = c.J;
    out->overlap01 = c.ovl01;
    out->norm1 = c.norm1;
    out->max_discarded_weight = c.max_disc;
    out->sweeps_done = c.sweeps_done;
    out->flags = c.flags;
  });
}

mpslcc_status mpslcc_local_dim(mpslcc_ctx* ctx, int site, int op, long* n_out, long* n_in) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(site >= 0 && site <= c.k - 2, ST_ARG, "site out of range");
    MPS* bra = (op == MPSLCC_OP_H0_00) ? &c.phi0 : &c.phi1;
    MPS* ket = (op == MPSLCC_OP_H0_00 || op == MPSLCC_OP_H_10 || op == MPSLCC_OP_S_10) ? &c.phi0 : &c.phi1;
    MPSLCC_REQUIRE(op >= 0 && op <= 5, ST_ARG, "unknown operator");
    MPSLCC_REQUIRE(bra->present && ket->present, ST_STATE, "MPS for this operator not present");
    std::vector<QN> mid;
    std::vector<long> off;
    long nb = 0, nk = 0;
    two_site_middle(*bra, site, mid, off, nb);
    two_site_middle(*ket, site, mid, off, nk);
    if (n_out) *n_out = nb;
    if (n_in) *n_in = nk;
  });
}

static void apply_heff_dev(Ctx& c, int site, int op, const double* d_psi, double* d_sigma, long n_in, long n_out,
                           int prec, bool one_site = false) {
  need_device(c);
  cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
  MPSLCC_REQUIRE(site >= 0 && site <= c.k - (one_site ? 1 : 2), ST_ARG, "site out of range");
  MPSLCC_REQUIRE(prec >= MPSLCC_FP64 && prec <= MPSLCC_BF16X6, ST_ARG, "bad precision");
  Family& F = family_for(c, op);
  SigmaPlan P;
  const int saved = c.gemm_prec;
  c.gemm_prec = c.opts.tc_environments ? MPSLCC_BF16X3 : MPSLCC_FP64;
  try {
    if (one_site) make_sigma_plan1(c, F, site, P);
    else make_sigma_plan(c, F, site, P);
  } catch (...) {
    c.gemm_prec = saved;
    throw;
  }
  c.gemm_prec = saved;
  MPSLCC_REQUIRE(P.nk == n_in && P.nb == n_out, ST_ARG, "vector length does not match the local dimension");
  sigma_apply(c, P, d_psi, d_sigma, prec);
}

mpslcc_status mpslcc_apply_heff(mpslcc_ctx* ctx, int site, int op, const double* psi, double* sigma, long n_in,
                                long n_out, int prec) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(psi && sigma, ST_ARG, "null vector");
    MPSLCC_REQUIRE(n_in >= 0 && n_out >= 0, ST_ARG, "negative vector length");
    require_finite(psi, (size_t)n_in, "psi");
    need_device(c);
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    DBuf x, y;
    x.alloc(&c, std::max(n_in, 1L) * sizeof(double));
    y.alloc(&c, std::max(n_out, 1L) * sizeof(double));
    cuda_check(cudaMemcpyAsync(x.p, psi, n_in * sizeof(double), cudaMemcpyHostToDevice, c.s()), "psi h2d");
    apply_heff_dev(c, site, op, x.d(), y.d(), n_in, n_out, prec);
    cuda_check(cudaMemcpyAsync(sigma, y.p, n_out * sizeof(double), cudaMemcpyDeviceToHost, c.s()), "sigma d2h");
    cuda_check(cudaStreamSynchronize(c.s()), "apply sync");
  });
}

mpslcc_status mpslcc_local_dim1(mpslcc_ctx* ctx, int site, int op, long* n_out, long* n_in) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(site >= 0 && site <= c.k - 1, ST_ARG, "site out of range");
    MPSLCC_REQUIRE(op >= 0 && op <= 5, ST_ARG, "unknown operator");
    MPS* bra = (op == MPSLCC_OP_H0_00) ? &c.phi0 : &c.phi1;
    MPS* ket = (op == MPSLCC_OP_H0_00 || op == MPSLCC_OP_H_10 || op == MPSLCC_OP_S_10) ? &c.phi0 : &c.phi1;
    MPSLCC_REQUIRE(bra->present && ket->present, ST_STATE, "MPS for this operator not present");
    std::vector<QN> mid;
    std::vector<long> off;
    long nb = 0, nk = 0;
    one_site_middle(*bra, site, mid, off, nb);
    one_site_middle(*ket, site, mid, off, nk);
    if (n_out) *n_out = nb;
    if (n_in) *n_in = nk;
  });
}

mpslcc_status mpslcc_apply_heff1(mpslcc_ctx* ctx, int site, int op, const double* psi, double* sigma, long n_in,
                                 long n_out, int prec) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(psi && sigma, ST_ARG, "null vector");
    MPSLCC_REQUIRE(n_in >= 0 && n_out >= 0, ST_ARG, "negative vector length");
    require_finite(psi, (size_t)n_in, "psi");
    need_device(c);
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    DBuf x, y;
    x.alloc(&c, std::max(n_in, 1L) * sizeof(double));
    y.alloc(&c, std::max(n_out, 1L) * sizeof(double));
    cuda_check(cudaMemcpyAsync(x.p, psi, n_in * sizeof(double), cudaMemcpyHostToDevice, c.s()), "psi h2d");
    apply_heff_dev(c, site, op, x.d(), y.d(), n_in, n_out, prec, true);
    cuda_check(cudaMemcpyAsync(sigma, y.p, n_out * sizeof(double), cudaMemcpyDeviceToHost, c.s()), "sigma d2h");
    cuda_check(cudaStreamSynchronize(c.s()), "apply sync");
  });
}

mpslcc_status mpslcc_apply_heff_device(mpslcc_ctx* ctx, int site, int op, const double* d_psi, double* d_sigma,
                                       long n_in, long n_out, int prec) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(d_psi && d_sigma, ST_ARG, "null vector");
    apply_heff_dev(c, site, op, d_psi, d_sigma, n_in, n_out, prec);
  });
}

mpslcc_status mpslcc_load_mps(mpslcc_ctx* ctx, int which, int n_sites, const int* bond_nsec, const int* bond_qn,
                              const int* bond_dim, const int* site_nblk, const int* blk_desc, const double* data,
                              long n_data) {
  return guard(ctx, [&](Ctx& c) {
    need_device(c);
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    MPSLCC_REQUIRE(which >= 0 && which <= Ctx::MAX_ORDER, ST_ARG, "which must be in [0, 8]");
    MPSLCC_REQUIRE(c.have_mpo && n_sites == c.k, ST_ARG, "n_sites must equal n_orb");
    MPSLCC_REQUIRE(bond_nsec && bond_qn && bond_dim && site_nblk && blk_desc && data, ST_ARG, "null input");
    int k = n_sites;
    MPS m;
    m.k = k;
    m.target = QN(c.n_elec, c.two_sz);
    m.bond.resize(k + 1);
    int qi = 0, di = 0;
    for (int b = 0; b <= k; ++b) {
      MPSLCC_REQUIRE(bond_nsec[b] >= 1, ST_ARG, "empty bond");
      for (int i = 0; i < bond_nsec[b]; ++i) {
        QN q(bond_qn[qi], bond_qn[qi + 1]);
        qi += 2;
        int d = bond_dim[di++];
        MPSLCC_REQUIRE(d >= 1, ST_ARG, "sector dimension must be positive");
        if (i > 0) MPSLCC_REQUIRE(m.bond[b].q.back() < q, ST_ARG, "bond sectors must be strictly ascending");
        m.bond[b].q.push_back(q);
        m.bond[b].d.push_back(d);
      }
    }
    MPSLCC_REQUIRE(m.bond[0].size() == 1 && m.bond[0].q[0] == QN(0, 0), ST_ARG, "left boundary must be (0,0)");
    MPSLCC_REQUIRE(m.bond[k].size() == 1 && m.bond[k].q[0] == m.target, ST_ARG,
                   "right boundary must be (n_elec, two_sz)");
    m.mask.assign(k, {});
    m.site.resize(k);
    struct Blk { int ia, s, ib; long off; };
    std::vector<std::vector<Blk>> blks(k);
    long pos = 0;
    int bi = 0;
    for (int p = 0; p < k; ++p) {
      std::vector<int> seen(4, which >= 1 ? 1 : 0);
      for (int t = 0; t < site_nblk[p]; ++t) {
        int ia = blk_desc[3 * bi], s = blk_desc[3 * bi + 1], ib = blk_desc[3 * bi + 2];
        ++bi;
        MPSLCC_REQUIRE(ia >= 0 && ia < m.bond[p].size() && ib >= 0 && ib < m.bond[p + 1].size() && s >= 0 && s < 4,
                       ST_ARG, "block index out of range");
        MPSLCC_REQUIRE(m.bond[p].q[ia] + LOCAL_Q[s] == m.bond[p + 1].q[ib], ST_ARG,
                       "block violates quantum-number conservation");
        blks[p].push_back({ia, s, ib, pos});
        pos += (long)m.bond[p].d[ia] * m.bond[p + 1].d[ib];
        seen[s] = 1;
      }
      for (int s = 0; s < 4; ++s)
        if (seen[s]) m.mask[p].push_back(s);
      MPSLCC_REQUIRE(!m.mask[p].empty(), ST_ARG, "site without blocks");
    }
    MPSLCC_REQUIRE(pos == n_data, ST_ARG, "n_data does not match the block sizes");
    require_finite(data, (size_t)n_data, "MPS data");
    for (int p = 0; p < k; ++p) {
      long tot;
      std::vector<long> off = layout_offsets(m, p, 0, &tot);
      Fused FL = fuse_left(m.bond[p], m.mask[p]);
      std::vector<double> host(std::max(tot, 1L), 0.0);
      for (const auto& b : blks[p]) {
        int f = FL.find(m.bond[p + 1].q[b.ib]);
        const Piece* pc = FL.piece(f, b.ia, b.s);
        int da = m.bond[p].d[b.ia], db = m.bond[p + 1].d[b.ib];
        for (int r = 0; r < da; ++r)
          for (int j = 0; j < db; ++j)
            host[off[b.ib] + (long)(pc->off + r) * db + j] = data[b.off + (long)r * db + j];
      }
      DBuf d;
      d.alloc(&c, host.size() * sizeof(double));
      cuda_check(cudaMemcpyAsync(d.p, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c.s()),
                 "upload site");
      cuda_check(cudaStreamSynchronize(c.s()), "upload site sync");
      set_site_lf(c, m, p, std::move(d));
    }
    m.present = true;
    reset_families(c);
    if (which == 0) {
      c.phi0 = std::move(m);
      c.have_E0 = false;
    } else {
      *c.phi_of(which) = std::move(m);
    }
    c.have_E2 = c.e3_valid = c.e_valid = false;
    c.series_valid = false;
  });
}

mpslcc_status mpslcc_export_mps(mpslcc_ctx* ctx, int which, int* meta, long* n_int, double* data, long* n_data) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(which >= 0 && which <= Ctx::MAX_ORDER, ST_ARG, "which must be in [0, 8]");
    MPS& m = *c.phi_of(which);
    MPSLCC_REQUIRE(m.present, ST_STATE, "MPS not present");
    int k = m.k;
    std::vector<int> nsec, qn, dims, nblk, desc;
    long nd = 0;
    for (int b = 0; b <= k; ++b) {
      nsec.push_back(m.bond[b].size());
      for (int i = 0; i < m.bond[b].size(); ++i) {
        qn.push_back(m.bond[b].q[i].n);
        qn.push_back(m.bond[b].q[i].s);
        dims.push_back(m.bond[b].d[i]);
      }
    }
    for (int p = 0; p < k; ++p) {
      int cnt = 0;
      for (int ia = 0; ia < m.bond[p].size(); ++ia)
        for (int s : m.mask[p]) {
          int ib = m.bond[p + 1].find(m.bond[p].q[ia] + LOCAL_Q[s]);
          if (ib < 0) continue;
          desc.push_back(ia);
          desc.push_back(s);
          desc.push_back(ib);
          nd += (long)m.bond[p].d[ia] * m.bond[p + 1].d[ib];
          ++cnt;
        }
      nblk.push_back(cnt);
    }
    long ni = (long)(nsec.size() + qn.size() + dims.size() + nblk.size() + desc.size());
    if (n_int) *n_int = ni;
    if (n_data) *n_data = nd;
    if (!meta || !data) return;
    int* o = meta;
    for (auto* v : {&nsec, &qn, &dims, &nblk, &desc})
      for (int x : *v) *o++ = x;
    need_device(c);
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    long pos = 0;
    for (int p = 0; p < k; ++p) {
      ensure_lf(c, m, p);
      long tot;
      std::vector<long> off = layout_offsets(m, p, 0, &tot);
      std::vector<double> host(std::max(tot, 1L));
      cuda_check(cudaMemcpyAsync(host.data(), m.site[p].lf.p, tot * sizeof(double), cudaMemcpyDeviceToHost, c.s()),
                 "site d2h");
      cuda_check(cudaStreamSynchronize(c.s()), "site d2h sync");
      Fused FL = fuse_left(m.bond[p], m.mask[p]);
      for (int ia = 0; ia < m.bond[p].size(); ++ia)
        for (int s : m.mask[p]) {
          int ib = m.bond[p + 1].find(m.bond[p].q[ia] + LOCAL_Q[s]);
          if (ib < 0) continue;
          int f = FL.find(m.bond[p + 1].q[ib]);
          const Piece* pc = FL.piece(f, ia, s);
          int da = m.bond[p].d[ia], db = m.bond[p + 1].d[ib];
          for (int r = 0; r < da; ++r)
            for (int j = 0; j < db; ++j) data[pos++] = host[off[ib] + (long)(pc->off + r) * db + j];
        }
    }
  });
}

mpslcc_status mpslcc_mpo_bond_dims(mpslcc_ctx* ctx, int which, int* bond_dims) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(c.have_mpo, ST_STATE, "build_mpo first");
    MPSLCC_REQUIRE(which >= 0 && which <= 3 && bond_dims, ST_ARG, "bad argument");
    for (int b = 0; b <= c.k; ++b) bond_dims[b] = c.mpo[which].bond[b].n;
  });
}

mpslcc_status mpslcc_export_mpo_site(mpslcc_ctx* ctx, int which, int site, int* idx, double* val, long* count) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(c.have_mpo, ST_STATE, "build_mpo first");
    MPSLCC_REQUIRE(which >= 0 && which <= 3 && site >= 0 && site < c.k && count, ST_ARG, "bad argument");
    const auto& e = c.mpo[which].site[site].e;
    *count = (long)e.size();
    if (!idx || !val) return;
    for (size_t i = 0; i < e.size(); ++i) {
      idx[4 * i] = e[i].w0;
      idx[4 * i + 1] = e[i].w1;
      idx[4 * i + 2] = e[i].so;
      idx[4 * i + 3] = e[i].si;
      val[i] = e[i].val;
    }
  });
}

mpslcc_status mpslcc_get_stats(mpslcc_ctx* ctx, mpslcc_stats* out) {
  return guard(ctx, [&](Ctx& c) {
    MPSLCC_REQUIRE(out, ST_ARG, "null output");
    std::memset(out, 0, sizeof(*out));
    out->sigma_flops = c.st.sigma_flops;
    out->sigma_seconds = c.st.sigma_seconds;
    out->sigma_calls = c.st.sigma_calls;
    out->gemm_launches = c.st.gemm_launches;
    out->kernel_launches = c.st.kernel_launches;
    out->env_flops = c.st.env_flops;
    out->last_sweep_seconds = c.st.last_sweep_seconds;
    out->last_sweep_sigma_seconds = c.st.last_sweep_sigma_seconds;
    out->last_sweep_sigma_flops = c.st.last_sweep_sigma_flops;
    out->last_sweep_sigma_calls = c.st.last_sweep_sigma_calls;
    out->last_sweep_kernel_launches = c.st.last_sweep_kernel_launches;
    out->max_bond_dim = c.st.max_bond_dim;
    out->mpo_max_bond = c.have_mpo ? c.mpo[MPO_H].max_bond() : 0;
    out->tc_phase1_seconds = c.st.tc_phase1_s;
    out->tc_phase2_seconds = c.st.tc_phase2_s;
    out->tc_phase1_bytes = c.st.tc_phase1_bytes;
    out->tc_phase2_bytes = c.st.tc_phase2_bytes;
    out->f64_phase1_seconds = c.st.f64_phase1_s;
    out->f64_phase2_seconds = c.st.f64_phase2_s;
    out->tc_launches = c.st.tc_launches;
    out->t_plan = c.st.t_plan;
    out->t_trunc = c.st.t_trunc;
    out->t_env = c.st.t_env;
    out->t_fuse_left = c.st.t_fuse_left;
    out->t_fuse_right = c.st.t_fuse_right;
    out->t_tc_prepare = c.st.t_tc_prepare;
    out->ahead_used = c.st.ahead_used;
    out->ahead_missed = c.st.ahead_missed;
    out->t_solve = c.st.t_solve;
    out->t_rhs = c.st.t_rhs;
    out->n_noconv = c.st.n_noconv;
    out->n_indefinite = c.st.n_indefinite;
    out->n_j_rise = c.st.n_j_rise;
    out->max_rel_residual = c.st.max_rel_residual;
    out->tune_trials = c.st.tune_trials;
    out->tc_launches_n256 = c.st.tc_cap_launches[0];
    out->tc_launches_n128 = c.st.tc_cap_launches[1];
    out->tc_launches_n64 = c.st.tc_cap_launches[2];
    out->tc_launches_n64x2 = c.st.tc_cap_launches[3];
  });
}

mpslcc_status mpslcc_debug_tc_gemm(mpslcc_ctx* ctx, int prec, int m, int n, int k, const double* A,
                                   const double* B, double* C, int mode, int ksplit) {
  return guard(ctx, [&](Ctx& c) {
    need_device(c);
    MPSLCC_REQUIRE(prec >= MPSLCC_TF32 && prec <= MPSLCC_BF16X3, ST_ARG, "prec must be TF32, BF16 or BF16X3");
    MPSLCC_REQUIRE(!(prec == MPSLCC_BF16X3 && (mode == 1 || mode == 3)), ST_ARG, "split operands need an FP32 output mode");
    MPSLCC_REQUIRE(m >= 1 && n >= 1 && k >= 1 && A && B && C && mode >= 0 && mode <= 2, ST_ARG, "bad argument");
    cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    tc_selftest(c, prec, m, n, k, A, B, C, mode, std::max(1, ksplit));
  });
}

mpslcc_status mpslcc_tc_gemm_noalloc(int device, void* stream, int prec, int m, int n, int k, const double* d_A,
                                     const double* d_B, double* d_C) {
  try {
    tc_gemm_noalloc(device, (cudaStream_t)stream, prec, m, n, k, d_A, d_B, d_C);
    return MPSLCC_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    return (mpslcc_status)e.status;
  } catch (...) {
    return MPSLCC_E_INTERNAL;
  }
}

size_t mpslcc_tc_gemm_noalloc_scratch_bytes(void) { return tc_gemm_noalloc_max_bytes(); }

mpslcc_status mpslcc_reset_stats(mpslcc_ctx* ctx) {
  return guard(ctx, [&](Ctx& c) { c.st = Stats(); });
}

}  // extern "C"
