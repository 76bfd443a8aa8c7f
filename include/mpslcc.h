/*
 * mpslcc.h -- C ABI of the GB300 (sm_103a) MPS-LCC hot-path library.
 *
 * Method: Sharma & Alavi, "Multireference linearized coupled cluster theory
 * for strongly correlated systems using matrix product states".  The library
 * builds matrix product operators for H and the Fink zeroth-order H0
 * (Theory section, Eq. "part"), optimises a DMRG reference Phi0 (Eq. EH), and
 * optimises the first-order wavefunction Phi1 as one MPS by minimising the
 * Hylleraas functional (Eq. 1b, read consistently with Eq. 1) with two-site
 * sweeps (Implementation section).  The hot operation is the local
 * effective-Hamiltonian application ("sigma vector", Fig. 3): the derivative
 * of the functional with respect to the local tensor.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Orbitals are the MPS sites 0..n_orb-1; local basis of one orbital:
 *   0=|0>, 1=|up>, 2=|dn>, 3=|up dn> = a+_up a+_dn |0>; occupation-number
 *   states are prod_p (a+_p,up)^n (a+_p,dn)^n |vac> in ascending p.
 * - Quantum numbers are U(1)xU(1): (N, 2S_z).  Bond b (0..n_orb) sits left of
 *   site b; its sector labels are left-cumulative (electrons and 2S_z of sites
 *   0..b-1) and are listed in ascending (N, 2S_z) order.
 * - Local (two-site) vector layout at position l (sites l, l+1): middle
 *   sectors q ascending by (N, 2S_z); each sector is a row-major block with
 *   rows = (s_l ascending, bond-l sector ascending, index within sector) and
 *   cols = (s_l+1 ascending, bond-(l+2) sector ascending, index), restricted
 *   to the local states each site allows.  A sector appears iff both its row
 *   and column spaces are non-empty.
 * - All arrays passed in are owned by the caller and only read during the
 *   call; outputs go to caller-allocated buffers.  The context owns all its
 *   device memory.  Functions never abort: on failure they return a status,
 *   leave the context in its previous valid state, and record a message
 *   readable with mpslcc_last_error().  One context per host thread.
 * - Call order: create -> build_mpo -> (set_spaces) -> dmrg_reference ->
 *   lcc_sweep -> energy.  Out-of-order calls return MPSLCC_E_STATE.
 */
#ifndef MPSLCC_H
#define MPSLCC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpslcc_ctx mpslcc_ctx;

typedef enum {
  MPSLCC_OK = 0,
  MPSLCC_E_ARG = 1,      /* invalid argument (sizes, symmetry, parity)     */
  MPSLCC_E_STATE = 2,    /* call out of order                              */
  MPSLCC_E_CUDA = 3,     /* CUDA / cuSOLVER error                          */
  MPSLCC_E_NOMEM = 4,    /* device allocation failed                       */
  MPSLCC_E_NOCONV = 5,   /* iterative solver did not converge; result kept */
  MPSLCC_E_TIMEOUT = 6,  /* a bounded device wait gave up                  */
  MPSLCC_E_INTERNAL = 7,
  MPSLCC_E_NUMERIC = 8   /* a non-finite value met inside an iterative
                            solver (breakdown); see the sweep calls        */
} mpslcc_status;

/* FP64 DFMA; TF32 or BF16 tensor-core operands (FP32 accumulation); BF16X3:
   operands split into BF16 hi + lo parts, hi*hi + hi*lo + lo*hi accumulated
   in FP32 (about 2^-17 relative accuracy); BF16X6: three BF16 parts h, m, l,
   the six products hh hm mh mm hl lh accumulated in FP32 (about 2^-24, the
   level of the FP32 accumulation; used for residuals) */
typedef enum {
  MPSLCC_FP64 = 0,
  MPSLCC_TF32 = 1,
  MPSLCC_BF16 = 2,
  MPSLCC_BF16X3 = 3,
  MPSLCC_BF16X6 = 4
} mpslcc_prec;

/* Operators for mpslcc_apply_heff / mpslcc_local_dim. */
typedef enum {
  MPSLCC_OP_H0_11 = 0,   /* P1^T H0 P1 : LCC matrix (without the -E0 shift)  */
  MPSLCC_OP_H0_00 = 1,   /* P0^T H0 P0 : reference (DMRG) matrix             */
  MPSLCC_OP_H_10 = 2,    /* P1^T H P0  : transition, input in Phi0's space   */
  MPSLCC_OP_U_11 = 3,    /* P1^T U P1  : perturbation U = H - H0             */
  MPSLCC_OP_S_10 = 4,    /* P1^T P0    : overlap, input in Phi0's space      */
  MPSLCC_OP_H_11 = 5     /* P1^T H P1                                        */
} mpslcc_op;

typedef struct {
  int device;            /* CUDA device ordinal; -1 = host-only context that
                            can build and export MPOs but runs no kernels   */
  void* stream;          /* cudaStream_t to run on; NULL = library-owned    */
  int prec;              /* mpslcc_prec of the inner sigma products          */
  double tol;            /* solver residual tolerance (relative)             */
  int max_iter;          /* solver iteration cap per site                    */
  int solver;            /* 0 = CG, 1 = MINRES, 2 = auto (CG, MINRES when a
                            non-positive curvature is met)                   */
  int davidson_max_subspace;
  int refine_steps;      /* outer FP64 refinement steps (mixed precision)    */
  unsigned long long seed;   /* initial-guess MPS seed                       */
  int verbose;
  /* Optional device allocator (e.g. a framework's caching allocator).  NULL
     means cudaMallocAsync / cudaFreeAsync on the context stream. */
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, size_t bytes, void* user);
  void* alloc_user;
  int init_guess;        /* reference start: 0 = random MPS over all allowed
                            sectors (opts.seed), 1 = product state filling
                            the active orbitals of lowest h_pp            */
  double wait_timeout_s; /* bound on every device-side wait of the tensor-core
                            kernels, seconds (0 = 2 s, at most 60 s); a wait
                            that runs out makes the call return
                            MPSLCC_E_TIMEOUT and leaves the context usable  */
  int tc_environments;   /* 1: the environments and fused operators that
                            mpslcc_apply_heff builds run on the tensor cores
                            as inside mixed-precision sweeps (three-piece
                            BF16 split, about 2^-24 relative per product);
                            0: FP64                                        */
  int autotune;          /* tile-shape autotuner of the tensor-core sigma
                            phases: 1 (default) tries N tiles of 256, 128 and
                            64 rows on the first products of each position
                            and keeps the fastest; 0 uses 256              */
  int eig_reserved_sms;  /* SMs that the persistent tensor-core launches
                            leave free while a truncation's FP64
                            eigensolvers run on their side streams (the
                            next position's fused operators are built
                            meanwhile): 0 = default (32), < 0 = none       */
  int residual_fp64;     /* mixed-precision LCC sweeps: 1 forms the
                            right-hand side and the refinement residuals
                            with FP64 products on FP64 environments and
                            fused operators (the inner solves stay on the
                            tensor cores); 0 (default): BF16X6 products on
                            tensor-core environments                        */
} mpslcc_opts;

typedef struct {
  double E0;        /* <Phi0|H|Phi0> of the reference                        */
  double E2;        /* second order: Hylleraas minimum = <Phi0|H|Phi1>       */
  double E3;        /* third order: <Phi1|U|Phi1> (Eq. 2, n = 1)             */
  double E_lcc2;    /* E0 + E2                                               */
  double E_lcc3;    /* E0 + E2 + E3                                          */
  double hylleraas; /* last local Hylleraas value                           */
  double overlap01; /* <Phi1|Phi0>                                           */
  double norm1;     /* <Phi1|Phi1>                                           */
  double max_discarded_weight;
  int sweeps_done;
  int flags;        /* MPSLCC_FLAG_* of the last sweep call and the energies */
} mpslcc_energies;

/* Bits of mpslcc_energies.flags. */
enum {
  MPSLCC_FLAG_NOCONV = 1,     /* a local solve stopped at max_iter above its
                                 tolerance (the call returned E_NOCONV)      */
  MPSLCC_FLAG_INDEFINITE = 2, /* a local LCC matrix Q(H0 - E0)Q showed a
                                 non-positive curvature (MINRES was used): the
                                 Hylleraas functional has no minimum there,
                                 typically because Phi0 is not the lowest H0
                                 state of the reference class                */
  MPSLCC_FLAG_E2_POSITIVE = 4,/* E2 > 0: no Hylleraas minimum was reached     */
  MPSLCC_FLAG_J_ROSE = 8      /* the local Hylleraas value rose from one
                                 position to the next by more than 1e-6
                                 relative (beyond truncation effects)        */
};

typedef struct {
  double sigma_flops;       /* algorithmic flops of all sigma products       */
  double sigma_seconds;     /* device time inside sigma products             */
  long long sigma_calls;
  long long gemm_launches;
  long long kernel_launches;
  double env_flops;
  double last_sweep_seconds;
  double last_sweep_sigma_seconds;
  double last_sweep_sigma_flops;
  long long last_sweep_sigma_calls;
  long long last_sweep_kernel_launches;
  int max_bond_dim;
  int mpo_max_bond;         /* largest MPO bond dimension (H)                */
  double tc_phase1_seconds; /* device time of tensor-core sigma phase 1      */
  double tc_phase2_seconds; /* ... and phase 2                              */
  double tc_phase1_bytes;   /* algorithmic operand + result bytes, phase 1   */
  double tc_phase2_bytes;   /* ... phase 2                                   */
  double f64_phase1_seconds;/* device time of the FP64 sigma phases          */
  double f64_phase2_seconds;
  long long tc_launches;
  double t_plan;            /* LCC sweep wall seconds: fused operators      */
  double t_trunc;           /*   truncation (density matrix, FP64 eigh)      */
  double t_env;             /*   environment renormalisation                 */
  double t_solve;           /*   local linear solves                         */
  double t_rhs;             /*   right-hand side, projector, diagonal        */
  double t_fuse_left;       /* wall seconds building L' (all sweeps)         */
  double t_fuse_right;      /* ... building R'                               */
  double t_tc_prepare;      /* ... low-precision copies of L', R' and tasks  */
  long long ahead_used;     /* fused operators built during the previous
                               truncation and used by the next plan          */
  long long ahead_missed;   /* ... discarded (middle sectors had changed)    */
  long long n_noconv;       /* local solves (Davidson, CG / MINRES) that
                               stopped at max_iter above their tolerance    */
  long long n_indefinite;   /* local LCC solves that met non-positive
                               curvature and switched to MINRES             */
  long long n_j_rise;       /* positions whose local Hylleraas value rose
                               above the previous position's (1e-6 rel.)    */
  double max_rel_residual;  /* largest final relative residual |b - Ax|/|b|
                               of the local LCC solves of the last call      */
  long long tune_trials;    /* autotuner trial launches                      */
  long long tc_launches_n256; /* tensor-core sigma launches with N tiles of
                                 at most 256 rows (chosen by the autotuner)  */
  long long tc_launches_n128;
  long long tc_launches_n64;
  long long tc_launches_n64x2; /* ... N tiles of at most 64 rows, two CTAs
                                  per SM                                    */
} mpslcc_stats;

/* Fill *opts with defaults (device 0, FP64, tol 1e-10, max_iter 200, auto
   solver, subspace 24, refine 4, seed 7, autotuner on). */
void mpslcc_default_opts(mpslcc_opts* opts);

/* Create / destroy a context.  Errors: E_ARG (NULL), E_CUDA (device). */
mpslcc_status mpslcc_create(mpslcc_ctx** out, const mpslcc_opts* opts);
mpslcc_status mpslcc_destroy(mpslcc_ctx* ctx);
const char* mpslcc_last_error(const mpslcc_ctx* ctx);

/* Theory section, Eq. "part": build the MPOs of H, H0 and U = H - H0 from the
   one-body integrals h (n_orb x n_orb, row-major, symmetric) and chemists'
   two-electron integrals V = (ij|kl) (n_orb^4, row-major, 8-fold symmetric),
   H = sum h_ij a+_is a_js + 1/2 sum (ij|kl) a+_is a+_kt a_lt a_js, for
   n_elec electrons with 2S_z = two_sz.  Errors: E_ARG if n_elec +- two_sz is
   odd or out of range, or h / V lack their symmetry (tolerance 1e-10). */
mpslcc_status mpslcc_build_mpo(mpslcc_ctx* ctx, const double* h, const double* V,
                               int n_orb, int n_elec, int two_sz);

/* Theory section (Fink partition): orbitals 0..n_core-1 are core (occupancy
   2), the next n_active are active, the rest virtual (occupancy 0).  H0 keeps
   the terms that move no electrons between the three sets.  Default after
   build_mpo: n_core = 0, n_active = n_orb (H0 = H).  Rebuilds H0 and U;
   discards any reference and first-order state. */
mpslcc_status mpslcc_set_spaces(mpslcc_ctx* ctx, int n_core, int n_active);

/* Eq. EH: two-site DMRG for the reference Phi0 (lowest eigenvector of H0 in
   the reference class: core sites fixed to |up dn>, virtual sites to |0>),
   bond dimension M0, n_sweeps left-right-left sweeps, Davidson local solver.
   Writes E0 = <Phi0|H|Phi0>.  n_sweeps = 0 keeps a reference loaded by
   mpslcc_load_mps(0) and only evaluates its E0 in FP64 (E_STATE if none is
   loaded).  E_NOCONV if a local solve hit max_iter. */
mpslcc_status mpslcc_dmrg_reference(mpslcc_ctx* ctx, int M0, int n_sweeps, double* E0_out);

/* Eq. 1 (n = 1) in projector form: optimise Phi1 (bond dimension M1) by
   minimising J = <Phi1|Q(H0-E0)Q|Phi1> - 2<Phi1|b>, b = -Q H Phi0, with
   n_sweeps two-site sweeps; local linear solves by CG / MINRES with the
   precision of opts.prec for inner products and FP64 residuals.  Writes E2
   (the final Hylleraas value) to *E2_out.  The first call initialises Phi1
   from opts.seed; later calls continue from the current Phi1.
   order = n >= 2 (at most 8; Eq. 1 for n > 1): sweeps the order-n
   wavefunction Phi(n) (one MPS of bond dimension M1, initialised at the
   first call) by minimising <x|Q(H0-E0)Q|x> - 2<x|b_n> with
   b_n = -Q U Phi(n-1) + sum_{k=2..n-1} E(k) Q Phi(n-k), the E(k) from
   mpslcc_energy_series of the lower orders; needs Phi(n-1) (E_STATE
   otherwise) and writes the last local Hylleraas value to *E2_out.  The
   reference component <Phi0|Phi(n-1)> Phi0 of a truncated lower order
   (about 1e-8) is not projected from the U term.  Sweeping order n discards
   the wavefunctions of orders above n. */
mpslcc_status mpslcc_lcc_sweep(mpslcc_ctx* ctx, int M1, int order, int n_sweeps, double* E2_out);

/* One-site sweeps (Implementation section: only the tensor of one site is
   optimised at a time, a local problem of d M^2 entries instead of the
   two-site d^2 M^2) of the order-`order` wavefunction at its current bond
   dimensions: sites 0 .. n_orb-2 left to right, then n_orb-1 .. 1 right to
   left, each a local linear solve of Eq. 1 (as mpslcc_lcc_sweep) on the
   one-site local problem, after which the orthogonality centre moves to the
   neighbouring site without discarding weight.  The bond dimensions do not
   grow: run two-site sweeps (mpslcc_lcc_sweep) first.  Needs the wavefunction
   with its centre at site 0 (after a two-site sweep, or loaded after one);
   E_STATE if it is absent.  Writes the last local Hylleraas value to *J_out;
   E_NOCONV as mpslcc_lcc_sweep. */
mpslcc_status mpslcc_lcc_sweep_onesite(mpslcc_ctx* ctx, int order, int n_sweeps, double* J_out);

/* A window of a half sweep of mpslcc_lcc_sweep (Implementation section: the
   sweep optimises one position at a time): `count` two-site steps starting
   at position `first` (0..n_orb-2) and moving towards higher (dir = +1) or
   lower (dir = -1) positions, each a local linear solve, truncation to M1
   and environment update.  The local matrix is the LCC matrix only when
   `first` is the orthogonality centre of Phi1: position 0 after a full sweep
   (or a loaded state exported after one), or the position next to where a
   previous window in the same direction ended.  Used to time and compare
   precisions on representative positions.  Writes the last local Hylleraas
   value to *J_out.  Errors and E_NOCONV as mpslcc_lcc_sweep. */
mpslcc_status mpslcc_lcc_sweep_window(mpslcc_ctx* ctx, int M1, int order, int first, int count, int dir,
                                      double* J_out);

/* Eq. 1b and Eq. 2 (n = 1): energies of the current states, evaluated in
   FP64 from the MPS tensors as they are (after sweeps, or as loaded with
   mpslcc_load_mps): E0 of Phi0, and for Q Phi1 = Phi1 - <Phi0|Phi1> Phi0 the
   Hylleraas value E2 = J(Q Phi1) and E3 = <Q Phi1|U|Q Phi1>.  Needs E0
   (mpslcc_dmrg_reference); E2 / E3 are 0 while no Phi1 is present. */
mpslcc_status mpslcc_energy(mpslcc_ctx* ctx, mpslcc_energies* out);

/* Eq. 2 (Wigner 2n+1 rule): energy series E(0), E(1), ..., E(2N+1) of the
   current wavefunctions Phi(1..N) (N = highest order present), evaluated in
   FP64 with every Phi(n) projected as Q Phi(n) = Phi(n) - <Phi0|Phi(n)> Phi0.
   E(2) here is the Wigner form <Phi0|H|Q Phi1>; mpslcc_energy's E2 is the
   Hylleraas value (they agree at the exact first-order state).  Writes
   min(2N+2, max_terms) values to E and 2N+2 to *n_terms.  E_STATE without
   E0 and Phi1. */
mpslcc_status mpslcc_energy_series(mpslcc_ctx* ctx, double* E, int max_terms, int* n_terms);

/* Local dimension of the two-site vector at position site (0..n_orb-2) for
   operator op (output dimension for transition ops is the Phi1 space; *n_in
   receives the input dimension, may be NULL). */
mpslcc_status mpslcc_local_dim(mpslcc_ctx* ctx, int site, int op, long* n_out, long* n_in);

/* Fig. 3 / Implementation section: sigma = P_bra^T O P_ket psi at two-site
   position site, with environments built from the current MPS tensors (no
   canonical form is assumed).  psi (n_in doubles) and sigma (n_out doubles)
   are HOST arrays; prec selects FP64 or the TF32/BF16 tensor-core path.
   Errors: E_ARG (sizes), E_STATE (MPS for op not present). */
mpslcc_status mpslcc_apply_heff(mpslcc_ctx* ctx, int site, int op, const double* psi,
                                double* sigma, long n_in, long n_out, int prec);

/* One-site local problem at site `site` (0..n_orb-1): sigma = P_bra^T O P_ket
   psi with P the isometry of all sites but `site`; the local vector is the
   site's tensor in its left-fused layout (bond-(site+1) sectors q ascending,
   each a row-major block with rows = (s ascending, bond-site sector
   ascending, index) and columns = the index within q).  Host arrays, as
   mpslcc_apply_heff. */
mpslcc_status mpslcc_local_dim1(mpslcc_ctx* ctx, int site, int op, long* n_out, long* n_in);
mpslcc_status mpslcc_apply_heff1(mpslcc_ctx* ctx, int site, int op, const double* psi, double* sigma, long n_in,
                                 long n_out, int prec);

/* Same with DEVICE pointers (FP64, on the context stream); no host copies. */
mpslcc_status mpslcc_apply_heff_device(mpslcc_ctx* ctx, int site, int op, const double* d_psi,
                                       double* d_sigma, long n_in, long n_out, int prec);

/* Replace MPS `which` (0 = Phi0, n = 1..8 = Phi(n)) by caller data (checkpoint
   restore and test input).  bond_nsec[b] (b = 0..n_sites) sector counts;
   bond_qn: for every bond, 2*nsec ints (N, 2S_z) ascending; bond_dim: dims.
   site_nblk[p] block counts; blk_desc: per block (ia, s, ib) as sector
   indices of bond p, local state, sector index of bond p+1; data: the blocks
   row-major [dim_a x dim_b] concatenated in the order given (n_data doubles).
   Local states allowed at a site are those appearing in its blocks plus,
   for which = 1, all four.  Errors: E_ARG (inconsistent quantum numbers). */
mpslcc_status mpslcc_load_mps(mpslcc_ctx* ctx, int which, int n_sites, const int* bond_nsec,
                              const int* bond_qn, const int* bond_dim, const int* site_nblk,
                              const int* blk_desc, const double* data, long n_data);

/* Export MPS `which` in the load format.  Call with NULL buffers to query
   sizes (*n_int = ints needed in meta, *n_data = doubles); meta receives
   bond_nsec | bond_qn | bond_dim | site_nblk | blk_desc concatenated. */
mpslcc_status mpslcc_export_mps(mpslcc_ctx* ctx, int which, int* meta, long* n_int,
                                double* data, long* n_data);

/* MPO inspection (host only; works on a device = -1 context).  which: 0 = H,
   1 = H0, 2 = U.  bond_dims receives n_orb+1 ints.  mpslcc_export_mpo_site
   writes the site's nonzero entries as (w_left, w_right, s_out, s_in) ints
   and values; call with NULL to query the count. */
mpslcc_status mpslcc_mpo_bond_dims(mpslcc_ctx* ctx, int which, int* bond_dims);
mpslcc_status mpslcc_export_mpo_site(mpslcc_ctx* ctx, int which, int site, int* idx,
                                     double* val, long* count);

/* Diagnostic entry point: C = A B^T through the tensor-core GEMM kernel of
   the sigma path (one task; A m x k and B n x k row-major FP64 host arrays,
   rounded to prec = TF32 or BF16; C m x n FP64 host output).  mode 0 adds
   FP32 partial sums over `ksplit` K chunks atomically, 1 stores BF16, 2
   stores FP32.  There is no counterpart in the paper; it exists to test the
   kernel in isolation. */
mpslcc_status mpslcc_debug_tc_gemm(mpslcc_ctx* ctx, int prec, int m, int n, int k, const double* A,
                                   const double* B, double* C, int mode, int ksplit);

/* Allocation-free C = A B^T (the product of mpslcc_debug_tc_gemm with FP32
   output) for callers that cannot allocate device memory when they need it:
   a host framework that owns every device allocation and forbids new ones
   inside its step, or code whose device memory must all be reserved at
   start-up.  There is no counterpart in the paper.
   - d_A (m x k), d_B (n x k), d_C (m x n): row-major FP64 DEVICE arrays owned
     by the caller; prec is TF32, BF16 or BF16X3; work runs on `stream` (NULL =
     legacy default stream) of `device`, which must be the current device.
   - The call allocates nothing and needs no context: its operand copies, FP32
     result, task descriptors and error flag live in one file-scope device
     array of mpslcc_tc_gemm_noalloc_scratch_bytes() bytes (64 MiB), reserved
     on every GPU that loads the library until the process exits.  Problems
     whose scratch would exceed it return MPSLCC_E_ARG.
   - The first call on a device looks up the array's device address (set-up);
     make that first call before any stream capture.
   - Every call reuses the same array and overwrites what it needs (padding
     is cleared each call); calls that overlap on the GPU, from any stream or
     thread, race on it.  The call synchronises `stream` to read the kernel's
     error flag.  Returns MPSLCC_E_TIMEOUT if the kernel gave up waiting. */
mpslcc_status mpslcc_tc_gemm_noalloc(int device, void* stream, int prec, int m, int n, int k, const double* d_A,
                                     const double* d_B, double* d_C);
size_t mpslcc_tc_gemm_noalloc_scratch_bytes(void);

mpslcc_status mpslcc_get_stats(mpslcc_ctx* ctx, mpslcc_stats* out);
mpslcc_status mpslcc_reset_stats(mpslcc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MPSLCC_H */
