"""GB300-native MPS-LCC hot path: thin Python binding of ``libmpslcc.so``.

The binding only marshals arguments into the C ABI declared in
``include/mpslcc.h``; every step of the computation runs in the library's
CUDA kernels.  Importing this package does not build anything: if the shared
library is missing it raises ImportError (build it with
``paper_1509_00216_gb300._build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpslcc.so")

FP64, TF32, BF16, BF16X3, BF16X6 = 0, 1, 2, 3, 4
OP_H0_11, OP_H0_00, OP_H_10, OP_U_11, OP_S_10, OP_H_11 = range(6)
MPO_H, MPO_H0, MPO_U, MPO_ID = range(4)

STATUS = {0: "OK", 1: "E_ARG", 2: "E_STATE", 3: "E_CUDA", 4: "E_NOMEM", 5: "E_NOCONV", 6: "E_TIMEOUT",
          7: "E_INTERNAL", 8: "E_NUMERIC"}
E_NOCONV = 5
FLAG_NOCONV, FLAG_INDEFINITE, FLAG_E2_POSITIVE, FLAG_J_ROSE = 1, 2, 4, 8

EXPORTED = [
    "mpslcc_default_opts", "mpslcc_create", "mpslcc_destroy", "mpslcc_last_error", "mpslcc_build_mpo",
    "mpslcc_set_spaces", "mpslcc_dmrg_reference", "mpslcc_lcc_sweep", "mpslcc_lcc_sweep_window", "mpslcc_energy",
    "mpslcc_energy_series", "mpslcc_lcc_sweep_onesite", "mpslcc_local_dim1", "mpslcc_apply_heff1",
    "mpslcc_local_dim",
    "mpslcc_apply_heff", "mpslcc_apply_heff_device", "mpslcc_load_mps", "mpslcc_export_mps",
    "mpslcc_mpo_bond_dims", "mpslcc_export_mpo_site", "mpslcc_get_stats", "mpslcc_reset_stats",
    "mpslcc_debug_tc_gemm", "mpslcc_tc_gemm_noalloc", "mpslcc_tc_gemm_noalloc_scratch_bytes",
]

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Opts(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("prec", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("solver", C.c_int), ("davidson_max_subspace", C.c_int),
                ("refine_steps", C.c_int), ("seed", C.c_ulonglong), ("verbose", C.c_int),
                ("alloc", _ALLOC), ("free", _FREE), ("alloc_user", C.c_void_p),
                ("init_guess", C.c_int), ("wait_timeout_s", C.c_double), ("tc_environments", C.c_int),
                ("autotune", C.c_int), ("eig_reserved_sms", C.c_int),
                ("residual_fp64", C.c_int)]


class Energies(C.Structure):
    _fields_ = [("E0", C.c_double), ("E2", C.c_double), ("E3", C.c_double), ("E_lcc2", C.c_double),
                ("E_lcc3", C.c_double), ("hylleraas", C.c_double), ("overlap01", C.c_double),
                ("norm1", C.c_double), ("max_discarded_weight", C.c_double), ("sweeps_done", C.c_int),
                ("flags", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("sigma_flops", C.c_double), ("sigma_seconds", C.c_double), ("sigma_calls", C.c_longlong),
                ("gemm_launches", C.c_longlong), ("kernel_launches", C.c_longlong), ("env_flops", C.c_double),
                ("last_sweep_seconds", C.c_double), ("last_sweep_sigma_seconds", C.c_double),
                ("last_sweep_sigma_flops", C.c_double), ("last_sweep_sigma_calls", C.c_longlong),
                ("last_sweep_kernel_launches", C.c_longlong), ("max_bond_dim", C.c_int),
                ("mpo_max_bond", C.c_int), ("tc_phase1_seconds", C.c_double), ("tc_phase2_seconds", C.c_double),
                ("tc_phase1_bytes", C.c_double), ("tc_phase2_bytes", C.c_double),
                ("f64_phase1_seconds", C.c_double), ("f64_phase2_seconds", C.c_double),
                ("tc_launches", C.c_longlong), ("t_plan", C.c_double), ("t_trunc", C.c_double),
                ("t_env", C.c_double), ("t_solve", C.c_double), ("t_rhs", C.c_double),
                ("t_fuse_left", C.c_double), ("t_fuse_right", C.c_double), ("t_tc_prepare", C.c_double),
                ("ahead_used", C.c_longlong), ("ahead_missed", C.c_longlong), ("n_noconv", C.c_longlong),
                ("n_indefinite", C.c_longlong), ("n_j_rise", C.c_longlong), ("max_rel_residual", C.c_double),
                ("tune_trials", C.c_longlong), ("tc_launches_n256", C.c_longlong), ("tc_launches_n128", C.c_longlong),
                ("tc_launches_n64", C.c_longlong), ("tc_launches_n64x2", C.c_longlong)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with paper_1509_00216_gb300._build.build()")
    lib = C.CDLL(LIB_PATH)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    lp = C.POINTER(C.c_long)
    vp = C.c_void_p
    sig = {
        "mpslcc_default_opts": (None, [C.POINTER(Opts)]),
        "mpslcc_create": (C.c_int, [C.POINTER(vp), C.POINTER(Opts)]),
        "mpslcc_destroy": (C.c_int, [vp]),
        "mpslcc_last_error": (C.c_char_p, [vp]),
        "mpslcc_build_mpo": (C.c_int, [vp, dp, dp, C.c_int, C.c_int, C.c_int]),
        "mpslcc_set_spaces": (C.c_int, [vp, C.c_int, C.c_int]),
        "mpslcc_dmrg_reference": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "mpslcc_lcc_sweep": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, dp]),
        "mpslcc_lcc_sweep_window": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp]),
        "mpslcc_energy": (C.c_int, [vp, C.POINTER(Energies)]),
        "mpslcc_energy_series": (C.c_int, [vp, dp, C.c_int, ip]),
        "mpslcc_lcc_sweep_onesite": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "mpslcc_local_dim1": (C.c_int, [vp, C.c_int, C.c_int, lp, lp]),
        "mpslcc_apply_heff1": (C.c_int, [vp, C.c_int, C.c_int, dp, dp, C.c_long, C.c_long, C.c_int]),
        "mpslcc_local_dim": (C.c_int, [vp, C.c_int, C.c_int, lp, lp]),
        "mpslcc_apply_heff": (C.c_int, [vp, C.c_int, C.c_int, dp, dp, C.c_long, C.c_long, C.c_int]),
        "mpslcc_apply_heff_device": (C.c_int, [vp, C.c_int, C.c_int, vp, vp, C.c_long, C.c_long, C.c_int]),
        "mpslcc_load_mps": (C.c_int, [vp, C.c_int, C.c_int, ip, ip, ip, ip, ip, dp, C.c_long]),
        "mpslcc_export_mps": (C.c_int, [vp, C.c_int, ip, lp, dp, lp]),
        "mpslcc_mpo_bond_dims": (C.c_int, [vp, C.c_int, ip]),
        "mpslcc_export_mpo_site": (C.c_int, [vp, C.c_int, C.c_int, ip, dp, lp]),
        "mpslcc_get_stats": (C.c_int, [vp, C.POINTER(Stats)]),
        "mpslcc_reset_stats": (C.c_int, [vp]),
        "mpslcc_debug_tc_gemm": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int]),
        "mpslcc_tc_gemm_noalloc": (C.c_int, [C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp]),
        "mpslcc_tc_gemm_noalloc_scratch_bytes": (C.c_size_t, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


class MpsLccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MpsLccNoConvergence(UserWarning):
    """A sweep call returned MPSLCC_E_NOCONV: some local solves stopped at
    max_iter above their tolerance; the call's states and energies were kept."""


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def tc_gemm_noalloc(device, stream, prec, m, n, k, d_A, d_B, d_C):
    """C = A B^T with no device allocation (device pointers; see the header)."""
    st = lib().mpslcc_tc_gemm_noalloc(device, C.c_void_p(stream), prec, m, n, k, C.c_void_p(d_A),
                                      C.c_void_p(d_B), C.c_void_p(d_C))
    if st != 0:
        raise MpsLccError(st, "mpslcc_tc_gemm_noalloc failed")


class Context:
    """One library context (one GPU, one stream).  ``device=-1`` gives a
    host-only context that can build and export MPOs but runs no kernels.
    ``torch_memory=True`` routes device allocations through PyTorch's caching
    allocator on the current torch stream."""

    def __init__(self, device=0, prec=FP64, tol=1e-10, max_iter=200, seed=7, verbose=0, refine_steps=4,
                 davidson_max_subspace=24, torch_memory=False, init_guess=0, wait_timeout_s=0.0, alloc=None,
                 stream=None, tc_environments=False, autotune=True, eig_reserved_sms=0,
                 residual_fp64=False):
        L = lib()
        o = Opts()
        L.mpslcc_default_opts(C.byref(o))
        o.device = device
        o.prec = prec
        o.tol = tol
        o.max_iter = max_iter
        o.seed = seed
        o.verbose = verbose
        o.refine_steps = refine_steps
        o.davidson_max_subspace = davidson_max_subspace
        o.init_guess = init_guess
        o.wait_timeout_s = wait_timeout_s
        o.tc_environments = 1 if tc_environments else 0
        o.autotune = 1 if autotune else 0
        o.eig_reserved_sms = int(eig_reserved_sms)
        o.residual_fp64 = 1 if residual_fp64 else 0
        if stream is not None:
            o.stream = C.c_void_p(stream)
        self._cb = None
        self.last_status = 0
        # The allocator callbacks never let an exception escape: ctypes would
        # print it and hand the library an unset return value (not NULL), a
        # pointer the kernels would then use.  A failed allocation returns
        # NULL, which the library turns into MPSLCC_E_NOMEM.
        if alloc is not None:
            # caller-provided (alloc(nbytes) -> int pointer or 0, free(ptr, nbytes)) pair
            a_fn, f_fn = alloc

            def _a(nbytes, user):
                try:
                    return a_fn(int(nbytes)) or None
                except Exception:
                    return None

            def _f(ptr, nbytes, user):
                try:
                    f_fn(ptr, int(nbytes))
                except Exception:
                    pass

            self._cb = (_ALLOC(_a), _FREE(_f))
            o.alloc, o.free = self._cb
        elif torch_memory and device >= 0:
            import torch
            stream = torch.cuda.current_stream(device)
            o.stream = C.c_void_p(stream.cuda_stream)

            def _a(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
                except Exception:   # torch.OutOfMemoryError among others
                    return None

            def _f(ptr, nbytes, user):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            self._cb = (_ALLOC(_a), _FREE(_f))
            o.alloc, o.free = self._cb
        h = C.c_void_p()
        st = L.mpslcc_create(C.byref(h), C.byref(o))
        if st != 0:
            raise MpsLccError(st, "mpslcc_create failed")
        self.h = h
        self.n_orb = None

    def close(self):
        if getattr(self, "h", None):
            lib().mpslcc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st, soft_noconv=False):
        self.last_status = st
        if st == E_NOCONV and soft_noconv:
            warnings.warn(lib().mpslcc_last_error(self.h).decode(), MpsLccNoConvergence, stacklevel=3)
            return
        if st != 0:
            raise MpsLccError(st, lib().mpslcc_last_error(self.h).decode())

    # -- the hot-path calls ------------------------------------------------
    def build_mpo(self, h, V, n_elec, two_sz=0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        k = h.shape[0]
        self._check(lib().mpslcc_build_mpo(self.h, _dptr(h), _dptr(V), k, n_elec, two_sz))
        self.n_orb = k

    def set_spaces(self, n_core, n_active):
        self._check(lib().mpslcc_set_spaces(self.h, n_core, n_active))

    def dmrg_reference(self, M0, n_sweeps):
        e = C.c_double()
        self._check(lib().mpslcc_dmrg_reference(self.h, M0, n_sweeps, C.byref(e)), soft_noconv=True)
        return e.value

    def lcc_sweep(self, M1, n_sweeps, order=1):
        e = C.c_double()
        self._check(lib().mpslcc_lcc_sweep(self.h, M1, order, n_sweeps, C.byref(e)), soft_noconv=True)
        return e.value

    def lcc_window(self, M1, first, count, direction=1, order=1):
        """Two-site steps over positions first, first + direction, ... (see
        mpslcc_lcc_sweep_window); returns the last local Hylleraas value."""
        e = C.c_double()
        self._check(lib().mpslcc_lcc_sweep_window(self.h, M1, order, first, count, direction, C.byref(e)),
                    soft_noconv=True)
        return e.value

    def lcc_sweep_onesite(self, n_sweeps, order=1):
        """One-site sweeps at the current bond dimensions (after two-site sweeps)."""
        e = C.c_double()
        self._check(lib().mpslcc_lcc_sweep_onesite(self.h, order, n_sweeps, C.byref(e)), soft_noconv=True)
        return e.value

    def local_dim1(self, site, op):
        a, b = C.c_long(), C.c_long()
        self._check(lib().mpslcc_local_dim1(self.h, site, op, C.byref(a), C.byref(b)))
        return a.value, b.value

    def apply_heff1(self, site, op, psi, prec=FP64):
        """One-site sigma at `site` (host arrays)."""
        n_out, n_in = self.local_dim1(site, op)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        if psi.size != n_in:
            raise ValueError(f"psi has {psi.size} entries, local dimension is {n_in}")
        out = np.zeros(n_out)
        self._check(lib().mpslcc_apply_heff1(self.h, site, op, _dptr(psi), _dptr(out), n_in, n_out, prec))
        return out

    def energy_series(self):
        """E(0), E(1), ..., E(2N+1) of the wavefunctions present (Eq. 2)."""
        n = C.c_int()
        self._check(lib().mpslcc_energy_series(self.h, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        self._check(lib().mpslcc_energy_series(self.h, _dptr(out), n.value, C.byref(n)))
        return out

    def energy(self):
        e = Energies()
        self._check(lib().mpslcc_energy(self.h, C.byref(e)))
        return {f: getattr(e, f) for f, _ in Energies._fields_}

    def local_dim(self, site, op):
        a, b = C.c_long(), C.c_long()
        self._check(lib().mpslcc_local_dim(self.h, site, op, C.byref(a), C.byref(b)))
        return a.value, b.value

    def apply_heff(self, site, op, psi, prec=FP64):
        n_out, n_in = self.local_dim(site, op)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        if psi.size != n_in:
            raise ValueError(f"psi has {psi.size} entries, local dimension is {n_in}")
        out = np.zeros(n_out)
        self._check(lib().mpslcc_apply_heff(self.h, site, op, _dptr(psi), _dptr(out), n_in, n_out, prec))
        return out

    def apply_heff_device(self, site, op, d_psi_ptr, d_sigma_ptr, n_in, n_out, prec=FP64):
        self._check(lib().mpslcc_apply_heff_device(self.h, site, op, C.c_void_p(d_psi_ptr),
                                                   C.c_void_p(d_sigma_ptr), n_in, n_out, prec))

    # -- state transfer ------------------------------------------------------
    def load_mps(self, which, mps):
        """Load an MPS in the format of ``synth.random_mps``."""
        bonds, sites = mps["bonds"], mps["sites"]
        nsec = np.array([len(b) for b in bonds], dtype=np.int32)
        qn = np.array([x for b in bonds for s in b for x in (s[0], s[1])], dtype=np.int32)
        dims = np.array([s[2] for b in bonds for s in b], dtype=np.int32)
        nblk = np.array([len(s) for s in sites], dtype=np.int32)
        desc, data = [], []
        for s in sites:
            for key in sorted(s):
                desc.extend(key)
                data.append(np.ascontiguousarray(s[key], dtype=np.float64).ravel())
        desc = np.array(desc, dtype=np.int32)
        data = np.concatenate(data) if data else np.zeros(0)
        self._check(lib().mpslcc_load_mps(self.h, which, len(sites), _iptr(nsec), _iptr(qn), _iptr(dims),
                                          _iptr(nblk), _iptr(desc), _dptr(data), data.size))

    def export_mps(self, which):
        ni, nd = C.c_long(), C.c_long()
        self._check(lib().mpslcc_export_mps(self.h, which, None, C.byref(ni), None, C.byref(nd)))
        meta = np.zeros(ni.value, dtype=np.int32)
        data = np.zeros(nd.value)
        self._check(lib().mpslcc_export_mps(self.h, which, _iptr(meta), C.byref(ni), _dptr(data), C.byref(nd)))
        k = self.n_orb
        pos = 0
        nsec = meta[pos:pos + k + 1]; pos += k + 1
        tot = int(nsec.sum())
        qn = meta[pos:pos + 2 * tot].reshape(-1, 2); pos += 2 * tot
        dims = meta[pos:pos + tot]; pos += tot
        nblk = meta[pos:pos + k]; pos += k
        desc = meta[pos:].reshape(-1, 3)
        bonds, j = [], 0
        for b in range(k + 1):
            bonds.append([(int(qn[j + i, 0]), int(qn[j + i, 1]), int(dims[j + i])) for i in range(nsec[b])])
            j += nsec[b]
        sites, bi, dpos = [], 0, 0
        for p in range(k):
            blocks = {}
            for _ in range(nblk[p]):
                ia, s, ib = (int(x) for x in desc[bi])
                bi += 1
                da, db = bonds[p][ia][2], bonds[p + 1][ib][2]
                blocks[(ia, s, ib)] = data[dpos:dpos + da * db].reshape(da, db).copy()
                dpos += da * db
            sites.append(blocks)
        masks = [tuple(sorted({key[1] for key in s})) for s in sites]
        return dict(bonds=bonds, sites=sites, masks=masks)

    # -- MPO inspection -------------------------------------------------------
    def mpo_bond_dims(self, which=MPO_H):
        out = np.zeros(self.n_orb + 1, dtype=np.int32)
        self._check(lib().mpslcc_mpo_bond_dims(self.h, which, _iptr(out)))
        return out

    def export_mpo_site(self, which, site):
        n = C.c_long()
        self._check(lib().mpslcc_export_mpo_site(self.h, which, site, None, None, C.byref(n)))
        idx = np.zeros(4 * n.value, dtype=np.int32)
        val = np.zeros(n.value)
        self._check(lib().mpslcc_export_mpo_site(self.h, which, site, _iptr(idx), _dptr(val), C.byref(n)))
        return idx.reshape(-1, 4), val

    def stats(self):
        s = Stats()
        self._check(lib().mpslcc_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def debug_tc_gemm(self, A, B, prec=BF16, mode=0, ksplit=1):
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        m, k = A.shape
        n = B.shape[0]
        C_ = np.zeros((m, n))
        self._check(lib().mpslcc_debug_tc_gemm(self.h, prec, m, n, k, _dptr(A), _dptr(B), _dptr(C_), mode, ksplit))
        return C_

    def reset_stats(self):
        self._check(lib().mpslcc_reset_stats(self.h))
