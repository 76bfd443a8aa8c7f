"""GPU sigma vectors against the block-sparse CPU oracle (O2) at the
workloads' own sizes (Implementation section, Fig. 3: sigma = P_bra^T O P_ket
psi).  The determinant-space oracle cannot hold 16-30 orbitals; O2 recomputes
the same local products from U(1) x U(1) blocks with its own MPO, environments
and contraction order, so the comparison is element by element at sector
dimensions of tens to hundreds, with the library's grouped K-split phase-2
launches, and (with tensor-core environments) its batched FP64-emulation
tasks."""
import numpy as np
import pytest

import synth
from oracle import blocksparse as bs

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12
# workload index, M1, M0, positions
WORKLOADS = {
    "threeband_2x4": (3, 1000, 250, (11, 1, 21)),
    "abinitio_k24": (1, 256, 64, (11, 3)),
    "hubbard2d_4x4": (2, 500, 120, (7,)),
    "abinitio_k30": (4, 300, 80, (14,)),
}


def _frozen(m):
    m = dict(m)
    m["masks"] = [tuple(sorted({key[1] for key in s})) for s in m["sites"]]
    return m


def _envs(mpo, bra, ket, positions):
    """O2 environments (left at bond l, right at bond l+2) for each position."""
    k = len(bra["sites"])
    out = {l: [None, None] for l in positions}
    L = bs.boundary_left(mpo)
    for y in range(max(positions) + 1):
        if y in out:
            out[y][0] = L
        if y < max(positions):
            L = bs.update_left(mpo, L, bra, ket, y)
    R = bs.boundary_right(mpo)
    for y in range(k - 1, min(positions) + 1, -1):
        R = bs.update_right(mpo, R, bra, ket, y)
        if y - 2 in out:
            out[y - 2][1] = R
    if k - 2 in out:
        out[k - 2][1] = bs.boundary_right(mpo)
    return out


class Case:
    def __init__(self, mpslcc, name):
        cfg, M1, M0, self.positions = WORKLOADS[name]
        c = synth.config(cfg)
        self.c, self.k = c, c["n_orb"]
        ne = c["n_alpha"] + c["n_beta"]
        self.phi1 = synth.random_mps(self.k, ne, 0, M=M1, seed=31)
        self.phi0 = _frozen(synth.random_mps(self.k, ne, 0, M=M0, seed=32,
                                             masks=synth.site_masks(self.k, c["n_core"], c["n_active"],
                                                                    frozen=True)))
        self.mpo = {kind: bs.Mpo(c["h"], c["V"], kind, c["n_core"], c["n_active"]) for kind in ("H0", "H", "I")}
        self.env11 = _envs(self.mpo["H0"], self.phi1, self.phi1, self.positions)
        self.env10 = {kind: _envs(self.mpo[kind], self.phi1, self.phi0, self.positions) for kind in ("H", "I")}
        self.mpslcc = mpslcc

    def context(self, **kw):
        ctx = self.mpslcc.Context(device=0, **kw)
        ctx.build_mpo(self.c["h"], self.c["V"], self.c["n_alpha"] + self.c["n_beta"], 0)
        ctx.set_spaces(self.c["n_core"], self.c["n_active"])
        ctx.load_mps(0, self.phi0)
        ctx.load_mps(1, self.phi1)
        return ctx

    def oracle(self, op, l, psi):
        m = self.mpslcc
        if op == m.OP_H0_11:
            L, R = self.env11[l]
            return bs.sigma(self.mpo["H0"], self.phi1, self.phi1, l, psi, L, R)
        kind = "H" if op == m.OP_H_10 else "I"
        L, R = self.env10[kind][l]
        return bs.sigma(self.mpo[kind], self.phi1, self.phi0, l, psi, L, R)


_CASES = {}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def case(request, mpslcc):
    if request.param not in _CASES:
        _CASES.clear()
        _CASES[request.param] = Case(mpslcc, request.param)
    return _CASES[request.param]


def _errs(s, r):
    return (np.linalg.norm(s - r) / np.linalg.norm(r), np.abs(s - r).max() / np.abs(r).max())


def test_fp64_sigma_matches_blocksparse_oracle(mpslcc, case):
    """FP64 sigma of H0 on Phi1, of the H transition and of the overlap
    (ket = the frozen-class reference) at the middle and near the chain ends."""
    with case.context() as ctx:
        for l in case.positions:
            for op in (mpslcc.OP_H0_11, mpslcc.OP_H_10, mpslcc.OP_S_10):
                n_out, n_in = ctx.local_dim(l, op)
                psi = synth.random_vector(n_in, 1000 + 10 * l + op)
                s = ctx.apply_heff(l, op, psi)
                r = case.oracle(op, l, psi)
                assert len(s) == len(r) == n_out
                e2, emax = _errs(s, r)
                assert e2 <= FP64_RTOL and emax <= FP64_RTOL, (op, l, e2, emax)


# Relative 2-norm bounds of the tensor-core sigma at these sizes.  BF16X6
# products are exact in FP32, so its error is the FP32 accumulation of the
# phase-2 channel sum, K ~ 1e4 terms here: about sqrt(K) 2^-24 ~ 1e-5.
# BF16X3 drops the lo*lo product (about 2^-16 per term), TF32 and BF16 round
# each operand once (2^-11, 2^-9), and phase 1 stores its intermediate in
# the operand precision.
@pytest.mark.parametrize("prec,tol", [("BF16X3", 1e-4), ("BF16X6", 2e-5), ("TF32", 4e-3), ("BF16", 3e-2)])
def test_tensor_core_sigma_matches_blocksparse_oracle(mpslcc, case, prec, tol):
    """tcgen05 sigma (split-BF16, three-piece BF16, TF32 and plain BF16
    operands, FP32 accumulation) within each precision's bound of the FP64
    oracle, for the LCC matrix and the transition operator."""
    with case.context() as ctx:
        for l in case.positions:
            for op in (mpslcc.OP_H0_11, mpslcc.OP_H_10):
                _, n_in = ctx.local_dim(l, op)
                psi = synth.random_vector(n_in, 2000 + 10 * l + op)
                s = ctx.apply_heff(l, op, psi, prec=getattr(mpslcc, prec))
                e2, _ = _errs(s, case.oracle(op, l, psi))
                assert e2 <= tol, (prec, op, l, e2)


def test_tensor_core_environments_match_blocksparse_oracle(mpslcc, case):
    """Environments and fused operators built on the tensor cores (batched
    three-piece-BF16 FP64 emulation, as in mixed-precision sweeps) give a
    sigma within the emulation's accuracy of the FP64 oracle.  Each
    environment update is two products accumulated in FP32 over K up to a few
    thousand (about sqrt(K) 2^-24 ~ 4e-6 relative each); the middle position
    of a 24-orbital chain carries about 40 of them from both ends, hence a
    bound of 1e-4 (measured: 3e-5 at M1 = 1000)."""
    with case.context(tc_environments=True) as ctx:
        for l in case.positions:
            op = mpslcc.OP_H0_11
            _, n_in = ctx.local_dim(l, op)
            psi = synth.random_vector(n_in, 3000 + l)
            s = ctx.apply_heff(l, op, psi)
            e2, _ = _errs(s, case.oracle(op, l, psi))
            assert e2 <= 1e-4, (l, e2)
