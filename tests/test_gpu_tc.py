"""Tensor-core (tcgen05) path: the GEMM kernel in isolation, the mixed
precision sigma vector, and mixed-precision LCC energies against FP64."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _tf32(x):
    """Operand as the tensor core reads it: FP32 with the low 13 mantissa bits dropped."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("m,n,k", [(128, 64, 64), (130, 144, 136), (300, 17, 500), (64, 256, 1000),
                                   (1000, 130, 130)])
@pytest.mark.parametrize("mode,ksplit", [(0, 1), (0, 3), (1, 1), (2, 1)])
def test_tc_gemm_bf16(mpslcc, m, n, k, mode, ksplit):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k))
    with mpslcc.Context(device=0) as ctx:
        C = ctx.debug_tc_gemm(A, B, prec=mpslcc.BF16, mode=mode, ksplit=ksplit)
    ref = _bf16(A) @ _bf16(B).T
    if mode == 1:
        ref = _bf16(ref)
        tol = 1e-2
    else:
        tol = 1e-5
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < tol, err


@pytest.mark.parametrize("m,n,k", [(128, 64, 32), (130, 144, 136), (257, 40, 700)])
def test_tc_gemm_tf32(mpslcc, m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k))
    with mpslcc.Context(device=0) as ctx:
        C = ctx.debug_tc_gemm(A, B, prec=mpslcc.TF32, mode=2)
    ref = _tf32(A) @ _tf32(B).T
    assert np.abs(C - ref).max() / np.abs(ref).max() < 1e-5


@pytest.mark.parametrize("m,n,k,mode", [(130, 144, 136, 2), (300, 40, 900, 0), (64, 256, 64, 2)])
def test_tc_gemm_split_bf16(mpslcc, m, n, k, mode):
    """Split-BF16 operands (hi*hi + hi*lo + lo*hi in FP32) are accurate to
    about 2^-16 relative, far beyond one BF16 rounding."""
    rng = np.random.default_rng(m + 2 * n + 3 * k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k))
    with mpslcc.Context(device=0) as ctx:
        C = ctx.debug_tc_gemm(A, B, prec=mpslcc.BF16X3, mode=mode, ksplit=2 if mode == 0 else 1)
    ref = A @ B.T
    assert np.abs(C - ref).max() / np.abs(ref).max() < 2e-5


@pytest.fixture(scope="module")
def case6(mpslcc):
    k = 6
    h, V = synth.ab_initio(k, 6, seed=77)
    ctx = mpslcc.Context(device=0)
    ctx.build_mpo(h, V, 6, 0)
    ctx.set_spaces(1, 3)
    ctx.load_mps(1, synth.random_mps(k, 6, 0, M=40, seed=1))
    yield ctx
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("BF16", 3e-2), ("TF32", 4e-3), ("BF16X3", 1e-4), ("BF16X6", 1e-6)])
def test_sigma_low_precision_close_to_fp64(mpslcc, case6, prec, tol):
    """BF16X6 (three BF16 parts, six products) is limited by the FP32
    accumulation, about 2^-24 per rounding."""
    for l in range(5):
        n, _ = case6.local_dim(l, mpslcc.OP_H0_11)
        psi = synth.random_vector(n, 9 + l)
        s64 = case6.apply_heff(l, mpslcc.OP_H0_11, psi)
        slp = case6.apply_heff(l, mpslcc.OP_H0_11, psi, prec=getattr(mpslcc, prec))
        err = np.linalg.norm(slp - s64) / np.linalg.norm(s64)
        assert err < tol, (l, err)


@pytest.mark.parametrize("prec,tol", [("BF16X3", 1e-6)])
def test_mixed_precision_lcc_matches_fp64(mpslcc, prec, tol):
    """Mixed-precision sweeps reach the oracle's E0, E2 and E3 to 1e-6 at exact
    bond dimension (L=8 chain).  The reference ends with an FP64 sweep; the
    local LCC solves refine split-BF16 (BF16X3) corrections against BF16X6
    residuals, so the first-order state is accurate to ~2^-24 relative, which
    E3 = <Phi1|U|Phi1> (first order in the state's error) needs."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_energies.json")))
    g = g["hubbard1d_L8_U4"]
    c = synth.config(0)
    with mpslcc.Context(device=0, prec=getattr(mpslcc, prec), tol=1e-10, refine_steps=12) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 3)
        ctx.lcc_sweep(256, 3)
        e = ctx.energy()
    assert abs(e["E0"] - g["E0"]) < 1e-8
    assert abs(e["E2"] - g["E2"]) < tol, (e["E2"], g["E2"])
    assert abs(e["E3"] - g["E3"]) < tol, (e["E3"], g["E3"])


def test_fp64_residuals_make_the_mixed_lcc_energies_fp64_accurate(mpslcc):
    """With opts.residual_fp64 the right-hand side, the refinement residuals,
    the environments and the fused operators are FP64, and only the inner
    solves run on the tensor cores (split BF16): iterative refinement then
    converges to the FP64 solution, so E2 and E3 meet the oracle to 1e-9 on
    the L=8 chain at exact bond dimension (BF16X6 residuals stop near
    2^-24 and give ~3e-7 for E3)."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_energies.json")))
    g = g["hubbard1d_L8_U4"]
    c = synth.config(0)
    with mpslcc.Context(device=0, prec=mpslcc.BF16X3, tol=1e-12, refine_steps=12, residual_fp64=True) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 3)
        ctx.lcc_sweep(256, 3)
        e = ctx.energy()
    assert abs(e["E0"] - g["E0"]) < 1e-8
    assert abs(e["E2"] - g["E2"]) < 1e-9, (e["E2"], g["E2"])
    assert abs(e["E3"] - g["E3"]) < 1e-9, (e["E3"], g["E3"])


@pytest.mark.parametrize("prec", ["BF16X3", "BF16X6", "TF32"])
def test_autotuner_tries_every_tile_cap_and_results_do_not_depend_on_it(mpslcc, prec):
    """Repeated products at one position: the tile-shape autotuner runs each
    sigma phase once with N tiles of at most 256, 128 and 64 rows (4 / 6 / 8
    or, split, 2 / 3 / 4 pipeline stages) on one CTA per SM and with 64 on
    two CTAs per SM, then keeps the fastest.  The K
    splits do not depend on the tile shape, so every product is the same to
    the last bit."""
    k = 6
    h, V = synth.ab_initio(k, 6, seed=77)
    with mpslcc.Context(device=0) as ctx:
        ctx.build_mpo(h, V, 6, 0)
        ctx.set_spaces(1, 3)
        ctx.load_mps(1, synth.random_mps(k, 6, 0, M=40, seed=1))
        l = 2
        n, _ = ctx.local_dim(l, mpslcc.OP_H0_11)
        psi = synth.random_vector(n, 77)
        outs = [ctx.apply_heff(l, mpslcc.OP_H0_11, psi, prec=getattr(mpslcc, prec)) for _ in range(5)]
        st = ctx.stats()
    for cap in ("n256", "n128", "n64", "n64x2"):
        assert st["tc_launches_" + cap] >= 2, (cap, st["tc_launches_" + cap])
    assert st["tune_trials"] == 8
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
