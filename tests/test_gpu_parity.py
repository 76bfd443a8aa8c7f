"""GPU parity: the C-ABI library against the CPU oracle on seeded inputs."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import fci, lcc, mps as omps

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_energies.json")))
SIGMA_RTOL = 1e-12     # FP64 sigma vs dense oracle (relative, 2-norm)
ENERGY_TOL = 1e-10     # |dE| at exact bond dimension


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _masks_from_blocks(m):
    m = dict(m)
    m["masks"] = [tuple(sorted({key[1] for key in s})) for s in m["sites"]]
    return m


@pytest.fixture(scope="module")
def small_case(mpslcc):
    k, na, nb, nc, nact = 6, 3, 3, 1, 3
    h, V = synth.ab_initio(k, 6, seed=77)
    dets = fci.determinants(k, na, nb)
    H = fci.build_hamiltonian(h, V, dets)
    H0 = fci.fink_h0(H, dets, k, nc, nact)
    phi1 = synth.random_mps(k, na + nb, 0, M=24, seed=1)
    phi0 = _masks_from_blocks(synth.random_mps(k, na + nb, 0, M=8, seed=2,
                                               masks=synth.site_masks(k, nc, nact, frozen=True)))
    ctx = mpslcc.Context(device=0)
    ctx.build_mpo(h, V, na + nb, 0)
    ctx.set_spaces(nc, nact)
    ctx.load_mps(0, phi0)
    ctx.load_mps(1, phi1)
    yield dict(ctx=ctx, k=k, dets=dets, H=H, H0=H0, U=H - H0, phi0=phi0, phi1=phi1)
    ctx.close()


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_sigma_matches_dense_local_problem(mpslcc, small_case, l):
    """sigma = P^T O P psi (Implementation section, Fig. 3) for O = H0, U, H
    on Phi1 and H0 on Phi0, against the oracle's dense effective operator."""
    c = small_case
    ctx, dets = c["ctx"], c["dets"]
    cases = [(mpslcc.OP_H0_11, c["phi1"], c["phi1"], c["H0"]),
             (mpslcc.OP_U_11, c["phi1"], c["phi1"], c["U"]),
             (mpslcc.OP_H_11, c["phi1"], c["phi1"], c["H"]),
             (mpslcc.OP_H0_00, c["phi0"], c["phi0"], c["H0"]),
             (mpslcc.OP_H_10, c["phi1"], c["phi0"], c["H"]),
             (mpslcc.OP_S_10, c["phi1"], c["phi0"], None)]
    for op, bra, ket, O in cases:
        n_out, n_in = ctx.local_dim(l, op)
        eb, _ = omps.local_layout(bra, l)
        ek, _ = omps.local_layout(ket, l)
        assert (n_out, n_in) == (len(eb), len(ek))
        psi = synth.random_vector(n_in, seed=100 + 10 * l + op)
        sig = ctx.apply_heff(l, op, psi)
        Pb = omps.isometry(bra, l, dets)
        Pk = omps.isometry(ket, l, dets)
        ref = Pb.T @ (Pk @ psi) if O is None else Pb.T @ (O @ (Pk @ psi))
        assert _rel(sig, ref) <= SIGMA_RTOL, (op, l, _rel(sig, ref))


def test_sigma_hermitian(mpslcc, small_case):
    ctx = small_case["ctx"]
    for l in (0, 2, 4):
        n, _ = ctx.local_dim(l, mpslcc.OP_H0_11)
        a = synth.random_vector(n, 5)
        b = synth.random_vector(n, 6)
        ha = ctx.apply_heff(l, mpslcc.OP_H0_11, a)
        hb = ctx.apply_heff(l, mpslcc.OP_H0_11, b)
        assert abs(a @ hb - b @ ha) <= 1e-13 * (abs(a @ hb) + 1)


def test_config0_energies_at_exact_bond_dimension(mpslcc):
    """L=8 Hubbard chain in sine modes, (4e,4o) reference: M0 = 16 and
    M1 = 256 are exact, so E0, E2 and E3 equal the determinant-space values."""
    g = GOLDEN["hubbard1d_L8_U4"]
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-11) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        E0 = ctx.dmrg_reference(16, 3)
        assert abs(E0 - g["E0"]) <= ENERGY_TOL
        ctx.lcc_sweep(256, 3)
        e = ctx.energy()
    assert abs(e["E0"] - g["E0"]) <= ENERGY_TOL
    assert abs(e["E2"] - g["E2"]) <= ENERGY_TOL, (e["E2"], g["E2"])
    assert abs(e["E3"] - g["E3"]) <= ENERGY_TOL, (e["E3"], g["E3"])
    assert abs(e["overlap01"]) <= 1e-8


def test_product_start_reaches_exact_reference(mpslcc):
    """Starting the reference from the lowest-h_pp determinant (a bond
    dimension 1 product state), two-site sweeps grow the bonds to the exact
    M0 = 16 and reach the determinant-space E0 of the L=8 chain."""
    g = GOLDEN["hubbard1d_L8_U4"]
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-11, init_guess=1) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        E0 = ctx.dmrg_reference(16, 4)
    assert abs(E0 - g["E0"]) <= ENERGY_TOL, (E0, g["E0"])


def test_resume_from_exported_states(mpslcc):
    """Exported Phi0 and Phi1 load into a fresh context (a checkpoint): zero
    reference sweeps re-evaluate E0, and further LCC sweeps from the loaded
    first-order state reach the determinant-space energies."""
    g = GOLDEN["hubbard1d_L8_U4"]
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-11) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        E0 = ctx.dmrg_reference(16, 3)
        ctx.lcc_sweep(256, 1)
        p0, p1 = ctx.export_mps(0), ctx.export_mps(1)
    with mpslcc.Context(device=0, tol=1e-11) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.load_mps(0, p0)
        assert abs(ctx.dmrg_reference(16, 0) - E0) <= 1e-12
        ctx.load_mps(1, p1)
        ctx.lcc_sweep(256, 2)
        e = ctx.energy()
    assert abs(e["E2"] - g["E2"]) <= ENERGY_TOL, (e["E2"], g["E2"])
    assert abs(e["E3"] - g["E3"]) <= ENERGY_TOL, (e["E3"], g["E3"])


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (1.0, 1.0)])
def test_dimer_lcc_closed_form(mpslcc, t, U):
    """E0 = -2t + U/2, E2 = -U^2/(16t), E3 = 0 for the bonding/antibonding
    dimer with no active orbitals."""
    h, V = synth.hubbard_dimer(t, U, orbital_basis=True)
    with mpslcc.Context(device=0, tol=1e-12) as ctx:
        ctx.build_mpo(h, V, 2, 0)
        ctx.set_spaces(1, 0)
        ctx.dmrg_reference(4, 2)
        ctx.lcc_sweep(16, 2)
        e = ctx.energy()
    assert abs(e["E0"] - (-2 * t + U / 2)) <= 1e-12
    assert abs(e["E2"] + U * U / (16 * t)) <= 1e-11
    assert abs(e["E3"]) <= 1e-11


def test_full_active_space_gives_fci(mpslcc):
    """All orbitals active: the reference is FCI, E2 = E3 = 0."""
    h, V = synth.ab_initio(5, 6, seed=3)
    Efci, _, _, _ = fci.fci(h, V, 2, 2)
    with mpslcc.Context(device=0, tol=1e-12) as ctx:
        ctx.build_mpo(h, V, 4, 0)
        ctx.set_spaces(0, 5)
        E0 = ctx.dmrg_reference(64, 3)
        ctx.lcc_sweep(64, 2)
        e = ctx.energy()
    assert abs(E0 - Efci) <= 1e-10
    assert abs(e["E2"]) <= 1e-10 and abs(e["E3"]) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("BF16X3", 1e-4), ("BF16X6", 4e-6)])
def test_sigma_low_precision_all_operators(mpslcc, small_case, prec, tol):
    """The split-BF16 tensor-core sigma of every operator family (including the
    transition and overlap ones, whose bra and ket differ) stays within the
    split's accuracy of the FP64 sigma."""
    ctx = small_case["ctx"]
    for l in range(5):
        for op in (mpslcc.OP_H0_11, mpslcc.OP_U_11, mpslcc.OP_H_11, mpslcc.OP_H0_00, mpslcc.OP_H_10,
                   mpslcc.OP_S_10):
            n_out, n_in = ctx.local_dim(l, op)
            psi = synth.random_vector(n_in, seed=300 + 10 * l + op)
            s64 = ctx.apply_heff(l, op, psi)
            slp = ctx.apply_heff(l, op, psi, prec=getattr(mpslcc, prec))
            assert _rel(slp, s64) <= tol, (op, l, _rel(slp, s64))
