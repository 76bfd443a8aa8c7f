"""One-site local problem and sweeps (Implementation section: one tensor is
optimised at a time, the local problem of d M^2 entries), against the
oracle's dense one-site isometry P (oracle.mps.isometry1) and its energies."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import fci, lcc, mps as omps

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_energies.json")))


def _frozen(m):
    m = dict(m)
    m["masks"] = [tuple(sorted({key[1] for key in s})) for s in m["sites"]]
    return m


@pytest.fixture(scope="module")
def small(mpslcc):
    k, na, nb, nc, nact = 6, 3, 3, 1, 3
    h, V = synth.ab_initio(k, 6, seed=77)
    dets = fci.determinants(k, na, nb)
    H = fci.build_hamiltonian(h, V, dets)
    H0 = fci.fink_h0(H, dets, k, nc, nact)
    phi1 = synth.random_mps(k, 6, 0, M=24, seed=1)
    phi0 = _frozen(synth.random_mps(k, 6, 0, M=8, seed=2, masks=synth.site_masks(k, nc, nact, frozen=True)))
    ctx = mpslcc.Context(device=0)
    ctx.build_mpo(h, V, 6, 0)
    ctx.set_spaces(nc, nact)
    ctx.load_mps(0, phi0)
    ctx.load_mps(1, phi1)
    yield dict(ctx=ctx, k=k, dets=dets, H=H, H0=H0, phi0=phi0, phi1=phi1)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("BF16X3", 1e-4)])
def test_one_site_sigma_matches_dense_local_problem(mpslcc, small, prec, tol):
    c = small
    ctx, dets = c["ctx"], c["dets"]
    U = c["H"] - c["H0"]
    cases = [(mpslcc.OP_H0_11, c["phi1"], c["phi1"], c["H0"]), (mpslcc.OP_U_11, c["phi1"], c["phi1"], U),
             (mpslcc.OP_H_11, c["phi1"], c["phi1"], c["H"]), (mpslcc.OP_H0_00, c["phi0"], c["phi0"], c["H0"]),
             (mpslcc.OP_H_10, c["phi1"], c["phi0"], c["H"]), (mpslcc.OP_S_10, c["phi1"], c["phi0"], None)]
    for l in range(c["k"]):
        for op, bra, ket, O in cases:
            n_out, n_in = ctx.local_dim1(l, op)
            assert (n_out, n_in) == (len(omps.local_layout1(bra, l)), len(omps.local_layout1(ket, l)))
            psi = synth.random_vector(n_in, 500 + 10 * l + op)
            s = ctx.apply_heff1(l, op, psi, prec=getattr(mpslcc, prec))
            Pb, Pk = omps.isometry1(bra, l, dets), omps.isometry1(ket, l, dets)
            ref = Pb.T @ (Pk @ psi) if O is None else Pb.T @ (O @ (Pk @ psi))
            err = np.linalg.norm(s - ref) / np.linalg.norm(ref)
            assert err <= tol, (op, l, err)


def test_one_site_sweeps_reach_the_exact_energies(mpslcc):
    """L=8 chain: after one two-site sweep at the exact M1 = 256 the bond
    dimensions are exact, and one-site sweeps converge to the determinant-
    space E2 and E3."""
    g = GOLDEN["hubbard1d_L8_U4"]
    c = synth.config(0)
    with mpslcc.Context(device=0, tol=1e-12) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 3)
        ctx.lcc_sweep(256, 1)
        ctx.lcc_sweep_onesite(3)
        e = ctx.energy()
    assert abs(e["E2"] - g["E2"]) <= 1e-10, (e["E2"], g["E2"])
    assert abs(e["E3"] - g["E3"]) <= 1e-10, (e["E3"], g["E3"])


@pytest.mark.parametrize("prec", ["FP64", "BF16X3"])
def test_one_site_sweeps_at_truncated_bond_dimension(mpslcc, prec):
    """From two-site sweeps at M1 = 64, one-site sweeps do not raise the
    Hylleraas value, and the energies of the resulting states equal the
    oracle's evaluation of the exported states.  Bond dimensions never grow;
    they drop to the rank where the two-site truncation had kept zero-weight
    states to fill M (bond 1 holds at most 4 states of weight)."""
    c = synth.config(0)
    dets = fci.determinants(8, 4, 4)
    H = fci.build_hamiltonian(c["h"], c["V"], dets)
    H0 = fci.fink_h0(H, dets, 8, c["n_core"], c["n_active"])
    kw = dict(refine_steps=12) if prec != "FP64" else {}
    with mpslcc.Context(device=0, prec=getattr(mpslcc, prec), tol=1e-10, **kw) as ctx:
        ctx.build_mpo(c["h"], c["V"], 8, 0)
        ctx.set_spaces(c["n_core"], c["n_active"])
        ctx.dmrg_reference(16, 3)
        ctx.lcc_sweep(64, 2)
        J2 = ctx.energy()["E2"]
        dims2 = [sum(s[2] for s in b) for b in ctx.export_mps(1)["bonds"]]
        ctx.lcc_sweep_onesite(2)
        e = ctx.energy()
        p0, p1 = ctx.export_mps(0), ctx.export_mps(1)
    dims1 = [sum(s[2] for s in b) for b in p1["bonds"]]
    assert all(d1 <= d2 for d1, d2 in zip(dims1, dims2)), (dims1, dims2)
    assert dims1[4] == dims2[4] == 64
    assert e["E2"] <= J2 + 1e-9, (e["E2"], J2)
    o = lcc.state_energies(H, H0, omps.to_vector(p0, dets), omps.to_vector(p1, dets))
    assert abs(e["E2"] - o["E2"]) <= 1e-10 and abs(e["E3"] - o["E3"]) <= 1e-10
