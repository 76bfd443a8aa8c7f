"""Pins of the block-sparse oracle (O2) against the determinant-space oracle
(O1) and against invariants: O2 shares no code with O1's local problem
(dense isometry P, P^T O P) nor with the library, so agreement element by
element on every position, operator and bra/ket pairing pins its MPO signs,
channel bookkeeping, environment updates, contraction order and layout."""
import numpy as np
import pytest

import synth
from oracle import blocksparse as bs, fci, mps as omps


def _frozen(m):
    m = dict(m)
    m["masks"] = [tuple(sorted({key[1] for key in s})) for s in m["sites"]]
    return m


CASES = [  # k, n_alpha, n_beta, n_core, n_active, seed
    (4, 2, 2, 1, 2, 1),
    (5, 3, 2, 1, 2, 2),
    (6, 3, 3, 1, 3, 3),
    (6, 4, 2, 2, 2, 4),
]


@pytest.mark.parametrize("k,na,nb,nc,nact,seed", CASES)
def test_sigma_equals_dense_local_problem(k, na, nb, nc, nact, seed):
    h, V = synth.ab_initio(k, 6, seed=70 + seed)
    dets = fci.determinants(k, na, nb)
    H = fci.build_hamiltonian(h, V, dets)
    H0 = fci.fink_h0(H, dets, k, nc, nact)
    ops = {"H": H, "H0": H0, "U": H - H0, "I": None}
    mpos = {kind: bs.Mpo(h, V, kind, nc, nact) for kind in ops}
    ne, tsz = na + nb, na - nb
    phi1 = synth.random_mps(k, ne, tsz, M=24, seed=seed)
    other = synth.random_mps(k, ne, tsz, M=9, seed=seed + 10, isometric=False)
    ref = _frozen(synth.random_mps(k, ne, tsz, M=8, seed=seed + 20,
                                   masks=synth.site_masks(k, nc, nact, frozen=True)))
    for bra, ket in ((phi1, phi1), (phi1, other), (phi1, ref), (ref, ref)):
        for l in range(k - 1):
            _, _, nk = bs.local_blocks(ket, l)
            psi = synth.random_vector(nk, 5 + l)
            Pb, Pk = omps.isometry(bra, l, dets), omps.isometry(ket, l, dets)
            for kind, O in ops.items():
                s = bs.sigma(mpos[kind], bra, ket, l, psi)
                r = Pb.T @ (Pk @ psi) if O is None else Pb.T @ (O @ (Pk @ psi))
                err = np.linalg.norm(s - r) / max(np.linalg.norm(r), 1e-300)
                assert err < 1e-12, (kind, l, err)


def test_block_layout_matches_entry_layout():
    """Every entry (ia, a, s1, s2, ib, b) of O1's element-wise local layout
    sits where O2's block layout puts element (a, b) of block (ia, s1, s2, ib)."""
    m = synth.random_mps(6, 6, 0, M=20, seed=12, isometric=False)
    for l in range(5):
        entries, _ = omps.local_layout(m, l)
        _, blocks, n = bs.local_blocks(m, l)
        assert n == len(entries)
        for j, (ia, a, s1, s2, ib, b) in enumerate(entries):
            off, dr, ro, co, da, db = blocks[(ia, s1, s2, ib)]
            assert off + (ro + a) * dr + co + b == j


def test_full_environment_contraction_is_the_expectation_value():
    """Left environments carried to the last bond (and right environments to
    the first) give <bra|O|ket> of the determinant expansions (Eq. mps1)."""
    k, na, nb, nc, nact = 6, 3, 3, 1, 3
    h, V = synth.ab_initio(k, 6, seed=91)
    dets = fci.determinants(k, na, nb)
    H = fci.build_hamiltonian(h, V, dets)
    H0 = fci.fink_h0(H, dets, k, nc, nact)
    bra = synth.random_mps(k, 6, 0, M=16, seed=1, isometric=False)
    ket = synth.random_mps(k, 6, 0, M=11, seed=2, isometric=False)
    vb, vk = omps.to_vector(bra, dets), omps.to_vector(ket, dets)
    for kind, O in (("H", H), ("H0", H0), ("I", None)):
        mpo = bs.Mpo(h, V, kind, nc, nact)
        L = bs.boundary_left(mpo)
        for y in range(k):
            L = bs.update_left(mpo, L, bra, ket, y)
        R = bs.boundary_right(mpo)
        for y in range(k - 1, -1, -1):
            R = bs.update_right(mpo, R, bra, ket, y)
        want = vb @ vk if O is None else vb @ (O @ vk)
        assert abs(L[(0, 0)].ravel()[0] - want) < 1e-12 * max(1.0, abs(want))
        assert abs(R[(0, 0)].ravel()[0] - want) < 1e-12 * max(1.0, abs(want))


def test_sigma_hermitian_on_the_chain_workload():
    """<a|H_eff b> = <H_eff a|b> for the L=8 chain's H0 at every position."""
    c = synth.config(0)
    mpo = bs.Mpo(c["h"], c["V"], "H0", c["n_core"], c["n_active"])
    m = synth.random_mps(8, 8, 0, M=40, seed=4)
    for l in range(7):
        L, R = bs.environments(mpo, m, m, l)
        _, _, n = bs.local_blocks(m, l)
        a, b = synth.random_vector(n, 1), synth.random_vector(n, 2)
        ha = bs.sigma(mpo, m, m, l, a, L, R)
        hb = bs.sigma(mpo, m, m, l, b, L, R)
        assert abs(a @ hb - b @ ha) < 1e-13 * (1 + abs(a @ hb))


@pytest.mark.parametrize("cfg", [0, 3])
def test_mpo_bond_dimensions_equal_the_librarys(mpslcc, cfg):
    """O2's MPO and the library's label their channels the same way (one or
    two operators, left or right), so their bond dimensions per bond agree;
    checked on the L=8 chain and the 3-band workload (no GPU involved)."""
    c = synth.config(cfg)
    ctx = mpslcc.Context(device=-1)
    ctx.build_mpo(c["h"], c["V"], c["n_alpha"] + c["n_beta"], 0)
    ctx.set_spaces(c["n_core"], c["n_active"])
    for kind, which in (("H", mpslcc.MPO_H), ("H0", mpslcc.MPO_H0), ("U", mpslcc.MPO_U)):
        mpo = bs.Mpo(c["h"], c["V"], kind, c["n_core"], c["n_active"])
        assert list(ctx.mpo_bond_dims(which)) == mpo.bond_dims(), kind
    ctx.close()
