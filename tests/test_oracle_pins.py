"""Pins of the CPU oracle against closed forms, limits, invariants and brute
force -- none of them re-types the oracle's own formulas."""
import math

import numpy as np
import pytest

import synth
from oracle import fci, fock, lcc, mps as omps


def _sym_integrals(k, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((k, k))
    h = 0.5 * (h + h.T)
    V = np.zeros((k, k, k, k))
    for _ in range(3):
        B = rng.standard_normal((k, k)) * scale
        B = 0.5 * (B + B.T)
        V += np.einsum("ij,kl->ijkl", B, B)
    return h, V


def test_determinant_count():
    # C(8,4)^2 = 4900 determinants for the L=8 half-filled chain
    assert len(fci.determinants(8, 4, 4)) == 4900


@pytest.mark.parametrize("k,na,nb", [(2, 1, 1), (3, 2, 1), (4, 2, 2)])
def test_hamiltonian_matches_qubit_jordan_wigner(k, na, nb):
    """Element-by-element agreement with the qubit-JW Fock-space matrix."""
    h, V = _sym_integrals(k, 11 + k)
    dets = fci.determinants(k, na, nb)
    H = fci.build_hamiltonian(h, V, dets).toarray()
    F = fock.fock_hamiltonian(h, V)
    idx = [fock.qubit_index(int(d), 2 * k) for d in dets]
    Fs = F[idx][:, idx].toarray()
    np.testing.assert_allclose(H, Fs, atol=1e-12, rtol=0)
    # the Fock matrix does not mix (N, Sz) sectors
    assert abs(F - F.T).max() < 1e-12


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (1.0, 8.0), (0.5, 1.0)])
@pytest.mark.parametrize("orbital_basis", [False, True])
def test_hubbard_dimer_closed_form(t, U, orbital_basis):
    """Half-filled two-site Hubbard ground state: E = (U - sqrt(U^2+16t^2))/2."""
    h, V = synth.hubbard_dimer(t, U, orbital_basis)
    E, _, _, _ = fci.fci(h, V, 1, 1)
    assert abs(E - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_free_fermions():
    """U = 0: ground energy = sum of the lowest orbital energies per spin."""
    h, V = synth.hubbard_chain(6, 1.0, 0.0)
    E, _, _, _ = fci.fci(h, V, 3, 2)
    w = np.linalg.eigvalsh(h)
    assert abs(E - (w[:3].sum() + w[:2].sum())) < 1e-12


def test_atomic_limit():
    """t = 0 at half filling: every site singly occupied, E = 0."""
    h, V = synth.hubbard_chain(4, 0.0, 5.0)
    E, _, _, _ = fci.fci(h, V, 2, 2)
    assert abs(E) < 1e-12


def test_h0_term_filter_equals_class_mask():
    """Delta n_ex = 0 term selection == excitation-class block mask."""
    h, V = _sym_integrals(5, 3)
    k, nc, na = 5, 1, 2
    dets = fci.determinants(k, 2, 2)
    H = fci.build_hamiltonian(h, V, dets)
    H0_mask = fci.fink_h0(H, dets, k, nc, na).toarray()
    H0_terms = fci.build_hamiltonian(h, V, dets, fci.delta_nex_zero(k, nc, na)).toarray()
    np.testing.assert_allclose(H0_mask, H0_terms, atol=1e-12, rtol=0)
    assert abs(H0_mask).sum() < abs(H.toarray()).sum()


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (1.0, 1.0), (2.0, 3.0)])
def test_lcc_dimer_closed_form(t, U):
    """Bonding/antibonding dimer with no active orbitals: E0 = -2t + U/2,
    E(2) = -U^2/(16 t), E(3) = 0 (derived by hand: <D|H|HF> = U/2,
    E_D - E_HF = 4t, the singles have no right-hand side by parity)."""
    h, V = synth.hubbard_dimer(t, U, orbital_basis=True)
    r = lcc.lcc_energies(h, V, 1, 1, n_core=1, n_active=0)
    assert abs(r["E0"] - (-2 * t + U / 2)) < 1e-12
    assert abs(r["E2"] - (-U * U / (16 * t))) < 1e-12
    assert abs(r["E3"]) < 1e-12
    assert abs(r["J"] - r["E2"]) < 1e-12


def test_lcc_full_active_is_fci():
    """All orbitals active: the reference is FCI and E(2) = E(3) = 0."""
    h, V = _sym_integrals(4, 5)
    r = lcc.lcc_energies(h, V, 2, 2, n_core=0, n_active=4)
    assert abs(r["E0"] - r["Efci"]) < 1e-12
    assert abs(r["E2"]) < 1e-12 and abs(r["E3"]) < 1e-12


@pytest.mark.parametrize("k,nc", [(4, 2), (5, 2)])
def test_single_reference_limit(k, nc):
    """No active orbitals: the class-based solve equals an explicitly
    enumerated singles+doubles solve, and differs from textbook LCCSD
    (which keeps the S-D coupling)."""
    h, V = synth.ab_initio(k, 6, seed=41 + k)
    r = lcc.lcc_energies(h, V, nc, nc, n_core=nc, n_active=0)
    s = lcc.single_reference_lcc(h, V, nc)
    assert abs(r["E0"] - s["E0"]) < 1e-12
    assert abs(r["E2"] - s["E2"]) < 1e-12
    assert abs(r["E3"] - s["E3"]) < 1e-12
    assert abs(s["E2_lccsd"] - s["E2"]) > 1e-9


def test_wigner_rule_matches_direct_energies():
    """Eq. 2 (Wigner 2n+1) energies equal the direct E(n+1) = <Phi0|U|Phi(n)>."""
    c = synth.config(0)
    h, V = synth.hubbard_chain(6, 1.0, 2.0)
    eps, h, V = synth.to_orbital_basis(h, V)
    k = 6
    dets = fci.determinants(k, 3, 3)
    H = fci.build_hamiltonian(h, V, dets)
    H0 = fci.fink_h0(H, dets, k, 1, 4)
    E0, phi0 = fci.cas_ci(H, dets, k, 1, 4)
    r = lcc.rspt(H, H0, phi0, 3, dets, k, 1, 4)
    E, Ed = r["E"], r["Edirect"]
    assert abs(E[0] - E0) < 1e-12
    assert abs(E[1]) < 1e-12
    for n in range(1, 4):
        assert abs(E[n + 1] - Ed[n]) < 1e-10, (n, E[n + 1], Ed[n])
    # the series approaches FCI
    Efci, _ = fci.lowest_eigenpair(H)
    partial = np.cumsum(E)
    assert abs(partial[-1] - Efci) < abs(partial[1] - Efci)


def test_config0_reference_class_and_energies():
    """Config 0 (L=8 chain, sine modes): orbital energies are the closed-form
    -2 cos(pi m / 9); the reference class has C(4,2)^2 = 36 determinants."""
    c = synth.config(0)
    np.testing.assert_allclose(np.diag(c["h"]), c["eps"], atol=1e-12)
    assert abs(c["h"] - np.diag(np.diag(c["h"]))).max() < 1e-12
    dets = fci.determinants(8, 4, 4)
    idx = fci.reference_class_indices(dets, 8, 2, 4)
    assert len(idx) == 36


def test_isometry_complete_basis_spectrum():
    """At l=0 with a complete right-canonical basis P is unitary on the
    (N, Sz) space, so H_eff has the FCI spectrum."""
    k = 4
    h, V = _sym_integrals(k, 9)
    m = synth.random_mps(k, 4, 0, M=10 ** 6, seed=3)
    dets = fci.determinants(k, 2, 2)
    H = fci.build_hamiltonian(h, V, dets)
    P = omps.isometry(m, 0, dets)
    assert P.shape[0] == P.shape[1] == len(dets)
    np.testing.assert_allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-12)
    Heff = omps.effective_hamiltonian(m, 0, H, dets)
    np.testing.assert_allclose(np.linalg.eigvalsh(Heff),
                               np.linalg.eigvalsh(H.toarray()), atol=1e-11)


def test_isometry_reproduces_mps_vector():
    """P psi_local equals the full expansion of the MPS (Eq. mps1)."""
    k, l = 5, 2
    m = synth.random_mps(k, 5, 1, M=12, seed=8, isometric=False)
    dets = fci.determinants(k, 3, 2)
    full = omps.to_vector(m, dets)
    entries, _ = omps.local_layout(m, l)
    # contract sites l, l+1 into the local layout
    A, B = m["sites"][l], m["sites"][l + 1]
    psi = np.zeros(len(entries))
    for j, (ia, a, s1, s2, ib, b) in enumerate(entries):
        tot = 0.0
        for (x, s, y), blk in A.items():
            if x == ia and s == s1 and (y, s2, ib) in B:
                tot += blk[a] @ B[(y, s2, ib)][:, b]
        psi[j] = tot
    P = omps.isometry(m, l, dets)
    np.testing.assert_allclose(P @ psi, full, atol=1e-12)


def test_energy_formulas_hold_for_states_not_orthogonal_to_the_reference():
    """The energies are evaluated from overlaps of an MPS Phi1 that need not be
    exactly orthogonal to Phi0.  With s = <1|0> and Q Phi1 = Phi1 - s Phi0:
      J(Q Phi1)  = <1|H0|1> - E0 <1|1> - 2 s (<1|H0|0> - E0 s) + 2 (<1|H|0> - s E0),
      E3(Q Phi1) = <1|U|1> - 2 s (<1|H|0> - <1|H0|0>)      (<0|U|0> = 0).
    Checked against the definitions applied to Q Phi1 for the exact first-order
    state plus a reference admixture and plus a random perturbation."""
    c = synth.config(0)
    r = lcc.lcc_energies(c["h"], c["V"], 4, 4, c["n_core"], c["n_active"])
    H, H0, phi0, E0, x, b = (r["H"].toarray(), r["H0"].toarray(), r["phi0"], r["E0"], r["x"], r["b"])
    U = H - H0
    assert abs(phi0 @ U @ phi0) < 1e-12
    rng = np.random.default_rng(5)
    A = H0 - E0 * np.eye(len(phi0))
    for phi1 in (x + 0.3 * phi0, x + 0.01 * rng.standard_normal(len(x))):
        s = phi1 @ phi0
        q = phi1 - s * phi0
        J_def = q @ A @ q - 2.0 * (q @ b)
        E3_def = q @ U @ q
        J_form = (phi1 @ H0 @ phi1 - E0 * (phi1 @ phi1) - 2 * s * (phi1 @ H0 @ phi0 - E0 * s)
                  + 2 * (phi1 @ H @ phi0 - s * E0))
        E3_form = phi1 @ U @ phi1 - 2 * s * (phi1 @ H @ phi0 - phi1 @ H0 @ phi0)
        assert abs(J_form - J_def) < 1e-11
        assert abs(E3_form - E3_def) < 1e-11
    assert abs(r["J"] - r["E2"]) < 1e-12


def test_first_order_e3_equals_direct_third_order_energy():
    """E3 of the first-order solve (Eq. 2, n = 1: <Phi1|U|Phi1>) equals the
    third-order energy computed the other way, <Phi0|U|Phi(2)>, from the
    second-order wavefunction of the Eq. 1 recursion; E2 likewise equals
    <Phi0|U|Phi(1)> and the Wigner E(2), E(3).  A dropped term, sign or factor
    in first_order's E3 changes one side only."""
    c = synth.config(0)
    k = 8
    dets = fci.determinants(k, 4, 4)
    H = fci.build_hamiltonian(c["h"], c["V"], dets)
    H0 = fci.fink_h0(H, dets, k, c["n_core"], c["n_active"])
    E0, phi0 = fci.cas_ci(H, dets, k, c["n_core"], c["n_active"])
    r1 = lcc.first_order(H, H0, phi0, E0, dets, k, c["n_core"], c["n_active"])
    rs = lcc.rspt(H, H0, phi0, 2, dets, k, c["n_core"], c["n_active"])
    assert abs(r1["E2"] - rs["Edirect"][1]) < 1e-10
    assert abs(r1["E3"] - rs["Edirect"][2]) < 1e-10, (r1["E3"], rs["Edirect"][2])
    assert abs(r1["E3"] - rs["E"][3]) < 1e-10
    assert abs(r1["E3"]) > 1e-3  # a non-trivial third-order energy


def test_state_energies_at_the_solution_and_invariances():
    """Energies of given states: at the exact first-order vector they are the
    solve's E2 (= J) and E3; adding any multiple of Phi0 to Phi1 or rescaling
    Phi0 changes nothing (Q projects the reference out); Phi1 = Phi0 gives
    J = E3 = 0; and off the solution J exceeds E2 by exactly the quadratic
    form <d|A|d> of the Q-space deviation d (A positive definite here)."""
    c = synth.config(0)
    r = lcc.lcc_energies(c["h"], c["V"], 4, 4, c["n_core"], c["n_active"])
    H, H0, phi0, x = r["H"], r["H0"], r["phi0"], r["x"]
    e = lcc.state_energies(H, H0, phi0, x)
    assert abs(e["E0"] - r["E0"]) < 1e-12
    assert abs(e["J"] - r["E2"]) < 1e-11 and abs(e["E3"] - r["E3"]) < 1e-11
    assert abs(e["overlap01"]) < 1e-12
    e2 = lcc.state_energies(H, H0, 2.0 * phi0, x - 0.7 * phi0)
    assert abs(e2["J"] - e["J"]) < 1e-11 and abs(e2["E3"] - e["E3"]) < 1e-11
    assert abs(e2["overlap01"] + 0.7) < 1e-12
    e3 = lcc.state_energies(H, H0, phi0, phi0)
    assert abs(e3["J"]) < 1e-12 and abs(e3["E3"]) < 1e-12
    rng = np.random.default_rng(3)
    Hd, H0d = H.toarray(), H0.toarray()
    A = H0d - r["E0"] * np.eye(len(phi0))
    for _ in range(3):
        d = 1e-2 * rng.standard_normal(len(x))
        d -= phi0 * (phi0 @ d)
        ed = lcc.state_energies(H, H0, phi0, x + d)
        assert ed["J"] > r["E2"]
        assert abs((ed["J"] - r["E2"]) - d @ A @ d) < 1e-12


def test_one_site_isometry_reproduces_mps_vector():
    """P1 psi with psi = the site tensor of l in the one-site layout equals
    the full expansion of the MPS (Eq. mps1) at every site."""
    k = 5
    m = synth.random_mps(k, 5, 1, M=12, seed=8, isometric=False)
    dets = fci.determinants(k, 3, 2)
    full = omps.to_vector(m, dets)
    for l in range(k):
        entries = omps.local_layout1(m, l)
        psi = np.array([m["sites"][l][(ia, s, ib)][a, b] if (ia, s, ib) in m["sites"][l] else 0.0
                        for (ia, a, s, ib, b) in entries])
        P = omps.isometry1(m, l, dets)
        np.testing.assert_allclose(P @ psi, full, atol=1e-12)
