"""Fink-partitioned perturbation theory / MPS-LCC energies (oracle).

* Eq. 1 (Rayleigh-Schroedinger recursion): (H0 - E(0)) Phi(n) =
  Q(-U Phi(n-1) + sum_{k=1..n} E(k) Phi(n-k)), P = |Phi0><Phi0|, Q = 1 - P.
* "Projector approximation" paragraph: with an approximate Phi0 the zeroth
  order operator becomes H0~ = P H0 P + Q H0 Q and U~ = P H0 Q + Q H0 P + U;
  the first-order equation becomes (H0 - E0) Phi(1) = -Q H Phi(0) on the
  Q space, and E(2) = <Phi(0)|H|Phi(1)>.  The minus sign on the right-hand
  side follows Eq. 1 (the paragraph prints it without the sign).
* Eq. 2 (Wigner 2n+1 rule) for E(2n), E(2n+1).
* Eq. 1b (Hylleraas functional), read consistently with Eq. 1 as
  J(x) = <x|A|x> - 2<x|b>, A = Q(H0 - E0)Q, b = -Q H Phi0; J_min = E(2).

Everything is dense FP64 linear algebra in the determinant basis.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fci


def _dense(M):
    return M.toarray() if sp.issparse(M) else np.asarray(M)


def _solve_q(A, phi0, rhs, idx):
    """Solve Q A Q x = rhs (rhs orthogonal to phi0) on index set idx, with
    x orthogonal to phi0, via the nonsingular (Q A Q + P) on that set."""
    Ai = A[np.ix_(idx, idx)]
    f = phi0[idx]
    Af = Ai @ f
    fAf = f @ Af
    M = Ai - np.outer(f, Af) - np.outer(Af, f) + (fAf + 1.0) * np.outer(f, f)
    x = np.zeros(len(phi0))
    x[idx] = np.linalg.solve(M, rhs[idx])
    return x


def _active_index(rhs, dets, n_orb, n_core, n_active, phi0, tol=1e-13):
    """Determinants of the excitation classes that carry right-hand side or
    the reference; other classes decouple under H0 and stay zero."""
    nc, nv = fci.excitation_class(dets, n_orb, n_core, n_active)
    cls = nc * 1000 + nv
    keep = set(np.unique(cls[np.abs(rhs) > tol]).tolist())
    keep |= set(np.unique(cls[np.abs(phi0) > tol]).tolist())
    return np.nonzero(np.isin(cls, list(keep)))[0]


def first_order(H, H0, phi0, E0, dets, n_orb, n_core, n_active):
    """First-order wavefunction and energies (Eq. 1 with n=1, projector form).

    Returns dict(x, b, E2, E3, J, norm2) where
      b  = -Q H Phi0,
      x solves Q (H0 - E0) Q x = b, x orthogonal to Phi0,
      E2 = <Phi0|H|x>           (projector-form second-order energy),
      E3 = <x|H - H0|x>         (Eq. 2 with n=1, E(1)=0),
      J  = <x|A|x> - 2<x|b>     (Hylleraas value; equals E2 at the solution).
    """
    Hd = _dense(H)
    H0d = _dense(H0)
    n = Hd.shape[0]
    b = -(Hd @ phi0)
    b -= phi0 * (phi0 @ b)
    A = H0d - E0 * np.eye(n)
    idx = _active_index(b, dets, n_orb, n_core, n_active, phi0)
    x = _solve_q(A, phi0, b, idx)
    Q = lambda v: v - phi0 * (phi0 @ v)
    Ax = Q(A @ Q(x))
    E2 = phi0 @ (Hd @ x)
    E3 = x @ ((Hd - H0d) @ x)
    J = x @ Ax - 2.0 * (x @ b)
    return dict(x=x, b=b, E2=E2, E3=E3, J=J, norm2=x @ x)


def state_energies(H, H0, phi0, phi1):
    """Energies of GIVEN states, as the definitions state them (Eq. 1b read
    consistently with Eq. 1, and Eq. 2 with n = 1), for a reference phi0 and a
    first-order vector phi1 that need not be optimal nor orthogonal to phi0
    (an MPS of finite bond dimension is neither):
      E0 = <phi0|H|phi0> / <phi0|phi0>,
      q  = Q phi1 with Q = 1 - |phi0><phi0| (phi0 normalised),
      b  = -Q H phi0,
      J  = <q|(H0 - E0)|q> - 2 <q|b>          (Hylleraas value of q),
      E3 = <q|H - H0|q>,
      s  = <phi1|phi0>, norm1 = <phi1|phi1>.
    """
    Hd = _dense(H)
    H0d = _dense(H0)
    f = np.asarray(phi0, dtype=float)
    f = f / np.linalg.norm(f)
    E0 = f @ (Hd @ f)
    s = float(np.asarray(phi1) @ f)
    q = np.asarray(phi1, dtype=float) - s * f
    b = -(Hd @ f)
    b = b - f * (f @ b)
    J = q @ (H0d @ q) - E0 * (q @ q) - 2.0 * (q @ b)
    E3 = q @ ((Hd - H0d) @ q)
    return dict(E0=E0, J=J, E2=J, E3=E3, overlap01=s, norm1=float(np.asarray(phi1) @ np.asarray(phi1)))


def lcc_energies(h, V, n_alpha, n_beta, n_core, n_active):
    """E0 (CAS-CI reference), E2, E3 and FCI for a small Hamiltonian."""
    k = h.shape[0]
    dets = fci.determinants(k, n_alpha, n_beta)
    H = fci.build_hamiltonian(h, V, dets)
    H0 = fci.fink_h0(H, dets, k, n_core, n_active)
    E0, phi0 = fci.cas_ci(H, dets, k, n_core, n_active)
    r = first_order(H, H0, phi0, E0, dets, k, n_core, n_active)
    Efci, _ = fci.lowest_eigenpair(H)
    r.update(E0=E0, phi0=phi0, Efci=Efci, dets=dets, H=H, H0=H0)
    return r


def rspt(H, H0, phi0, nmax, dets, n_orb, n_core, n_active):
    """Perturbation series to order nmax with H0~ / U~ of the projector
    approximation (exact H0 partition when phi0 is an eigenvector of H0).

    Returns dict(E=list of E(0..2*nmax+1) via Wigner, Edirect=list of
    E(n+1) = <Phi0|U~|Phi(n)>, Phi=list of Phi(n))."""
    Hd = _dense(H)
    H0d = _dense(H0)
    n = Hd.shape[0]
    P = np.outer(phi0, phi0)
    Qm = np.eye(n) - P
    H0t = P @ H0d @ P + Qm @ H0d @ Qm
    Ut = Hd - H0t
    E0 = phi0 @ H0d @ phi0
    E = {0: E0, 1: phi0 @ Ut @ phi0}
    Phi = [phi0]
    A = H0t - E0 * np.eye(n)
    idx = np.arange(n)
    for m in range(1, nmax + 1):
        rhs = -Ut @ Phi[m - 1]
        for kk in range(1, m + 1):
            rhs = rhs + E[kk] * Phi[m - kk]
        rhs = rhs - phi0 * (phi0 @ rhs)
        x = _solve_q(A, phi0, rhs, idx)
        Phi.append(x)
        # Wigner 2n+1 energies from Phi(m) (Eq. 2)
        e2n = Phi[m - 1] @ Ut @ Phi[m]
        for kk in range(1, m + 1):
            for j in range(1, m):
                e2n -= E[2 * m - kk - j] * (Phi[kk] @ Phi[j])
        E[2 * m] = e2n
        e2n1 = Phi[m] @ Ut @ Phi[m]
        for kk in range(1, m + 1):
            for j in range(1, m + 1):
                e2n1 -= E[2 * m + 1 - kk - j] * (Phi[kk] @ Phi[j])
        E[2 * m + 1] = e2n1
    Edirect = [phi0 @ Ut @ Phi[m] for m in range(len(Phi))]
    return dict(E=[E[i] for i in sorted(E)], Edirect=Edirect, Phi=Phi)


# ----------------------------------------------------------------------------
# single-reference limit (zero active orbitals), explicit singles + doubles
# ----------------------------------------------------------------------------
def singles_doubles_space(n_orb: int, n_core: int):
    """Hartree-Fock determinant (core orbitals doubly occupied) and its
    singles and doubles, enumerated by explicit excitation (spin conserving)."""
    occ = [2 * p + s for p in range(n_core) for s in (0, 1)]
    vir = [2 * p + s for p in range(n_core, n_orb) for s in (0, 1)]
    hf = 0
    for j in occ:
        hf |= 1 << j
    singles, doubles = set(), set()
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                singles.add(hf ^ (1 << i) ^ (1 << a))
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(vir):
                for b in vir[aa + 1:]:
                    if (i % 2 + j % 2) == (a % 2 + b % 2):
                        doubles.add(hf ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << b))
    return hf, sorted(singles), sorted(doubles)


def single_reference_lcc(h, V, n_core):
    """Eq. 1 at n=1 with no active orbitals, written directly in the singles
    and doubles space: each excitation level L is solved separately,
    (H_LL - E_HF) x_L = -H_{L,HF}, since Fink's H0 does not couple levels.

    Returns dict(E0, E2, E3) and the textbook LCCSD energy of Eq. lccT
    (singles-doubles coupling kept) as ``E2_lccsd`` for comparison."""
    k = h.shape[0]
    hf, S, D = singles_doubles_space(k, n_core)
    space = np.array(sorted([hf] + S + D), dtype=np.int64)
    H = _dense(fci.build_hamiltonian(h, V, space))
    pos = {int(d): i for i, d in enumerate(space)}
    i0 = pos[hf]
    E0 = H[i0, i0]
    x = np.zeros(len(space))
    for level in (S, D):
        idx = np.array([pos[d] for d in level], dtype=np.int64)
        if len(idx) == 0:
            continue
        A = H[np.ix_(idx, idx)] - E0 * np.eye(len(idx))
        x[idx] = np.linalg.solve(A, -H[idx, i0])
    E2 = H[i0] @ x
    # H0 is block diagonal by level: U x has only off-level blocks
    lev = np.zeros(len(space), dtype=np.int64)
    for d in S:
        lev[pos[d]] = 1
    for d in D:
        lev[pos[d]] = 2
    H0 = H * (lev[:, None] == lev[None, :])
    E3 = x @ ((H - H0) @ x)
    sd = np.array([pos[d] for d in S + D], dtype=np.int64)
    A = H[np.ix_(sd, sd)] - E0 * np.eye(len(sd))
    y = np.linalg.solve(A, -H[sd, i0])
    return dict(E0=E0, E2=E2, E3=E3, E2_lccsd=H[i0, sd] @ y)
