"""Determinant-space Hamiltonian, Fink partition and full CI (oracle).

Follows the Theory section of Sharma & Alavi:
* Eq. "part": H = sum t_ij a+_i a_j + sum <ij|kl> a+_i a+_j a_l a_k, written
  here in spatial-orbital chemists' notation with the conventional 1/2,
  H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum_{pqrs,s,t} (pq|rs) a+_ps a+_rt a_st a_qs.
* The partition into core (occupancy 2), active (0, 1, 2) and virtual (0)
  orbitals; H0 keeps the terms that move no electrons between the three
  sets (Delta n_ex = 0, counting both spins), U = H - H0.  A term conserves
  every set's electron count iff it connects determinants of the same
  excitation class (N_core, N_virt), so H0_IJ = H_IJ * [class_I == class_J].

Determinants are bit masks over spin orbitals ordered 0a, 0b, 1a, 1b, ...;
|D> = prod_{j ascending} a+_j |vac>, so a_j|D> carries (-1)^(#occupied < j).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def spin_orbital(p: int, spin: int) -> int:
    return 2 * p + spin


def determinants(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """All determinants with n_alpha up and n_beta down electrons, sorted."""
    out = []
    for occa in itertools.combinations(range(n_orb), n_alpha):
        ma = 0
        for p in occa:
            ma |= 1 << (2 * p)
        for occb in itertools.combinations(range(n_orb), n_beta):
            mb = 0
            for p in occb:
                mb |= 1 << (2 * p + 1)
            out.append(ma | mb)
    return np.array(sorted(out), dtype=np.int64)


def _apply(D, sign, valid, j, create: bool):
    """Apply a+_j (create) or a_j to every determinant in D (vectorised)."""
    bit = np.int64(1) << np.int64(j)
    occ = (D & bit) != 0
    valid = valid & (~occ if create else occ)
    parity = np.bitwise_count(D & (bit - 1)) & 1
    sign = np.where(parity == 1, -sign, sign)
    return D ^ bit, sign, valid


def apply_string(ops, D):
    """Apply an operator string [(j, create), ...] (leftmost first in the
    product, i.e. applied last) to all determinants in D."""
    sign = np.ones(D.shape, dtype=np.float64)
    valid = np.ones(D.shape, dtype=bool)
    for j, create in reversed(ops):
        D, sign, valid = _apply(D, sign, valid, j, create)
    return D, sign, valid


def hamiltonian_terms(h: np.ndarray, V: np.ndarray, tol: float = 1e-14):
    """Yield (coef, ops) for every term of H in the spin-orbital expansion."""
    k = h.shape[0]
    for p in range(k):
        for q in range(k):
            if abs(h[p, q]) > tol:
                for s in (0, 1):
                    yield h[p, q], [(2 * p + s, True), (2 * q + s, False)]
    for p, q, r, s_ in itertools.product(range(k), repeat=4):
        v = V[p, q, r, s_]
        if abs(v) <= tol:
            continue
        for a in (0, 1):
            for b in (0, 1):
                # 1/2 (pq|rs) a+_{p a} a+_{r b} a_{s b} a_{q a}
                yield 0.5 * v, [(2 * p + a, True), (2 * r + b, True),
                                (2 * s_ + b, False), (2 * q + a, False)]


def build_hamiltonian(h: np.ndarray, V: np.ndarray, dets: np.ndarray,
                      term_filter=None) -> sp.csr_matrix:
    """Sparse H in the determinant basis ``dets`` (sorted int64 masks).

    ``term_filter(ops) -> bool`` keeps a subset of the terms (used to build
    H0 directly from the Delta n_ex = 0 rule as a cross-check of the class
    mask)."""
    n = len(dets)
    rows, cols, vals = [], [], []
    col_idx = np.arange(n)
    for coef, ops in hamiltonian_terms(h, V):
        if term_filter is not None and not term_filter(ops):
            continue
        D2, sign, valid = apply_string(ops, dets)
        if not valid.any():
            continue
        D2 = D2[valid]
        pos = np.searchsorted(dets, D2)
        pos = np.minimum(pos, n - 1)
        hit = dets[pos] == D2
        rows.append(pos[hit])
        cols.append(col_idx[valid][hit])
        vals.append(coef * sign[valid][hit])
    if rows:
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        v = np.concatenate(vals)
    else:
        r = c = np.zeros(0, dtype=np.int64)
        v = np.zeros(0)
    return sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()


def orbital_sets(n_orb: int, n_core: int, n_active: int):
    """Set label per spatial orbital: 0 core, 1 active, 2 virtual."""
    return np.array([0 if p < n_core else (1 if p < n_core + n_active else 2)
                     for p in range(n_orb)])


def excitation_class(dets: np.ndarray, n_orb: int, n_core: int, n_active: int):
    """(N_core, N_virt) of every determinant, both spins counted."""
    core = 0
    virt = 0
    for p in range(n_orb):
        if p < n_core:
            core |= (3 << (2 * p))
        elif p >= n_core + n_active:
            virt |= (3 << (2 * p))
    nc = np.bitwise_count(dets & np.int64(core))
    nv = np.bitwise_count(dets & np.int64(virt))
    return nc.astype(np.int64), nv.astype(np.int64)


def delta_nex_zero(n_orb: int, n_core: int, n_active: int):
    """Term filter: keep terms that conserve each set's electron count."""
    sets = orbital_sets(n_orb, n_core, n_active)

    def keep(ops):
        cnt = [0, 0, 0]
        for j, create in ops:
            cnt[sets[j // 2]] += 1 if create else -1
        return cnt == [0, 0, 0]
    return keep


def fink_h0(H: sp.csr_matrix, dets, n_orb, n_core, n_active) -> sp.csr_matrix:
    """H0 = H restricted to blocks within one excitation class."""
    nc, nv = excitation_class(dets, n_orb, n_core, n_active)
    cls = nc * 1000 + nv
    Hc = H.tocoo()
    keep = cls[Hc.row] == cls[Hc.col]
    return sp.coo_matrix((Hc.data[keep], (Hc.row[keep], Hc.col[keep])),
                         shape=H.shape).tocsr()


def lowest_eigenpair(H, idx=None):
    """Lowest eigenpair of H (optionally restricted to index set ``idx``)."""
    if idx is not None:
        H = H[idx][:, idx]
    Hd = H.toarray() if sp.issparse(H) else np.asarray(H)
    w, U = np.linalg.eigh(Hd)
    return w[0], U[:, 0]


def fci(h, V, n_alpha, n_beta):
    """Full CI ground state energy and vector."""
    k = h.shape[0]
    dets = determinants(k, n_alpha, n_beta)
    H = build_hamiltonian(h, V, dets)
    E, c = lowest_eigenpair(H)
    return E, c, dets, H


def reference_class_indices(dets, n_orb, n_core, n_active):
    nc, nv = excitation_class(dets, n_orb, n_core, n_active)
    return np.nonzero((nc == 2 * n_core) & (nv == 0))[0]


def cas_ci(H, dets, n_orb, n_core, n_active):
    """Reference: lowest eigenpair of H within the reference class (core full,
    virtual empty), embedded in the full determinant space.  Within that class
    H0 = H, so E0 = <Phi0|H|Phi0> = <Phi0|H0|Phi0>."""
    idx = reference_class_indices(dets, n_orb, n_core, n_active)
    E0, c = lowest_eigenpair(H, idx)
    phi0 = np.zeros(len(dets))
    phi0[idx] = c
    return E0, phi0
