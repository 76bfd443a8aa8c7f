"""Seeded synthetic inputs shared by the CPU oracle and the GPU library.

This module only *generates inputs*: one-body integrals h_ij, two-electron
integrals (ij|kl) in chemists' notation, orbital partitions, and random
block-sparse matrix product states.  It contains none of the MPS-LCC method's
arithmetic (no Hamiltonian application, no environments, no solvers), so both
the oracle (``oracle/``) and the GPU path (``paper_1509_00216_gb300``) may use
it without sharing method code.

The paper's own workloads (first-row dimers, Cr2, diamond, 2D Hubbard, 3-band
Hubbard; Sharma & Alavi, "Benchmarks" section) need molecular integrals that
are not available, so the lattice and ab-initio-like Hamiltonians below stand
in for them.  Every generator is deterministic given its seed.

Conventions
-----------
* ``h``: (k, k) symmetric one-body integrals t_ij (Eq. "part", first sum).
* ``V``: (k, k, k, k) chemists' integrals (ij|kl) with 8-fold symmetry; the
  Hamiltonian is  H = sum_{ij,s} h_ij a+_is a_js
                    + 1/2 sum_{ijkl,s,t} (ij|kl) a+_is a+_kt a_lt a_js.
* Orbitals of lattice models are rotated into the non-interacting (U=0)
  eigenbasis, sorted by orbital energy, so that core / active / virtual sets
  (Fink partition, Theory section) are contiguous blocks of the MPS ordering.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

SEED_BASE = 150900216


# ----------------------------------------------------------------------------
# lattice Hamiltonians in the site basis
# ----------------------------------------------------------------------------
def hubbard_chain(L: int, t: float, U: float, pbc: bool = False):
    """1D Hubbard chain: h_{j,j+1} = -t, (jj|jj) = U (open boundary by default)."""
    h = np.zeros((L, L))
    for j in range(L - 1):
        h[j, j + 1] = h[j + 1, j] = -t
    if pbc and L > 2:
        h[0, L - 1] = h[L - 1, 0] = -t
    V = np.zeros((L, L, L, L))
    for j in range(L):
        V[j, j, j, j] = U
    return h, V


def snake_index(x: int, y: int, Lx: int) -> int:
    """Snake (boustrophedon) MPS ordering of a 2D lattice site."""
    return y * Lx + (x if y % 2 == 0 else Lx - 1 - x)


def hubbard_2d(Lx: int, Ly: int, t: float, U: float):
    """Periodic Lx x Ly Hubbard lattice, nearest-neighbour hopping -t, snake order."""
    n = Lx * Ly
    h = np.zeros((n, n))
    for y in range(Ly):
        for x in range(Lx):
            i = snake_index(x, y, Lx)
            for dx, dy in ((1, 0), (0, 1)):
                j = snake_index((x + dx) % Lx, (y + dy) % Ly, Lx)
                if j != i:
                    h[i, j] -= t
                    h[j, i] -= t
    V = np.zeros((n, n, n, n))
    for i in range(n):
        V[i, i, i, i] = U
    return h, V


def three_band(Lx: int, Ly: int, tpd: float, tpp: float, dpd: float,
               Ud: float, Up: float):
    """Periodic 3-band (Cu d, O px, O py) Hubbard model in the hole picture.

    Orbital order: cell-major (snake order over cells), within a cell d, px, py.
    eps_d = 0, eps_p = dpd.  d-p hopping is +tpd toward the +x/2 and -y/2 oxygen
    and -tpd toward the other two; p-p hopping between px(R + sx x/2) and
    py(R + sy y/2) is -sx*sy*tpp.  Periodic duplicates are summed.
    """
    ncell = Lx * Ly
    n = 3 * ncell

    def cell(x, y):
        return snake_index(x % Lx, y % Ly, Lx)

    def d(x, y):
        return 3 * cell(x, y)

    def px(x, y):  # oxygen at (x + 1/2, y)
        return 3 * cell(x, y) + 1

    def py(x, y):  # oxygen at (x, y + 1/2)
        return 3 * cell(x, y) + 2

    h = np.zeros((n, n))
    for y in range(Ly):
        for x in range(Lx):
            h[d(x, y), d(x, y)] += 0.0
            h[px(x, y), px(x, y)] += dpd
            h[py(x, y), py(x, y)] += dpd
            # d - p
            nb = [(px(x, y), +tpd), (px(x - 1, y), -tpd),
                  (py(x, y), -tpd), (py(x, y - 1), +tpd)]
            for j, v in nb:
                h[d(x, y), j] += v
                h[j, d(x, y)] += v
            # p - p around this Cu
            for sx in (+1, -1):
                for sy in (+1, -1):
                    a = px(x, y) if sx > 0 else px(x - 1, y)
                    b = py(x, y) if sy > 0 else py(x, y - 1)
                    h[a, b] += -sx * sy * tpp
                    h[b, a] += -sx * sy * tpp
    V = np.zeros((n, n, n, n))
    for c in range(ncell):
        V[3 * c, 3 * c, 3 * c, 3 * c] = Ud
        V[3 * c + 1, 3 * c + 1, 3 * c + 1, 3 * c + 1] = Up
        V[3 * c + 2, 3 * c + 2, 3 * c + 2, 3 * c + 2] = Up
    return h, V


# ----------------------------------------------------------------------------
# synthetic ab initio integrals
# ----------------------------------------------------------------------------
def ab_initio(k: int, n_chol: int, seed: int, frontier: tuple | None = None):
    """Synthetic molecular-like integrals.

    h_ii = sorted(2 N(0,1)), h_ij = h_ji ~ N(0, 0.05) (standard deviation),
    (ij|kl) = sum_{L=1..n_chol} B^L_ij B^L_kl with symmetric B^L whose entries
    are N(0, 0.1/sqrt(L)).  ``frontier=(first, count, width)`` places ``count``
    diagonal energies starting at orbital ``first`` (0-based) at
    h_mid + linspace(-width/2, width/2, count), a near-degenerate frontier.
    """
    rng = np.random.default_rng(seed)
    diag = np.sort(2.0 * rng.standard_normal(k))
    off = rng.normal(0.0, 0.05, size=(k, k))
    h = np.triu(off, 1)
    h = h + h.T + np.diag(diag)
    if frontier is not None:
        first, count, width = frontier
        mid = h[first + count // 2, first + count // 2]
        vals = mid + np.linspace(-width / 2, width / 2, count)
        for j in range(count):
            h[first + j, first + j] = vals[j]
    V = np.zeros((k, k, k, k))
    for L in range(1, n_chol + 1):
        B = rng.normal(0.0, 0.1 / math.sqrt(L), size=(k, k))
        B = np.triu(B) + np.triu(B, 1).T
        V += np.einsum("ij,kl->ijkl", B, B)
    return h, V


# ----------------------------------------------------------------------------
# orbital rotation (input preparation)
# ----------------------------------------------------------------------------
def deterministic_eigenbasis(h: np.ndarray, tol: float = 1e-8):
    """Eigenvectors of h sorted by energy; degenerate levels are fixed by
    Gram-Schmidt of the site unit vectors projected into each level."""
    w, U = np.linalg.eigh(h)
    n = len(w)
    C = np.zeros_like(U)
    i = 0
    while i < n:
        j = i
        while j + 1 < n and abs(w[j + 1] - w[i]) < tol:
            j += 1
        Vg = U[:, i:j + 1]
        g = j - i + 1
        P = Vg @ Vg.T
        basis = []
        for site in range(n):
            u = P[:, site].copy()
            for b in basis:
                u -= (b @ u) * b
            nu = np.linalg.norm(u)
            if nu > 1e-6:
                basis.append(u / nu)
            if len(basis) == g:
                break
        C[:, i:j + 1] = np.array(basis).T
        i = j + 1
    return w, C


def rotate(h: np.ndarray, V: np.ndarray, C: np.ndarray):
    """Transform integrals to the orbital basis given by the columns of C."""
    h2 = C.T @ h @ C
    V2 = np.einsum("ijkl,ip->pjkl", V, C, optimize=True)
    V2 = np.einsum("pjkl,jq->pqkl", V2, C, optimize=True)
    V2 = np.einsum("pqkl,kr->pqrl", V2, C, optimize=True)
    V2 = np.einsum("pqrl,ls->pqrs", V2, C, optimize=True)
    return h2, V2


def to_orbital_basis(h, V, tol=1e-8):
    eps, C = deterministic_eigenbasis(h, tol)
    h2, V2 = rotate(h, V, C)
    return eps, h2, V2


def check_partition_gap(eps, n_core, n_active, tol=1e-8):
    """The core/active and active/virtual boundaries must not split a level."""
    k = len(eps)
    for b in (n_core, n_core + n_active):
        if 0 < b < k:
            if abs(eps[b] - eps[b - 1]) <= tol:
                raise ValueError(f"partition boundary {b} splits a degenerate level")


# ----------------------------------------------------------------------------
# the five benchmark workloads
# ----------------------------------------------------------------------------
CONFIG_NAMES = [
    "hubbard1d_L8_U4",
    "abinitio_k24",
    "hubbard2d_4x4_U8",
    "threeband_2x4",
    "abinitio_k30",
]


def config(i: int) -> dict:
    """Seeded Hamiltonian and run parameters of workload ``i`` (0-based)."""
    seed = SEED_BASE + i
    if i == 0:
        h, V = hubbard_chain(8, 1.0, 4.0)
        # closed-form sine modes, phi_m(j) = sqrt(2/9) sin(pi m j / 9)
        L = 8
        C = np.array([[math.sqrt(2.0 / (L + 1)) * math.sin(math.pi * m * j / (L + 1))
                       for m in range(1, L + 1)] for j in range(1, L + 1)])
        eps = np.array([-2.0 * math.cos(math.pi * m / (L + 1)) for m in range(1, L + 1)])
        h, V = rotate(h, V, C)
        d = dict(n_orb=8, n_alpha=4, n_beta=4, n_core=2, n_active=4,
                 M0=16, M1=64, sweeps=4)
    elif i == 1:
        h, V = ab_initio(24, 72, seed)
        eps = np.diag(h).copy()
        d = dict(n_orb=24, n_alpha=12, n_beta=12, n_core=8, n_active=8,
                 M0=128, M1=512, sweeps=4)
    elif i == 2:
        h, V = hubbard_2d(4, 4, 1.0, 8.0)
        eps, h, V = to_orbital_basis(h, V)
        d = dict(n_orb=16, n_alpha=7, n_beta=7, n_core=5, n_active=6,
                 M0=250, M1=1000, sweeps=4)
    elif i == 3:
        h, V = three_band(2, 4, 1.3, 0.65, 3.6, 8.4, 0.0)
        eps, h, V = to_orbital_basis(h, V)
        n_active = 18
        # move the active/virtual boundary outward until it sits in a gap
        while n_active < 24 and abs(eps[n_active] - eps[n_active - 1]) <= 1e-8:
            n_active += 1
        d = dict(n_orb=24, n_alpha=9, n_beta=9, n_core=0, n_active=n_active,
                 M0=500, M1=2000, sweeps=4)
    elif i == 4:
        h, V = ab_initio(30, 90, seed, frontier=(9, 6, 0.05))
        eps = np.diag(h).copy()
        d = dict(n_orb=30, n_alpha=12, n_beta=12, n_core=6, n_active=12,
                 M0=800, M1=4000, sweeps=2)
    else:
        raise ValueError(i)
    if i in (2, 3):
        check_partition_gap(eps, d["n_core"], d["n_active"])
    d.update(name=CONFIG_NAMES[i], h=np.ascontiguousarray(h),
             V=np.ascontiguousarray(V), eps=np.asarray(eps), seed=seed)
    return d


def hubbard_dimer(t: float, U: float, orbital_basis: bool = False):
    """Two-site Hubbard model; optionally in the bonding/antibonding basis."""
    h, V = hubbard_chain(2, t, U)
    if orbital_basis:
        C = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
        h, V = rotate(h, V, C)
    return h, V


# ----------------------------------------------------------------------------
# random block-sparse MPS (for sigma-vector parity)
# ----------------------------------------------------------------------------
# local basis of one spatial orbital: 0=|0>, 1=|up>, 2=|dn>, 3=|up dn>
LOCAL_N = (0, 1, 1, 2)
LOCAL_2SZ = (0, 1, -1, 0)


def site_masks(n_orb: int, n_core: int = 0, n_active: int | None = None,
               frozen: bool = False):
    """Allowed local states per site.  With ``frozen`` the core sites only
    allow |up dn> and the virtual sites only |0> (the reference class)."""
    if n_active is None:
        n_active = n_orb - n_core
    masks = []
    for p in range(n_orb):
        if frozen and p < n_core:
            masks.append((3,))
        elif frozen and p >= n_core + n_active:
            masks.append((0,))
        else:
            masks.append((0, 1, 2, 3))
    return masks


def _reachable(masks, start):
    """QN sets reachable after each site, sweeping from ``start`` (list of sets)."""
    out = [set(start)]
    for m in masks:
        nxt = set()
        for (n, sz) in out[-1]:
            for s in m:
                nxt.add((n + LOCAL_N[s], sz + LOCAL_2SZ[s]))
        out.append(nxt)
    return out


def _counts(masks):
    """Number of left-block configurations per QN at each bond."""
    cnt = [{(0, 0): 1}]
    for m in masks:
        nxt = {}
        for (n, sz), c in cnt[-1].items():
            for s in m:
                q = (n + LOCAL_N[s], sz + LOCAL_2SZ[s])
                nxt[q] = nxt.get(q, 0) + c
        cnt.append(nxt)
    return cnt


def bond_sectors(masks, n_elec: int, two_sz: int, M: int):
    """Allowed QN sectors per bond (k+1 bonds, boundaries included) with dims
    min(#left configs, #right configs) scaled so that the total is <= M.

    Bond QNs are left-cumulative (electrons and 2S_z of sites left of it)."""
    k = len(masks)
    left = _counts(masks)
    right_rev = _counts(list(reversed(masks)))
    bonds = []
    for b in range(k + 1):
        secs = []
        for q, cl in left[b].items():
            rq = (n_elec - q[0], two_sz - q[1])
            cr = right_rev[k - b].get(rq, 0)
            if cr > 0:
                secs.append((q[0], q[1], min(cl, cr)))
        secs.sort()
        tot = sum(s[2] for s in secs)
        if tot > M:
            f = M / tot
            secs = [(n, sz, max(1, int(math.floor(d * f)))) for (n, sz, d) in secs]
        bonds.append(secs)
    return bonds


def random_mps(n_orb: int, n_elec: int, two_sz: int, M: int, seed: int,
               masks=None, isometric: bool = True):
    """Random block-sparse MPS.

    Returns dict(bonds=[[(n, 2sz, dim)...] for bond 0..k], sites=[{(ia, s, ib):
    array(dim_a, dim_b)}]) where site p joins bond p (left) and bond p+1.
    With ``isometric`` each site is made right-orthonormal (rows of the
    a x (s b) matrix orthonormal) from a Gaussian draw via QR, so the MPS is
    in right-canonical form apart from its first site.
    """
    if masks is None:
        masks = site_masks(n_orb)
    rng = np.random.default_rng(seed)
    bonds = bond_sectors(masks, n_elec, two_sz, M)
    k = n_orb
    sites = []
    for p in range(k):
        la, lb = bonds[p], bonds[p + 1]
        idx_b = {(n, sz): j for j, (n, sz, _) in enumerate(lb)}
        blocks = {}
        # group by left sector: right-orthonormal rows of a x (s b)
        for ia, (na, sza, da) in enumerate(la):
            cols = []
            for s in masks[p]:
                qb = (na + LOCAL_N[s], sza + LOCAL_2SZ[s])
                if qb in idx_b:
                    ib = idx_b[qb]
                    cols.append((s, ib, lb[ib][2]))
            if not cols:
                continue
            ncol = sum(c[2] for c in cols)
            X = rng.standard_normal((da, ncol))
            if isometric:
                if ncol >= da:
                    Q, _ = np.linalg.qr(X.T)
                    X = Q.T[:da]
                else:
                    X = X / math.sqrt(ncol)
            else:
                X = X / math.sqrt(max(ncol, 1))
            off = 0
            for (s, ib, db) in cols:
                blocks[(ia, s, ib)] = np.ascontiguousarray(X[:, off:off + db])
                off += db
        sites.append(blocks)
    return dict(bonds=bonds, sites=sites, n_elec=n_elec, two_sz=two_sz,
                masks=[tuple(m) for m in masks])


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    return v / np.linalg.norm(v)
