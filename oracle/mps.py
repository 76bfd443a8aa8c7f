"""MPS expansion and the dense local problem (oracle).

* Eq. mps1: |Psi> = sum A^{n1} A^{n2} ... A^{nk} |n1 ... nk>, with the
  occupation basis of one spatial orbital 0=|0>, 1=|up>, 2=|dn>,
  3=|up dn> = a+_up a+_dn |0>, and |n1 ... nk> = prod_p (a+_p,up)^.. (a+_p,dn)^.. |vac>
  in ascending orbital order (the determinant convention of ``oracle.fci``).
* Implementation section (Fig. 3 and the sweep paragraph): fixing every site
  tensor but the ones being optimised makes the functional quadratic in the
  local tensor; its derivative is P^T H P psi where P maps the local tensor
  to the full space.  For a two-site position (l, l+1),
  P[(..., s_l, s_l+1, ...), (a, s_l, s_l+1, b)] = L[config_left, a] R[b, config_right],
  L / R being the contractions of sites < l and > l+1.

The local vector layout is the library's documented layout (``include/mpslcc.h``):
middle sectors q ascending by (N, 2S_z); inside a sector a row-major block
[rows = (s_l ascending, left-bond sector ascending, a), cols = (s_l+1
ascending, right-bond sector ascending, b)].
"""
from __future__ import annotations

import numpy as np

LOCAL_N = (0, 1, 1, 2)
LOCAL_2SZ = (0, 1, -1, 0)


def _site_bits(p: int, s: int) -> int:
    m = 0
    if s in (1, 3):
        m |= 1 << (2 * p)
    if s in (2, 3):
        m |= 1 << (2 * p + 1)
    return m


def _qn(bond, i):
    return (bond[i][0], bond[i][1])


def left_basis(mps, l: int):
    """Contract sites 0..l-1: list of (det_mask, sector_index, row_vector)."""
    bonds, sites, masks = mps["bonds"], mps["sites"], mps["masks"]
    cur = [(0, 0, np.ones(1))]
    for p in range(l):
        nxt = []
        for (mask, ia, v) in cur:
            for s in masks[p]:
                for (ja, js, jb), blk in sites[p].items():
                    if ja == ia and js == s:
                        nxt.append((mask | _site_bits(p, s), jb, v @ blk))
        cur = nxt
    return cur


def right_basis(mps, l: int):
    """Contract sites l+2..k-1: list of (det_mask, sector_index, col_vector)."""
    bonds, sites, masks = mps["bonds"], mps["sites"], mps["masks"]
    k = len(sites)
    cur = [(0, 0, np.ones(1))]
    for p in range(k - 1, l + 1, -1):
        nxt = []
        for (mask, ib, v) in cur:
            for s in masks[p]:
                for (ja, js, jb), blk in sites[p].items():
                    if jb == ib and js == s:
                        nxt.append((mask | _site_bits(p, s), ja, blk @ v))
        cur = nxt
    return cur


def local_layout(mps, l: int):
    """Entries (ia, a, s1, s2, ib, b) of the two-site local vector, in order,
    plus the list of middle sectors with (dimFL, dimFR)."""
    bonds, masks = mps["bonds"], mps["masks"]
    bl, br = bonds[l], bonds[l + 2]

    def fl(q):
        pieces = []
        for s in sorted(masks[l]):
            for ia in range(len(bl)):
                qa = _qn(bl, ia)
                if (qa[0] + LOCAL_N[s], qa[1] + LOCAL_2SZ[s]) == q:
                    pieces.append((ia, s, bl[ia][2]))
        return pieces

    def fr(q):
        pieces = []
        for s in sorted(masks[l + 1]):
            for ib in range(len(br)):
                qb = _qn(br, ib)
                if (qb[0] - LOCAL_N[s], qb[1] - LOCAL_2SZ[s]) == q:
                    pieces.append((s, ib, br[ib][2]))
        return pieces

    cand = set()
    for ia in range(len(bl)):
        for s in masks[l]:
            cand.add((bl[ia][0] + LOCAL_N[s], bl[ia][1] + LOCAL_2SZ[s]))
    entries, sectors = [], []
    for q in sorted(cand):
        L, R = fl(q), fr(q)
        dl = sum(p[2] for p in L)
        dr = sum(p[2] for p in R)
        if dl == 0 or dr == 0:
            continue
        sectors.append((q, dl, dr))
        for (ia, s1, da) in L:
            for a in range(da):
                for (s2, ib, db) in R:
                    for b in range(db):
                        entries.append((ia, a, s1, s2, ib, b))
    return entries, sectors


def isometry(mps, l: int, dets: np.ndarray) -> np.ndarray:
    """Dense P [n_dets x n_local] of the two-site position (l, l+1)."""
    entries, _ = local_layout(mps, l)
    n_loc = len(entries)
    left = left_basis(mps, l)
    right = right_basis(mps, l)
    groups = {}
    for j, (ia, a, s1, s2, ib, b) in enumerate(entries):
        groups.setdefault((ia, s1, s2, ib), []).append((j, a, b))
    byL, byR = {}, {}
    for (m, ia, v) in left:
        byL.setdefault(ia, []).append((m, v))
    for (m, ib, v) in right:
        byR.setdefault(ib, []).append((m, v))
    P = np.zeros((len(dets), n_loc))
    for (ia, s1, s2, ib), cols in groups.items():
        if ia not in byL or ib not in byR:
            continue
        mL = np.array([m for m, _ in byL[ia]], dtype=np.int64)
        VL = np.array([v for _, v in byL[ia]])
        mR = np.array([m for m, _ in byR[ib]], dtype=np.int64)
        VR = np.array([v for _, v in byR[ib]])
        mid = _site_bits(l, s1) | _site_bits(l + 1, s2)
        full = (mL[:, None] | mR[None, :]) | mid
        pos = np.searchsorted(dets, full.ravel())
        pos = np.minimum(pos, len(dets) - 1)
        ok = dets[pos] == full.ravel()
        js = np.array([c[0] for c in cols])
        aa = np.array([c[1] for c in cols])
        bb = np.array([c[2] for c in cols])
        vals = np.einsum("xa,yb->xyab", VL, VR).reshape(len(mL) * len(mR), VL.shape[1], VR.shape[1])
        block = vals[:, aa, bb]  # [nL*nR, ncols]
        P[np.ix_(pos[ok], js)] += block[ok]
    return P


def effective_hamiltonian(mps, l: int, H, dets) -> np.ndarray:
    """Dense H_eff = P^T H P at two-site position l (the local problem)."""
    P = isometry(mps, l, dets)
    return P.T @ (H @ P)


def transition_operator(bra, ket, l: int, H, dets) -> np.ndarray:
    """P_bra^T H P_ket: maps the ket's local vector to the bra's local space."""
    Pb = isometry(bra, l, dets)
    Pk = isometry(ket, l, dets)
    return Pb.T @ (H @ Pk)


def to_vector(mps, dets: np.ndarray) -> np.ndarray:
    """Full determinant-space amplitudes of the MPS."""
    k = len(mps["sites"])
    out = np.zeros(len(dets))
    for (m, ib, v) in left_basis(mps, k):
        pos = np.searchsorted(dets, m)
        if pos < len(dets) and dets[pos] == m:
            out[pos] += v[0]
    return out


# ----------------------------------------------------------------------------
# one-site local problem (Implementation section: only the tensor of one site
# is optimised at a time)
# ----------------------------------------------------------------------------
def local_layout1(mps, l: int):
    """Entries (ia, a, s, ib, b) of the one-site local vector at site l, in
    order: bond-(l+1) sectors q ascending (those reachable from bond l), each a
    row-major block with rows = (s ascending, bond-l sector ascending, a) and
    columns = the index b within sector q of bond l+1."""
    bonds, masks = mps["bonds"], mps["masks"]
    bl, br = bonds[l], bonds[l + 1]
    entries = []
    for ib, (n, z, db) in enumerate(br):
        rows = []
        for s in sorted(masks[l]):
            for ia, (na, za, da) in enumerate(bl):
                if (na + LOCAL_N[s], za + LOCAL_2SZ[s]) == (n, z):
                    rows.append((s, ia, da))
        for (s, ia, da) in rows:
            for a in range(da):
                for b in range(db):
                    entries.append((ia, a, s, ib, b))
    return entries


def isometry1(mps, l: int, dets: np.ndarray) -> np.ndarray:
    """Dense P [n_dets x n_local] of site l: P[(.., s_l, ..), (ia, a, s, ib, b)]
    = L[config_left, a] R[b, config_right] delta(s_l, s), L / R the
    contractions of sites < l and > l."""
    entries = local_layout1(mps, l)
    left = left_basis(mps, l)
    right = right_basis(mps, l - 1)
    byL, byR = {}, {}
    for (m, ia, v) in left:
        byL.setdefault(ia, []).append((m, v))
    for (m, ib, v) in right:
        byR.setdefault(ib, []).append((m, v))
    P = np.zeros((len(dets), len(entries)))
    for j, (ia, a, s, ib, b) in enumerate(entries):
        for (mL, vL) in byL.get(ia, []):
            for (mR, vR) in byR.get(ib, []):
                full = mL | mR | _site_bits(l, s)
                pos = np.searchsorted(dets, full)
                if pos < len(dets) and dets[pos] == full:
                    P[pos, j] += vL[a] * vR[b]
    return P
