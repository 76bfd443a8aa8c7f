"""Block-sparse CPU oracle (O2) for the local problem at any bond dimension.
TEST INFRASTRUCTURE ONLY: used by tests/ and by bench.py's CPU-baseline leg;
the library never imports it and it imports nothing of the library.

The determinant-space oracle (``oracle.fci`` / ``oracle.mps``) cannot hold
24 orbitals, so at the sizes the GPU library is run at, the sigma vector of
the Implementation section (Fig. 3: the derivative of the functional with
respect to the local tensor, P^T O P psi) is recomputed here from
U(1) x U(1) blocks with plain numpy matrix products:

* ``Mpo`` -- a matrix product operator for H, the Fink H0 (Theory section,
  terms that move no electrons between core, active and virtual sets), U =
  H - H0, or the identity, built from h and (pq|rs) alone.  Every term of the
  spin-orbital Hamiltonian (Eq. "part" with the 1/2 of chemists' integrals)
  is written as an operator string in ascending site order (a fermionic sign
  per transposition); in the Jordan-Wigner representation of the occupation
  basis its matrix is a Kronecker product whose factor at site y is the
  product of its operators at y times the parity P = (-1)^n when an odd
  number of its operators lie right of y.  At each bond the term is carried
  by one channel named after the part of the string still to come ("nothing
  yet", "done") or by its left operators (one, or two when the left block is
  the smaller side) or its right operators (one, or two): a channel named by
  right operators sums all terms sharing them, with their coefficients, so
  the bond dimension stays O(k^2) (Implementation section).  The coefficient
  enters at the site where the term's channel changes from left-named to
  right-named.
* environments -- the transition elements of Fig. 2 contracted site by site:
  L_{y+1}[w'] = sum_{w, s, s'} W_y[w, w'](s, s') A_bra^{s T} L_y[w] A_ket^{s'},
  and R_y likewise from the right, stored per (bra sector, ket sector) pair as
  [channels of the matching class x bra dim x ket dim].
* ``sigma`` -- P_bra^T O P_ket psi at two-site position (l, l+1) contracted
  in the order right environment, W_{l+1}, W_l, left environment.

Exact in exact arithmetic; FP64 here.  The local-vector layout is the one of
``include/mpslcc.h`` (pinned in tests against ``oracle.mps.local_layout``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

LOCAL_N = (0, 1, 1, 2)
LOCAL_2SZ = (0, 1, -1, 0)
# elementary operators: kind 0 = a+ up, 1 = a+ dn, 2 = a up, 3 = a dn
KIND_DN = ((1, 1), (1, -1), (-1, -1), (-1, 1))   # (dN, d2Sz) each kind applies


def _local_ops():
    """4x4 matrices [s_out, s_in] of the elementary operators on one orbital
    with |up dn> = a+_up a+_dn |0> (so a+_dn |up> = -|up dn>)."""
    cu = np.zeros((4, 4))
    cu[1, 0] = 1.0   # |0>  -> |up>
    cu[3, 2] = 1.0   # |dn> -> |up dn>
    cd = np.zeros((4, 4))
    cd[2, 0] = 1.0   # |0>  -> |dn>
    cd[3, 1] = -1.0  # |up> -> -|up dn>
    return [cu, cd, cu.T.copy(), cd.T.copy()]


OPS = _local_ops()
PARITY = np.diag([1.0, -1.0, -1.0, 1.0])

# channel label types
L_I, L_P1, L_P2, L_S2, L_S1, L_H = 0, 1, 2, 3, 4, 5


# ---------------------------------------------------------------------------
# terms
# ---------------------------------------------------------------------------
def _terms(h, V, tol=1e-14):
    """All operator strings of H as arrays: sites [N, 4], kinds [N, 4], n [N]
    (2 or 4 operators, unused slots -1) and coefficients [N], in the order
    written (not yet sorted)."""
    k = h.shape[0]
    S, Kd, C, Nn = [], [], [], []
    p, q = np.nonzero(np.abs(h) > tol)
    for s in (0, 1):
        st = np.full((len(p), 4), -1, dtype=np.int64)
        kd = np.full((len(p), 4), -1, dtype=np.int64)
        st[:, 0], st[:, 1] = p, q
        kd[:, 0], kd[:, 1] = s, 2 + s
        S.append(st), Kd.append(kd), C.append(h[p, q]), Nn.append(np.full(len(p), 2))
    idx = np.nonzero(np.abs(V) > tol)
    P, Q, R, T = idx
    v = V[idx]
    for a in (0, 1):
        for b in (0, 1):
            # 1/2 (pq|rs) a+_{p a} a+_{r b} a_{s b} a_{q a}
            st = np.stack([P, R, T, Q], axis=1).astype(np.int64)
            kd = np.tile(np.array([a, b, 2 + b, 2 + a], dtype=np.int64), (len(v), 1))
            S.append(st), Kd.append(kd), C.append(0.5 * v), Nn.append(np.full(len(v), 4))
    return np.concatenate(S), np.concatenate(Kd), np.concatenate(Nn), np.concatenate(C)


def _canonical(st, kd, n, c):
    """Sort each string by (site, spin), stable, with the sign of the
    permutation; drop strings that create or annihilate one spin orbital
    twice; merge equal strings."""
    big = 10 ** 6
    key = np.where(st >= 0, st * 2 + (kd & 1), big)
    order = np.argsort(key, axis=1, kind="stable")
    inv = np.zeros(len(c), dtype=np.int64)
    for i in range(4):
        for j in range(i + 1, 4):
            inv += order[:, i] > order[:, j]
    st = np.take_along_axis(st, order, axis=1)
    kd = np.take_along_axis(kd, order, axis=1)
    key = np.take_along_axis(key, order, axis=1)
    sign = np.where(inv % 2 == 1, -1.0, 1.0)
    zero = np.zeros(len(c), dtype=bool)
    for i in range(3):
        zero |= (key[:, i] == key[:, i + 1]) & (key[:, i] < big) & (kd[:, i] == kd[:, i + 1])
    keep = ~zero
    st, kd, n, c = st[keep], kd[keep], n[keep], (c * sign)[keep]
    code = np.zeros(len(c), dtype=np.int64)
    for i in range(4):
        code = code * 512 + np.where(st[:, i] >= 0, st[:, i] * 4 + kd[:, i] + 1, 0)
    u, first, inverse = np.unique(code, return_index=True, return_inverse=True)
    csum = np.zeros(len(u))
    np.add.at(csum, inverse, c)
    keep = np.abs(csum) > 1e-13
    return st[first][keep], kd[first][keep], n[first][keep], csum[keep]


def _set_filter(st, kd, n, n_core, n_active, kind):
    """Fink partition: H0 keeps the strings whose creations and annihilations
    balance within each of the core / active / virtual sets; U the others."""
    sets = np.where(st < n_core, 0, np.where(st < n_core + n_active, 1, 2))
    bal = np.zeros((len(n), 3), dtype=np.int64)
    for i in range(4):
        valid = st[:, i] >= 0
        d = np.where(kd[:, i] < 2, 1, -1) * valid
        for s in range(3):
            bal[:, s] += d * (sets[:, i] == s)
    conserving = np.all(bal == 0, axis=1)
    return conserving if kind == "H0" else ~conserving


# ---------------------------------------------------------------------------
# MPO
# ---------------------------------------------------------------------------
class Mpo:
    """MPO of one operator.  ``bond_classes[b]``: list of (dN, d2Sz) classes
    of bond b (the change the left part of a channel applies); ``class_n[b]``
    their channel counts; ``W[y]``: dict (c_left, c_right, s_out, s_in) ->
    sparse [channels of c_left x channels of c_right] for site y."""

    def __init__(self, h, V, kind="H", n_core=0, n_active=None):
        k = h.shape[0]
        self.k = k
        if n_active is None:
            n_active = k - n_core
        if kind == "I":
            self._identity(k)
            return
        st, kd, n, c = _canonical(*_terms(np.asarray(h, float), np.asarray(V, float)))
        if kind in ("H0", "U"):
            m = _set_filter(st, kd, n, n_core, n_active, kind)
            st, kd, n, c = st[m], kd[m], n[m], c[m]
        self.n_terms = len(c)
        if len(c) == 0:
            self._identity(k, zero=True)
            return
        self._build(k, st, kd, n, c)

    # labels ---------------------------------------------------------------
    @staticmethod
    def _label(st, kd, n, b, k):
        """Channel label (int64) of every string at bond b."""
        nl = np.sum((st >= 0) & (st < b), axis=1)
        rows = np.arange(len(n))
        lab = np.full(len(n), L_I << 40, dtype=np.int64)
        def enc(t, kinds, sa, sb):
            return (np.int64(t) << 40) | (kinds.astype(np.int64) << 24) | (sa.astype(np.int64) << 12) | sb.astype(np.int64)
        last = st[rows, n - 1]
        lastk = kd[rows, n - 1]
        small = b <= k - b
        lab = np.where(nl == n, np.int64(L_H) << 40, lab)
        m1 = (nl == 1) & (n > 1)
        lab = np.where(m1, enc(L_P1, kd[:, 0], st[:, 0], np.zeros_like(n)), lab)
        m3 = (nl == n - 1) & (nl >= 2)
        lab = np.where(m3, enc(L_S1, lastk, last, np.zeros_like(n)), lab)
        m2 = (nl == 2) & (n == 4)
        if small:
            lab = np.where(m2, enc(L_P2, kd[:, 0] * 4 + kd[:, 1], st[:, 0], st[:, 1]), lab)
        else:
            lab = np.where(m2, enc(L_S2, kd[:, 2] * 4 + kd[:, 3], st[:, 2], st[:, 3]), lab)
        return lab

    @staticmethod
    def _label_dq(lab):
        t = int(lab >> 40)
        kinds = int((lab >> 24) & 0xFFFF)
        if t == L_P1:
            return KIND_DN[kinds]
        if t == L_P2:
            a, b = KIND_DN[kinds // 4], KIND_DN[kinds % 4]
            return (a[0] + b[0], a[1] + b[1])
        if t == L_S1:
            a = KIND_DN[kinds]
            return (-a[0], -a[1])
        if t == L_S2:
            a, b = KIND_DN[kinds // 4], KIND_DN[kinds % 4]
            return (-(a[0] + b[0]), -(a[1] + b[1]))
        return (0, 0)

    @staticmethod
    def _label_nops(lab):
        t = int(lab >> 40)
        return {L_P1: 1, L_S1: 1, L_P2: 2, L_S2: 2}.get(t, 0)

    def _build(self, k, st, kd, n, c):
        labs = np.stack([self._label(st, kd, n, b, k) for b in range(k + 1)], axis=1)
        # channels per bond, ordered by class then label
        self.bond_classes, self.class_n, self.chan = [], [], []
        for b in range(k + 1):
            u = np.unique(labs[:, b])
            dq = [self._label_dq(int(x)) for x in u]
            order = sorted(range(len(u)), key=lambda i: (dq[i], int(u[i])))
            classes, counts, chan = [], [], {}
            for i in order:
                if not classes or classes[-1] != dq[i]:
                    classes.append(dq[i])
                    counts.append(0)
                chan[int(u[i])] = (len(classes) - 1, counts[-1])
                counts[-1] += 1
            self.bond_classes.append(classes)
            self.class_n.append(counts)
            self.chan.append(chan)
        # site tensors: entries (class0, pos0, class1, pos1, 4x4)
        self.W = []
        factor_cache = {}
        for y in range(k):
            ent = {}
            def add(l0, l1, M):
                c0, p0 = self.chan[y][l0]
                c1, p1 = self.chan[y + 1][l1]
                key = (c0, p0, c1, p1)
                if key in ent:
                    ent[key] = ent[key] + M
                else:
                    ent[key] = M.copy()
            # channels passing through site y unchanged: identity or parity
            for l in set(self.chan[y]) & set(self.chan[y + 1]):
                add(l, l, PARITY if self._label_nops(l) % 2 else np.eye(4))
            active = labs[:, y] != labs[:, y + 1]
            idx = np.nonzero(active)[0]
            l0 = labs[idx, y]
            l1 = labs[idx, y + 1]
            # local factor key: kinds of the ops at y (in order) and the parity
            # of the number of ops right of y
            fk = np.zeros(len(idx), dtype=np.int64)
            nright = np.zeros(len(idx), dtype=np.int64)
            for i in range(4):
                s_i = st[idx, i]
                at = s_i == y
                fk = np.where(at, fk * 5 + kd[idx, i] + 1, fk)
                nright += (s_i > y)
            fk = fk * 2 + (nright % 2)
            pre0 = np.isin(l0 >> 40, [L_I, L_P1, L_P2])
            pre1 = np.isin(l1 >> 40, [L_I, L_P1, L_P2])
            switch = pre0 & ~pre1
            # structural entries (no coefficient): one per (l0, l1, factor)
            ns = ~switch
            if ns.any():
                trip = np.unique(np.stack([l0[ns], l1[ns], fk[ns]], axis=1), axis=0)
                for a, b, f in trip:
                    add(int(a), int(b), self._factor(int(f), factor_cache))
            # entries where the coefficient enters: summed per (l0, l1, factor)
            if switch.any():
                trip = np.stack([l0[switch], l1[switch], fk[switch]], axis=1)
                u, inv = np.unique(trip, axis=0, return_inverse=True)
                cs = np.zeros(len(u))
                np.add.at(cs, inv.ravel(), c[idx[switch]])
                for (a, b, f), cv in zip(u, cs):
                    add(int(a), int(b), cv * self._factor(int(f), factor_cache))
            self.W.append(self._blocks(y, ent))

    @staticmethod
    def _factor(key, cache):
        if key in cache:
            return cache[key]
        f = key
        par = f % 2
        f //= 2
        kinds = []
        while f > 0:
            kinds.append(f % 5 - 1)
            f //= 5
        kinds.reverse()
        M = np.eye(4)
        for x in kinds:
            M = M @ OPS[x]
        if par:
            M = M @ PARITY
        cache[key] = M
        return M

    def _blocks(self, y, ent):
        acc = {}
        for (c0, p0, c1, p1), M in ent.items():
            so, si = np.nonzero(M)
            for a, b in zip(so, si):
                acc.setdefault((c0, c1, int(a), int(b)), []).append((p0, p1, M[a, b]))
        out = {}
        for key, lst in acc.items():
            c0, c1 = key[0], key[1]
            r = [x[0] for x in lst]
            q = [x[1] for x in lst]
            v = [x[2] for x in lst]
            out[key] = sp.csr_matrix((v, (r, q)), shape=(self.class_n[y][c0], self.class_n[y + 1][c1]))
        return out

    def _identity(self, k, zero=False):
        self.bond_classes = [[(0, 0)] for _ in range(k + 1)]
        self.class_n = [[1] for _ in range(k + 1)]
        self.chan = [{0: (0, 0)} for _ in range(k + 1)]
        self.n_terms = 0
        self.W = []
        for y in range(k):
            v = 0.0 if (zero and y == 0) else 1.0
            self.W.append({(0, 0, s, s): sp.csr_matrix(np.array([[v]])) for s in range(4)})

    def bond_dims(self):
        return [int(sum(x)) for x in self.class_n]

    def class_of(self, b, dq):
        try:
            return self.bond_classes[b].index(tuple(dq))
        except ValueError:
            return -1


# ---------------------------------------------------------------------------
# environments
# ---------------------------------------------------------------------------
def _q(bond, i):
    return (bond[i][0], bond[i][1])


def _sector_index(bond):
    return {(s[0], s[1]): i for i, s in enumerate(bond)}


def boundary_left(mpo):
    return {(0, 0): np.ones((1, 1, 1))}


def boundary_right(mpo):
    return {(0, 0): np.ones((1, 1, 1))}


def _site_by_left(site):
    """(ia, s) -> list of (ib, block)"""
    out = {}
    for (ia, s, ib), blk in site.items():
        out.setdefault((ia, s), []).append((ib, blk))
    return out


def _site_by_right(site):
    """(ib, s) -> list of (ia, block)"""
    out = {}
    for (ia, s, ib), blk in site.items():
        out.setdefault((ib, s), []).append((ia, blk))
    return out


def update_left(mpo, L, bra, ket, y):
    """L_{y+1} from L_y and site y of the bra and ket MPS."""
    bb, bk = bra["bonds"], ket["bonds"]
    SB, SK = _site_by_left(bra["sites"][y]), _site_by_left(ket["sites"][y])
    W = mpo.W[y]
    out = {}
    for (ib, ik), E in L.items():
        qb, qk = _q(bb[y], ib), _q(bk[y], ik)
        c0 = mpo.class_of(y, (qb[0] - qk[0], qb[1] - qk[1]))
        for si in range(4):
            for ik2, Ak in SK.get((ik, si), []):
                EK = np.matmul(E, Ak)                              # [n0, mb, mk']
                qk2 = _q(bk[y + 1], ik2)
                for so in range(4):
                    for ib2, Ab in SB.get((ib, so), []):
                        qb2 = _q(bb[y + 1], ib2)
                        c1 = mpo.class_of(y + 1, (qb2[0] - qk2[0], qb2[1] - qk2[1]))
                        if c1 < 0:
                            continue
                        Wb = W.get((c0, c1, so, si))
                        if Wb is None or Wb.nnz == 0:
                            continue
                        T = np.matmul(Ab.T, EK)                    # [n0, mb', mk']
                        Y = (Wb.T @ T.reshape(T.shape[0], -1)).reshape(Wb.shape[1], T.shape[1], T.shape[2])
                        key = (ib2, ik2)
                        if key in out:
                            out[key] += Y
                        else:
                            out[key] = Y
    return out


def update_right(mpo, R, bra, ket, y):
    """R_y from R_{y+1} and site y of the bra and ket MPS."""
    bb, bk = bra["bonds"], ket["bonds"]
    SB, SK = _site_by_right(bra["sites"][y]), _site_by_right(ket["sites"][y])
    W = mpo.W[y]
    out = {}
    for (ib2, ik2), E in R.items():
        qb2, qk2 = _q(bb[y + 1], ib2), _q(bk[y + 1], ik2)
        c1 = mpo.class_of(y + 1, (qb2[0] - qk2[0], qb2[1] - qk2[1]))
        for si in range(4):
            for ik, Ak in SK.get((ik2, si), []):
                EK = np.matmul(E, Ak.T)                            # [n1, mb', mk]
                qk = _q(bk[y], ik)
                for so in range(4):
                    for ib, Ab in SB.get((ib2, so), []):
                        qb = _q(bb[y], ib)
                        c0 = mpo.class_of(y, (qb[0] - qk[0], qb[1] - qk[1]))
                        if c0 < 0:
                            continue
                        Wb = W.get((c0, c1, so, si))
                        if Wb is None or Wb.nnz == 0:
                            continue
                        T = np.matmul(Ab, EK)                      # [n1, mb, mk]
                        Y = (Wb @ T.reshape(T.shape[0], -1)).reshape(Wb.shape[0], T.shape[1], T.shape[2])
                        key = (ib, ik)
                        if key in out:
                            out[key] += Y
                        else:
                            out[key] = Y
    return out


def environments(mpo, bra, ket, l):
    """Left environment at bond l and right environment at bond l+2."""
    k = len(bra["sites"])
    L = boundary_left(mpo)
    for y in range(l):
        L = update_left(mpo, L, bra, ket, y)
    R = boundary_right(mpo)
    for y in range(k - 1, l + 1, -1):
        R = update_right(mpo, R, bra, ket, y)
    return L, R


# ---------------------------------------------------------------------------
# the two-site local vector
# ---------------------------------------------------------------------------
def local_blocks(mps, l):
    """Block layout of the two-site local vector at position l: list of
    middle sectors (q, dimFL, dimFR, offset) in ascending q, and for every
    block (ia, s1, s2, ib) its (sector offset, dimFR, row offset, column
    offset, da, db).  Rows of a sector run over (s1 ascending, bond-l sector
    ascending, index), columns over (s2 ascending, bond-(l+2) sector
    ascending, index)."""
    bl, br = mps["bonds"][l], mps["bonds"][l + 2]
    m1, m2 = sorted(mps["masks"][l]), sorted(mps["masks"][l + 1])
    rows, cols = {}, {}
    for s in m1:
        for ia, (n, z, d) in enumerate(bl):
            q = (n + LOCAL_N[s], z + LOCAL_2SZ[s])
            rows.setdefault(q, []).append((s, ia, d))
    for s in m2:
        for ib, (n, z, d) in enumerate(br):
            q = (n - LOCAL_N[s], z - LOCAL_2SZ[s])
            cols.setdefault(q, []).append((s, ib, d))
    sectors, blocks, off = [], {}, 0
    for q in sorted(set(rows) & set(cols)):
        dl = sum(x[2] for x in rows[q])
        dr = sum(x[2] for x in cols[q])
        if dl == 0 or dr == 0:
            continue
        sectors.append((q, dl, dr, off))
        ro = 0
        for (s1, ia, da) in rows[q]:
            co = 0
            for (s2, ib, db) in cols[q]:
                blocks[(ia, s1, s2, ib)] = (off, dr, ro, co, da, db)
                co += db
            ro += da
        off += dl * dr
    return sectors, blocks, off


def _unpack(vec, blocks):
    out = {}
    for key, (off, dr, ro, co, da, db) in blocks.items():
        view = vec[off:].reshape(-1, dr) if False else None
        out[key] = vec[off + ro * dr: off + (ro + da) * dr].reshape(da, dr)[:, co:co + db]
    return out


def _pack(blocks_out, layout_blocks, n):
    vec = np.zeros(n)
    for key, blk in blocks_out.items():
        off, dr, ro, co, da, db = layout_blocks[key]
        vec[off + ro * dr: off + (ro + da) * dr].reshape(da, dr)[:, co:co + db] += blk
    return vec


def sigma(mpo, bra, ket, l, psi, L=None, R=None):
    """sigma = P_bra^T O P_ket psi at two-site position (l, l+1), psi in the
    ket's local layout, sigma in the bra's."""
    if L is None or R is None:
        L, R = environments(mpo, bra, ket, l)
    _, kblocks, nk = local_blocks(ket, l)
    _, bblocks, nb = local_blocks(bra, l)
    assert len(psi) == nk
    P = _unpack(np.asarray(psi, float), kblocks)
    bl, br = bra["bonds"], ket["bonds"]
    Wl, Wr = mpo.W[l], mpo.W[l + 1]
    # right environments grouped by ket sector at bond l+2
    Rk = {}
    for (ib, ik), E in R.items():
        Rk.setdefault(ik, []).append((ib, E))
    # step 1: Z1[(ka, s1, s2, jb)] = psi R^T  -> [n2, m_ka, m_jb] (class of (jb, kb))
    Z1 = {}
    for (ka, s1, s2, kb), blk in P.items():
        for jb, E in Rk.get(kb, []):
            qj, qk = _q(bl[l + 2], jb), _q(br[l + 2], kb)
            c2 = mpo.class_of(l + 2, (qj[0] - qk[0], qj[1] - qk[1]))
            Z = np.matmul(blk, np.transpose(E, (0, 2, 1)))       # [n2, m_ka, m_jb]
            key = (ka, s1, s2, jb)
            Z1[key] = Z1[key] + Z if key in Z1 else Z
    # step 2: site l+1:  Z2[(ka, s1, t2, jb)][w1] = sum W_{l+1}[w1, w2](t2, s2) Z1[w2]
    Z2 = {}
    for (ka, s1, s2, jb), Z in Z1.items():
        qj = _q(bl[l + 2], jb)
        c2 = mpo.class_of(l + 2, (qj[0] - (_q(br[l], ka)[0] + LOCAL_N[s1] + LOCAL_N[s2]),
                                  qj[1] - (_q(br[l], ka)[1] + LOCAL_2SZ[s1] + LOCAL_2SZ[s2])))
        for t2 in range(4):
            dq1 = (qj[0] - LOCAL_N[t2] - (_q(br[l], ka)[0] + LOCAL_N[s1]),
                   qj[1] - LOCAL_2SZ[t2] - (_q(br[l], ka)[1] + LOCAL_2SZ[s1]))
            c1 = mpo.class_of(l + 1, dq1)
            if c1 < 0:
                continue
            Wb = Wr.get((c1, c2, t2, s2))
            if Wb is None or Wb.nnz == 0:
                continue
            Y = (Wb @ Z.reshape(Z.shape[0], -1)).reshape(Wb.shape[0], Z.shape[1], Z.shape[2])
            key = (ka, s1, t2, jb)
            Z2[key] = Z2[key] + Y if key in Z2 else Y
    # step 3: site l:  Z3[(ka, t1, t2, jb)][w0] = sum W_l[w0, w1](t1, s1) Z2[w1]
    Z3 = {}
    for (ka, s1, t2, jb), Z in Z2.items():
        qa = _q(br[l], ka)
        qj = _q(bl[l + 2], jb)
        dq1 = (qj[0] - LOCAL_N[t2] - (qa[0] + LOCAL_N[s1]), qj[1] - LOCAL_2SZ[t2] - (qa[1] + LOCAL_2SZ[s1]))
        c1 = mpo.class_of(l + 1, dq1)
        for t1 in range(4):
            dq0 = (dq1[0] - LOCAL_N[t1] + LOCAL_N[s1], dq1[1] - LOCAL_2SZ[t1] + LOCAL_2SZ[s1])
            c0 = mpo.class_of(l, dq0)
            if c0 < 0:
                continue
            Wb = Wl.get((c0, c1, t1, s1))
            if Wb is None or Wb.nnz == 0:
                continue
            Y = (Wb @ Z.reshape(Z.shape[0], -1)).reshape(Wb.shape[0], Z.shape[1], Z.shape[2])
            key = (ka, t1, t2, jb)
            Z3[key] = Z3[key] + Y if key in Z3 else Y
    # step 4: left environment: sigma[(ja, t1, t2, jb)] = sum_{ka, w0} L[(ja, ka)][w0] Z3[w0]
    Lk = {}
    for (ja, ka), E in L.items():
        Lk.setdefault(ka, []).append((ja, E))
    out = {}
    for (ka, t1, t2, jb), Z in Z3.items():
        for ja, E in Lk.get(ka, []):
            key = (ja, t1, t2, jb)
            if key not in bblocks:
                continue
            S = np.einsum("wab,wbc->ac", E, Z, optimize=True)
            out[key] = out[key] + S if key in out else S
    return _pack(out, bblocks, nb)
