"""Brute-force Fock-space Hamiltonian from qubit Jordan-Wigner matrices.

Used only to pin the signs of ``oracle.fci`` (and the MPO contraction) on
tiny systems: a_j = Z x ... x Z x a x 1 x ... x 1 over 2k spin-orbital qubits
(qubit 0 = spin orbital 0 is the most significant tensor factor).  The
Hamiltonian is Eq. "part" of the Theory section written with the 1/2 of the
spin-orbital expansion of chemists' integrals.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_Z = sp.csr_matrix(np.diag([1.0, -1.0]))
_I = sp.identity(2, format="csr")
_a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |1> -> |0>


def annihilator(j: int, n_qubits: int) -> sp.csr_matrix:
    op = None
    for q in range(n_qubits):
        f = _Z if q < j else (_a if q == j else _I)
        op = f if op is None else sp.kron(op, f, format="csr")
    return op


def fock_hamiltonian(h: np.ndarray, V: np.ndarray) -> sp.csr_matrix:
    k = h.shape[0]
    nq = 2 * k
    a = [annihilator(j, nq) for j in range(nq)]
    ad = [x.T.tocsr() for x in a]
    H = sp.csr_matrix((2 ** nq, 2 ** nq))
    for p in range(k):
        for q in range(k):
            if h[p, q] != 0.0:
                for s in (0, 1):
                    H = H + h[p, q] * (ad[2 * p + s] @ a[2 * q + s])
    for p in range(k):
        for q in range(k):
            for r in range(k):
                for t in range(k):
                    v = V[p, q, r, t]
                    if v == 0.0:
                        continue
                    for s1 in (0, 1):
                        for s2 in (0, 1):
                            H = H + 0.5 * v * (ad[2 * p + s1] @ ad[2 * r + s2]
                                               @ a[2 * t + s2] @ a[2 * q + s1])
    return H.tocsr()


def qubit_index(mask: int, n_qubits: int) -> int:
    """Kronecker index of the basis state whose spin orbital j is occupied
    when bit j of ``mask`` is set (spin orbital 0 = most significant)."""
    x = 0
    for j in range(n_qubits):
        if (mask >> j) & 1:
            x |= 1 << (n_qubits - 1 - j)
    return x
