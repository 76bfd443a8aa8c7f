"""CPU FP64 oracle for the MPS-LCC hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, obviously-correct restatement of what the
method computes, used to check the GPU library.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it;
the library itself never does, and this package never imports the library.

Modules
-------
``fci``   determinant space: the second-quantised Hamiltonian of the Theory
          section (Eq. "part"), the Fink partition H = H0 + U by excitation
          class, full CI and the reference (CAS-CI) eigenproblem.
``lcc``   first-order perturbation theory of Eq. 1 (n = 1) in the projector
          form of the "Projector approximation" paragraph, the Wigner 2n+1
          energies of Eq. 2 (E2, E3), the Hylleraas value of Eq. 1b, and the
          single-reference (zero active orbitals) limit as an explicit singles
          + doubles linear solve (Eqs. lccE / lccT family).
``mps``   expansion of a block-sparse MPS (Eq. mps1) into determinants and the
          local problem of the Implementation section: the isometry P of a
          two-site position and the dense effective Hamiltonian P^T H P.
``fock``  brute-force Fock space from qubit Jordan-Wigner matrices, used only
          to pin the determinant-space Hamiltonian's signs.

Parity pins live in ``tests/test_oracle_*.py`` (closed forms, limits,
invariants, brute force).
"""
