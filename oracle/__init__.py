"""CPU oracle for four-component LR-CCSD polarizabilities (test infrastructure).

This package is test infrastructure.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path: it is a plain, slow, complex128 restatement of the method in
PyTorch CPU ops and numpy, written to be checked by eye against the paper.

Modules
-------
``ccsd``  spin-orbital CCSD residual and energy for a general (non-canonical)
          Fock matrix, MP2, the ground-state T and left Lambda solves, and the
          linear-response pieces xi, eta, F.X, X(omega), Y(omega) and alpha
          (Sec. II.A, Eq. 9-10 and Eq. 29-35).
``fci``   determinant-space second quantisation: the projected residual
          <mu| e^-T H e^T |0> by brute force, FCI and the sum-over-states
          response function (Eq. 18).  Used only to pin ``ccsd``.
``fns``   FNS++ truncation: MP2, first-order perturbed amplitudes, the
          perturbation-sensitive density, natural spinors, semicanonical
          rotation (Sec. II.B-C, Eq. 39-50).

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute force, FCI, invariances); see the
``tests/test_oracle_*.py`` files.
"""
