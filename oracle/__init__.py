"""Plain FP64 CPU oracle for the THC-RR-CCSD residual.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

Modules
-------
integrals     T1 dressing of Cholesky vectors (Eqs. 24-27), ERI blocks,
              core Hamiltonian back-out and dressed Fock matrix.
closed_shell  Closed-shell T1-dressed CCSD residual as the paper's per-term
              equations (Eqs. 28-42) on full 4-index tensors, and the energy.
thc           THC amplitudes (Eq. 23), projection onto the amplitude factors
              (Eq. 6 with Eq. 14), metric eigenbasis (Eqs. 9-14).
spin_orbital  Independent spin-orbital CCSD (Stanton-Gauss intermediates)
              used to pin the closed-shell algebra.
fci           Two-electron full CI (pins CCSD with one occupied orbital).
solver        Jacobi + DIIS drivers for canonical and THC-projected CCSD.
density       MP2-like one-particle density matrices (App. II, Eqs. 47-48).
mlp           Float64 reference of the learned preconditioner's network.
"""
