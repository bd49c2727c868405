"""CPU FP64 oracle for PCAL on the P2 finite-element Kohn-Sham problem.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import or run anything in this package.  The product
path (``libofks.so`` and its binding) never does; it shares no code with this package.

Plain, slow and written to be checked against the paper by eye: every function names
the passage it follows.  Library primitives (sparse/dense matrix products, a sparse
direct solve, a Cholesky factorization) serve as single steps; nothing is blocked,
fused or reordered beyond what the formulas state.

Modules
  fem      P2 basis, 4-point quadrature, assembly of L, B and potential matrices (Sec. 2.2)
  xc       Slater exchange + Perdew-Zunger 1981 correlation (LDA; Sec. 2.1, Sec. 4.1)
  hartree  FEM Poisson solve for the Hartree potential with multipole boundary data (Sec. 2.2)
  pcal     Hamiltonian, energies, Alg. 2 (PCAL) with Eq. (lambda2), Eq. (PCAL-main),
           the preconditioner Eq. (precondition-T), BB2 step (Sec. 4.4), stopping test
           (Sec. 4.1), Cholesky-based initial guess (Sec. 4.2), Rayleigh-Ritz (Sec. 4.3)
  dense    generalized symmetric eigensolver (Cholesky + cyclic Jacobi) and a dense
           linear-mixing SCF used as an independent fixed-point check

Pins (``tests/test_oracle_*.py``, all ``-m "not gpu"``): exact polynomial integrals of
the P2 space, Gaussian-charge Hartree closed form, LDA thermodynamic identity and
uniform-gas values, hydrogenic eigenvalues, dense generalized eigenproblem, dense SCF
fixed point, the paper's invariants (diag(X^T B X) = 1 after each step, fea ~ 1e-15 at
p = 1, Rayleigh-Ritz leaves E unchanged, symmetric multipliers).

Parity unpinned: the absolute physical energies of the paper's molecules (its meshes and
geometries are unavailable; a loose plausibility check on LiH is all that remains).
"""
