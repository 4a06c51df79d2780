"""Oracle for the orbital minimization method (OMM) of Corsetti (arXiv:1312.1549).

TEST INFRASTRUCTURE ONLY. Nothing in the product (the CUDA library and its
Python binding) may import, call or link anything in this package; only the
tests, `__graft_entry__.smoke()` and the bench's CPU-baseline leg use it.

Contents (all plain float64 CPU code, written from the paper):

* `exact`  -- the result the OMM converges to, by its plain definition: the n
  lowest generalised eigenpairs of H x = eps S x (Sec. 2.1, Eqs. 1 and 7-8).
* `jacobi` -- a self-contained cyclic Jacobi eigensolver with Cholesky
  reduction, used to pin `exact` on tiny inputs without any library solver.
* `omm`    -- the OMM itself, step by step: eigenspectrum shift (Sec. 2.2, Eq. 9),
  CG with Polak-Ribiere directions, the gradient (Eq. 12), the quartic line
  search with directly computed coefficients (Eqs. 13-15), the state update
  (Eq. 16), the kinetic preconditioner (Eq. 17), the outputs, and the
  Cholesky flavour (reduction to standard form, end of Sec. 2.4).
* `hermitian` -- the same steps in complex arithmetic with Hermitian
  conjugates, as the paper writes them (Secs. 2.1-2.3), for k-point problems.

Parity status: every function here is pinned by a test in
tests/test_oracle_pins.py, tests/test_oracle_hermitian.py and tests/test_oracle_cg_pins.py (the
Polak-Ribiere coefficient, through its equality with the Hestenes-Stiefel one under exact line
searches) against brute force, closed forms, finite differences or invariants; none is "parity
unpinned" except the CG iteration count, which the paper does not fix.
"""
