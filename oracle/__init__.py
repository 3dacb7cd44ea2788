"""CPU oracle for the FFT-based fast direct Helmholtz solver (arXiv 1809.03808).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` use it.

What it computes, in FP64 (double-double where stated), sharing no code with
the CUDA path:

* ``fem``      -- the discrete operator A of Section 2 assembled element by
                  element from bilinear/trilinear elements by Gauss quadrature
                  of the weak form (eq. helmholtzWeak / bf-1st-order-abc), the
                  1D matrices of eqs. matrixK/matrixM, the circulant matrices
                  of eqs. matrixKper/matrixMper, the Kronecker forms of eqs.
                  A2D/A3D/B2D/B3D, and closed-form 1D eigenvalues (eq.
                  eigvaluesPer and the Neumann/Dirichlet analogues).
* ``solvers``  -- O1: banded LU with partial pivoting of the assembled A;
                  O2: tensor-product eigen-solve (dense generalized eigen-
                  decomposition on all axes but one, normalised as in eq.
                  EVPcondA, tridiagonal LU on the remaining axis); both
                  followed by iterative refinement with a double-double
                  residual.  Also the plain definitions of the intermediate
                  quantities of the three-step solve (Section 3.1): v = B^-1 f,
                  w = A^-1 (B - A) v, and their boundary rows.
* ``dd``       -- double-double (Dekker/Knuth error-free) arithmetic used for
                  residuals.

Every function states the passage it follows.  Pins (closed forms, brute
force, invariants) live in tests/test_oracle_pins.py.

Parity unpinned: none of the paper's printed numbers is a solution value --
the paper prints only CPU timings (Section 6, Tables tab2d..tab3d_2) -- so no
output is pinned to a value printed in the paper; every function here is
pinned instead to closed forms, brute force and invariants.
"""
