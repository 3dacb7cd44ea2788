"""Pins for the CPU oracle: closed forms, brute force and invariants.

Each test ties an oracle function to something other than itself, chosen so
that a plausible slip (dropped term, wrong sign or index, transposed operand)
fails at least one of them.  CPU only.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import dd, fem, solvers
from workloads import random_rhs

RNG = np.random.default_rng(12345)


# --------------------------- double-double ---------------------------------

def test_dd_two_prod_and_two_sum_are_exact():
    """Dekker/Knuth transformations: p + e == a*b and s + e == a + b exactly
    (checked in rational arithmetic)."""
    a = RNG.standard_normal(200) * 10.0 ** RNG.integers(-8, 8, 200)
    b = RNG.standard_normal(200) * 10.0 ** RNG.integers(-8, 8, 200)
    p, e = dd.two_prod(a, b)
    s, t = dd.two_sum(a, b)
    for i in range(200):
        assert Fraction(p[i]) + Fraction(e[i]) == Fraction(a[i]) * Fraction(b[i])
        assert Fraction(s[i]) + Fraction(t[i]) == Fraction(a[i]) + Fraction(b[i])


def test_residual_dd_matches_rational_arithmetic():
    """f - A u in double-double equals the exact rational residual of the
    operator with the same double entries, to ~1e-30 relative."""
    shape, h, om = (4, 5), (0.31, 0.27), 3.7
    u = random_rhs(shape, 1)
    f = fem.apply_A(u, h, om) + 1e-12 * random_rhs(shape, 2)
    r = fem.residual_dd(f, u, h, om)
    # exact: build 1D matrices in Fractions with the same double entries
    def mats(n, hh, kind):
        sub, diag, sup = fem._tri_coeffs(n, hh, om, kind)
        M = [[(Fraction(0), Fraction(0)) for _ in range(n)] for _ in range(n)]
        for j in range(n):
            M[j][j] = (Fraction(diag[j].real), Fraction(diag[j].imag))
            if j > 0:
                M[j][j - 1] = (Fraction(sub[j].real), Fraction(sub[j].imag))
            if j < n - 1:
                M[j][j + 1] = (Fraction(sup[j].real), Fraction(sup[j].imag))
        return M

    def cmul(a, b):
        return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])

    def apply(M, X, axis):
        n0, n1 = len(X), len(X[0])
        Y = [[(Fraction(0), Fraction(0)) for _ in range(n1)] for _ in range(n0)]
        for i in range(n0):
            for j in range(n1):
                acc = (Fraction(0), Fraction(0))
                for k in range(n0 if axis == 0 else n1):
                    m = M[i][k] if axis == 0 else M[j][k]
                    x = X[k][j] if axis == 0 else X[i][k]
                    if m != (0, 0):
                        t = cmul(m, x)
                        acc = (acc[0] + t[0], acc[1] + t[1])
                Y[i][j] = acc
        return Y

    U = [[(Fraction(u[i, j].real), Fraction(u[i, j].imag)) for j in range(shape[1])] for i in range(shape[0])]
    Kx, Mx = mats(shape[0], h[0], "K"), mats(shape[0], h[0], "M")
    Ky, My = mats(shape[1], h[1], "K"), mats(shape[1], h[1], "M")
    t1 = apply(Kx, apply(My, U, 1), 0)
    t2 = apply(Mx, apply(Ky, U, 1), 0)
    t3 = apply(Mx, apply(My, U, 1), 0)
    w2 = Fraction(-om ** 2)
    for i in range(shape[0]):
        for j in range(shape[1]):
            ex_re = Fraction(f[i, j].real) - (t1[i][j][0] + t2[i][j][0] + w2 * t3[i][j][0])
            ex_im = Fraction(f[i, j].imag) - (t1[i][j][1] + t2[i][j][1] + w2 * t3[i][j][1])
            assert abs(float(ex_re) - r[i, j].real) <= 1e-26 + 1e-15 * abs(float(ex_re))
            assert abs(float(ex_im) - r[i, j].imag) <= 1e-26 + 1e-15 * abs(float(ex_im))


# --------------------------- 1D matrices -------------------------------------

def test_1d_matrices_match_element_assembly():
    """eqs. matrixK / matrixM are the 1D element assembly of the weak form
    (including the -i w boundary term at both ends)."""
    n, h, om = 7, 0.2, 3.0
    A1 = fem.assemble((n,), (h,), om).toarray()
    K, M = fem.K1d(n, h, om), fem.M1d(n, h)
    np.testing.assert_allclose(A1, K - om ** 2 * M, atol=1e-13)
    # hand values of the paper's stencils
    assert K[0, 0] == pytest.approx((1 - 1j * om * h) / h)
    assert K[3, 3] == pytest.approx(2 / h) and K[3, 4] == pytest.approx(-1 / h)
    assert M[0, 0] == pytest.approx(2 * h / 6) and M[3, 3] == pytest.approx(4 * h / 6)
    assert M[3, 2] == pytest.approx(h / 6)


@pytest.mark.parametrize("shape,h", [((6, 5), (0.2, 0.3)), ((4, 5, 3), (0.5, 0.25, 0.4)),
                                     ((9, 2), (0.125, 1.0))])
@pytest.mark.parametrize("bc", ["abc", "neumann"])
def test_element_assembly_equals_kronecker_form(shape, h, bc):
    """Element-by-element assembly by quadrature == eq. A2D / A3D."""
    om = 4.1
    A1 = fem.assemble(shape, h, om, bc)
    A2 = fem.kron_operator(shape, h, om, bc=bc)
    assert abs(A1 - A2).max() < 1e-12 * abs(A2).max()


def test_operator_is_complex_symmetric_not_hermitian():
    A = fem.assemble((5, 6), (0.25, 0.2), 5.0)
    assert abs(A - A.T).max() == 0 or abs(A - A.T).max() < 1e-15
    assert abs(A - A.conj().T).max() > 1.0  # the -i w boundary term


def test_apply_A_matches_assembled_matrix():
    shape, h, om = (5, 4, 6), (0.3, 0.2, 0.25), 2.5
    u = random_rhs(shape, 3)
    A = fem.assemble(shape, h, om)
    np.testing.assert_allclose(fem.apply_A(u, h, om).ravel(), A @ u.ravel(), rtol=0, atol=1e-12)


# --------------------------- closed-form eigenvalues -------------------------

@pytest.mark.parametrize("n,h", [(9, 0.125), (33, 1 / 32), (16, 0.07)])
def test_neumann_and_dirichlet_closed_forms(n, h):
    """Linear-FEM eigenvalues 6/h^2 (1 - cos t)/(2 + cos t): Neumann with
    t = k pi/(n-1), Dirichlet (interior block) with t = k pi h / L."""
    K = fem.K1d(n, h, 0.0, bc="neumann").real
    M = fem.M1d(n, h)
    ev = np.sort(sl.eigh(K, M, eigvals_only=True))
    np.testing.assert_allclose(ev, np.sort(fem.eig_neumann(n, h)), rtol=1e-10, atol=1e-9)
    evd = np.sort(sl.eigh(K[1:-1, 1:-1], M[1:-1, 1:-1], eigvals_only=True))
    np.testing.assert_allclose(evd, np.sort(fem.eig_dirichlet(n, h)), rtol=1e-10)


@pytest.mark.parametrize("n,h", [(8, 0.1), (9, 1 / 8), (31, 0.03)])
def test_periodic_pencil_eigenvalues_and_dft_diagonalisation(n, h):
    """eq. eigvaluesPer equals the closed form, and the DFT matrix of eq.
    eigvectorsPer diagonalises the circulant K^B, M^B (eqs. matrixKper/Mper)."""
    lam = fem.eig_periodic(n, h)
    np.testing.assert_allclose(lam, fem.eig_periodic_closed(n, h), rtol=1e-12, atol=1e-9)
    KB, MB = fem.K1d_periodic(n, h), fem.M1d_periodic(n, h)
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    Fi = np.conj(F) / n
    DK = F @ KB @ Fi
    DM = F @ MB @ Fi
    assert np.abs(DK - np.diag(np.diag(DK))).max() < 1e-10 / h
    assert np.abs(DM - np.diag(np.diag(DM))).max() < 1e-12
    np.testing.assert_allclose(np.diag(DK).real / np.diag(DM).real, lam, rtol=1e-10, atol=1e-8)
    # the paper's FFT convention (eq. step1FFTfcoeff) is numpy's forward FFT
    x = random_rhs((n,), 4)
    naive = np.array([sum(np.exp(-2j * np.pi * l * k / n) * x[l] for l in range(n)) for k in range(n)])
    np.testing.assert_allclose(np.fft.fft(x), naive, rtol=1e-12, atol=1e-12)


def test_abc_pencil_eigenpairs():
    """eq. EVP1a with eq. EVPcondA: K V = M V Lam, V^T M V = I, V^T K V = Lam;
    and the w -> 0 limit reduces to the Neumann closed form."""
    n, h = 41, 1 / 40
    om = 2 * np.pi / (10 * h)
    lam, V = solvers.abc_pencil_eig(n, h, om)
    K, M = fem.K1d(n, h, om), fem.M1d(n, h)
    assert np.abs(K @ V - M @ V * lam[None, :]).max() < 1e-9 * np.abs(K).max()
    assert np.abs(V.T @ M @ V - np.eye(n)).max() < 1e-10
    assert np.abs(V.T @ K @ V - np.diag(lam)).max() < 1e-9 * np.abs(lam).max()
    # absorbing: every eigenvalue is pushed into the lower half plane
    assert np.all(lam.imag < 0)
    lam0, _ = solvers.abc_pencil_eig(n, h, 1e-9)
    np.testing.assert_allclose(np.sort(lam0.real), np.sort(fem.eig_neumann(n, h)), rtol=1e-8, atol=1e-6)


# --------------------------- solvers -----------------------------------------

@pytest.mark.parametrize("shape,h,om", [((7, 9), (1 / 6, 1 / 8), 9.0),
                                         ((5, 6, 4), (0.25, 0.2, 1 / 3), 6.0),
                                         ((12, 3), (0.1, 0.4), 15.0)])
def test_banded_and_tensor_agree_with_dense_lu(shape, h, om):
    f = random_rhs(shape, 7)
    u0 = solvers.solve_dense(f, h, om)
    u1 = solvers.solve_banded_lu(f, h, om)
    u2 = solvers.TensorSolver(shape, h, om).solve(f)
    n0 = np.linalg.norm(u0)
    assert np.linalg.norm(u1 - u0) / n0 < 1e-12
    assert np.linalg.norm(u2 - u0) / n0 < 1e-11
    # tensor solver with every choice of the tridiagonal axis
    for t in range(len(shape)):
        u3 = solvers.TensorSolver(shape, h, om, tri_axis=t).solve(f)
        assert np.linalg.norm(u3 - u0) / n0 < 1e-11


@pytest.mark.parametrize("k,m", [(0, 0), (3, 2), (5, 7)])
def test_separable_closed_form_neumann(k, m):
    """Neumann on all faces: f = (M1 phi_k) (x) (M2 phi_m) gives
    u = phi_k (x) phi_m / (lam_k + lam_m - w^2), phi cosines (closed form)."""
    n1, n2, h1, h2, om = 9, 11, 0.125, 0.1, 3.3
    phik = np.cos(k * np.pi * np.arange(n1) / (n1 - 1))
    phim = np.cos(m * np.pi * np.arange(n2) / (n2 - 1))
    lam = fem.eig_neumann(n1, h1)[k] + fem.eig_neumann(n2, h2)[m]
    f = np.outer(fem.M1d(n1, h1) @ phik, fem.M1d(n2, h2) @ phim).astype(complex)
    u = solvers.solve_banded_lu(f, (h1, h2), om, bc="neumann")
    np.testing.assert_allclose(u, np.outer(phik, phim) / (lam - om ** 2), rtol=1e-11, atol=1e-12)


def test_reciprocity():
    """A is complex symmetric, so g^T A^-1 f = f^T A^-1 g."""
    shape, h, om = (10, 13), (0.1, 1 / 12), 12.0
    f, g = random_rhs(shape, 8), random_rhs(shape, 9)
    uf = solvers.solve_banded_lu(f, h, om)
    ug = solvers.solve_banded_lu(g, h, om)
    a, b = np.sum(g * uf), np.sum(f * ug)
    assert abs(a - b) < 1e-12 * abs(a)


def test_plane_wave_second_order_convergence():
    """Manufactured plane wave with absorbing data: nodal error falls ~4x per
    halving of h (linear elements, second order)."""
    om, direction = 2 * np.pi, (math.cos(0.4), math.sin(0.4))
    errs = []
    for n in (17, 33, 65, 129):
        h = (1 / (n - 1),) * 2
        f, ue = fem.plane_wave_load((n, n), h, om, direction)
        u = solvers.solve_banded_lu(f, h, om)
        errs.append(np.linalg.norm(u - ue) / np.linalg.norm(ue))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 2e-3
    assert all(3.5 < r < 4.5 for r in ratios[1:]), (errs, ratios)


def test_plane_wave_3d_converges():
    om, direction = 2 * np.pi, (0.3, 0.5, 0.8)
    errs = []
    for n in (9, 17):
        h = (1 / (n - 1),) * 3
        f, ue = fem.plane_wave_load((n, n, n), h, om, direction)
        u = solvers.solve_banded_lu(f, h, om)
        errs.append(np.linalg.norm(u - ue) / np.linalg.norm(ue))
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_refinement_reaches_double_precision():
    shape, h, om = (33, 65), (1 / 32, 1 / 64), 2 * np.pi / (10 / 64)
    f = random_rhs(shape, 10)
    u, hist = solvers.oracle_solve(f, h, om, method="tensor")
    assert hist[-1] < 1e-14
    ub = solvers.solve_banded_lu(f, h, om)
    assert np.linalg.norm(u - ub) / np.linalg.norm(ub) < 1e-12


# --------------------------- Section 3.1 structure ---------------------------

@pytest.mark.parametrize("shape,axis", [((7, 9), 1), ((7, 9), 0), ((5, 4, 6), 2)])
def test_three_step_identities(shape, axis):
    """B - A is supported on the boundary rows of the periodic axis only (eq.
    BminA), and u = v + w after Step 2 (Section 3.1)."""
    h = tuple(1.0 / (n - 1) for n in shape)
    om = 7.0
    A = fem.kron_operator(shape, h, om)
    B = fem.kron_operator(shape, h, om, periodic_axis=axis)
    D = (B - A).tocoo()
    idx = np.array(np.unravel_index(np.arange(A.shape[0]), shape))
    onb = (idx[axis] == 0) | (idx[axis] == shape[axis] - 1)
    keep = np.abs(D.data) > 0
    assert np.all(onb[D.row[keep]]) and np.all(onb[D.col[keep]])
    f = random_rhs(shape, 11)
    v, w, u = solvers.step_definitions(f, h, om, axis)
    assert np.linalg.norm(v + w - u) / np.linalg.norm(u) < 1e-12


@pytest.mark.parametrize("shape,h", [((7, 9), (0.2, 0.13)), ((5, 6, 4), (0.3, 0.2, 0.25)),
                                     ((40, 33), (0.01, 0.02)), ((3, 3, 3), (1.0, 0.5, 0.25))])
def test_c_residual_equals_pinned_numpy_residual(shape, h):
    """The C double-double residual (for large grids) reproduces the numpy one,
    which is pinned to exact rational arithmetic above."""
    u = random_rhs(shape, 1)
    f = fem.apply_A(u, h, 3.3) + 1e-9 * random_rhs(shape, 2)
    r1 = fem.residual_dd(f, u, h, 3.3)
    r2 = fem.residual_dd_c(f, u, h, 3.3)
    assert np.array_equal(r1, r2)


@pytest.mark.parametrize("n,h,rho,phi", [(8, 0.1, 1.0, np.pi / 2), (9, 1 / 8, 0.5, 0.0), (31, 0.03, 2.0, np.pi)])
def test_gamma_circulant_is_diagonalised_by_scaled_dft(n, h, rho, phi):
    """The damped auxiliary: with gamma = e^{rho + i phi} and t = (rho + i phi)/n,
    F D^-1 K^B_gamma D F^-1 is diagonal with D = diag(e^{t j}), eigenvalues
    (2 - 2 cosh(t + i theta_l))/h and h (4 + 2 cosh(t + i theta_l))/6
    (gamma = 1 reduces to eq. eigvaluesPer)."""
    g = np.exp(rho + 1j * phi)
    t = (rho + 1j * phi) / n
    KB, MB = fem.K1d_periodic(n, h, g), fem.M1d_periodic(n, h, g)
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    D = np.diag(np.exp(t * np.arange(n)))
    Di = np.diag(np.exp(-t * np.arange(n)))
    Fi = np.conj(F) / n
    th = 2 * np.pi * np.arange(n) / n
    for Mat, ev in ((KB, (2 - 2 * np.cosh(t + 1j * th)) / h), (MB, h * (4 + 2 * np.cosh(t + 1j * th)) / 6)):
        Dg = F @ Di @ Mat @ D @ Fi
        assert np.abs(Dg - np.diag(np.diag(Dg))).max() < 1e-10 * np.abs(ev).max()
        np.testing.assert_allclose(np.diag(Dg), ev, rtol=1e-10, atol=1e-10 * np.abs(ev).max())
    # gamma = 1 is the paper's circulant
    assert np.allclose(fem.K1d_periodic(n, h, 1.0), fem.K1d_periodic(n, h).real)


def test_damped_auxiliary_step_identities():
    """u = v + w also holds with the gamma-circulant auxiliary (B - A stays on
    the boundary rows of the periodic axis)."""
    shape, h, om = (7, 9), (1 / 6, 1 / 8), 7.0
    f = random_rhs(shape, 12)
    g = np.exp(1.0 + 0.5j * np.pi)
    v, w, u = solvers.step_definitions(f, h, om, axis=1, gamma=g)
    assert np.linalg.norm(v + w - u) / np.linalg.norm(u) < 1e-12
    A = fem.kron_operator(shape, h, om)
    B = fem.kron_operator(shape, h, om, periodic_axis=1, gamma=g)
    D = (B - A).tocoo()
    keep = np.abs(D.data) > 0
    iy = np.unravel_index(np.arange(A.shape[0]), shape)[1]
    onb = (iy == 0) | (iy == shape[1] - 1)
    assert np.all(onb[D.row[keep]]) and np.all(onb[D.col[keep]])


# --------------------------- mixed absorbing / Neumann axes -----------------

MIXED = [((6, 5), (0.2, 0.3), ("neumann", "abc")), ((6, 5), (0.2, 0.3), ("abc", "neumann")),
         ((4, 5, 3), (0.5, 0.25, 0.4), ("abc", "neumann", "abc")),
         ((4, 5, 3), (0.5, 0.25, 0.4), ("neumann", "neumann", "abc"))]


@pytest.mark.parametrize("shape,h,bc", MIXED)
def test_mixed_boundaries_assembly_and_operators(shape, h, bc):
    """Gamma_N on some axes (Section 2, k11 = 1 in eq. matrixK): the element
    assembly (boundary mass only on absorbing faces) equals the Kronecker form
    with per-axis K corners, and apply_A / residual_dd (numpy and C) apply that
    same matrix."""
    om = 3.7
    A1 = fem.assemble(shape, h, om, bc)
    A2 = fem.kron_operator(shape, h, om, bc=bc)
    assert abs(A1 - A2).max() < 1e-12 * abs(A2).max()
    # a Neumann axis has real corners: the boundary term is only on absorbing faces
    assert abs(A1 - fem.assemble(shape, h, om, "abc")).max() > 0.1
    u = random_rhs(shape, 5)
    np.testing.assert_allclose(fem.apply_A(u, h, om, bc).ravel(), A1 @ u.ravel(), rtol=0, atol=1e-12)
    f = fem.apply_A(u, h, om, bc) + 1e-9 * random_rhs(shape, 6)
    r1 = fem.residual_dd(f, u, h, om, bc)
    np.testing.assert_allclose(r1.ravel(), f.ravel() - A1 @ u.ravel(), rtol=0, atol=1e-13)
    assert np.array_equal(r1, fem.residual_dd_c(f, u, h, om, bc))


@pytest.mark.parametrize("shape,h,bc", MIXED)
def test_mixed_boundaries_solvers_agree_with_dense_lu(shape, h, bc):
    om = 5.1
    f = random_rhs(shape, 8)
    u0 = solvers.solve_dense(f, h, om, bc)
    n0 = np.linalg.norm(u0)
    assert np.linalg.norm(solvers.solve_banded_lu(f, h, om, bc) - u0) / n0 < 1e-12
    for t in range(len(shape)):
        u3 = solvers.TensorSolver(shape, h, om, tri_axis=t, bc=bc).solve(f)
        assert np.linalg.norm(u3 - u0) / n0 < 1e-11
    u4, hist = solvers.oracle_solve(f, h, om, method="tensor", bc=bc)
    assert np.linalg.norm(u4 - u0) / n0 < 1e-12 and hist[-1] < 1e-14


def test_neumann_pencil_eigen_is_the_cosine_basis():
    """abc_pencil_eig of a Neumann axis: eigenvalues of the closed form and
    V^T M V = I with V[0, k]^2 = V[n-1, k]^2 (cosines, parity (-1)^k)."""
    n, h = 12, 0.09
    lam, V = solvers.abc_pencil_eig(n, h, 4.0, "neumann")
    np.testing.assert_allclose(np.sort(lam.real), np.sort(fem.eig_neumann(n, h)), rtol=1e-10, atol=1e-8)
    M = fem.M1d(n, h)
    np.testing.assert_allclose(V.T @ M @ V, np.eye(n), atol=1e-10)
    np.testing.assert_allclose(V[0] ** 2, V[-1] ** 2, rtol=1e-8, atol=1e-12)


# --------------------------- cost-model network (autotuner) ------------------

def test_mlp_oracle_gradient_matches_finite_differences():
    """The numpy reference of the cost model's backprop against central
    differences of its own loss (every parameter)."""
    from oracle import mlp

    rng = np.random.default_rng(3)
    n_in, n_h, B = 5, 7, 11
    p = rng.standard_normal(mlp.num_params(n_in, n_h)) * 0.5
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal(B)
    L, g = mlp.loss_and_gradient(p, X, T, n_in, n_h)
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = eps
        fd[i] = (mlp.loss_and_gradient(p + e, X, T, n_in, n_h)[0] - mlp.loss_and_gradient(p - e, X, T, n_in, n_h)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_mlp_oracle_forward_by_hand():
    """One sample through a 1-input, 1-wide network, written out."""
    from oracle import mlp

    p = np.array([0.3, -0.1, 0.7, 0.2, -1.5, 0.25])  # W1, b1, W2, b2, w3, b3
    y, _ = mlp.forward(p, np.array([[2.0]]), 1, 1)
    h1 = np.tanh(0.3 * 2.0 - 0.1)
    h2 = np.tanh(0.7 * h1 + 0.2)
    assert y[0] == pytest.approx(-1.5 * h2 + 0.25, abs=1e-15)


# ------------------ the modified (reduced-dispersion) elements -------------

def test_modified_element_1d_matrices_by_hand():
    """The modified rule's 1D mass: h/12 (1, 10, 1) with corners 5h/12 (the
    mean of the consistent and the lumped mass); the stiffness is unchanged
    (the quadrature integrates the constant derivatives exactly)."""
    n, h = 5, 0.3
    M = fem.M1d(n, h, "q1mod")
    ref = (np.diag([5, 10, 10, 10, 5]) + np.eye(n, k=1) + np.eye(n, k=-1)) * h / 12
    np.testing.assert_allclose(M, ref, rtol=1e-15, atol=0)
    Mc, Ml = fem.M1d(n, h, "q1"), np.diag([0.5, 1, 1, 1, 0.5]) * h
    np.testing.assert_allclose(M, 0.5 * (Mc + Ml), rtol=1e-14, atol=1e-16)
    # element assembly in 1D reproduces it
    A1 = fem.assemble((n,), (h,), 0.0, "neumann", elem="q1mod").toarray()
    A2 = fem.assemble((n,), (h,), 1.0, "neumann", elem="q1mod").toarray()
    np.testing.assert_allclose(A1 - A2, M, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("shape,h,bc", [((5, 7), (0.3, 0.2), "abc"), ((6, 4), (0.1, 0.25), ("neumann", "abc")),
                                        ((4, 5, 3), (0.2, 0.15, 0.3), "abc"),
                                        ((3, 4, 5), (0.3, 0.2, 0.1), ("abc", "neumann", "abc"))])
def test_modified_element_assembly_equals_kronecker_form(shape, h, bc):
    """Element-by-element assembly with the modified rule (every integral,
    boundary mass included) equals the Kronecker form with the modified 1D
    mass on every axis: the tensor structure the fast solver needs."""
    om = 3.7
    A = fem.assemble(shape, h, om, bc, elem="q1mod").toarray()
    B = fem.kron_operator(shape, h, om, bc=bc, elem="q1mod").toarray()
    assert np.abs(A - B).max() <= 1e-12 * np.abs(B).max()
    assert np.abs(A - fem.assemble(shape, h, om, bc).toarray()).max() > 1e-3 * np.abs(B).max()
    u = random_rhs(shape, 3)
    np.testing.assert_allclose(fem.apply_A(u, h, om, bc, elem="q1mod").ravel(), B @ u.ravel(), rtol=1e-12, atol=1e-12)


def test_modified_element_dispersion_is_fourth_order():
    """A sampled plane wave exp(i k d.x) with |k| = w makes the interior
    stencil's defect (A u) / ((M (x) M) u) = sum_j K^_j/M^_j - w^2 vanish to
    fourth order in w h for the modified elements, to second order for the
    paper's (the defect falls ~16x and ~4x per halving of h)."""
    om, d = 20.0, np.array([np.cos(0.7), np.sin(0.7)])
    defects = {}
    for elem in ("q1", "q1mod"):
        out = []
        for n in (41, 81, 161):
            h = (1.0 / (n - 1),) * 2
            x = np.meshgrid(*[np.arange(n) * hh for hh in h], indexing="ij")
            u = np.exp(1j * om * (d[0] * x[0] + d[1] * x[1]))
            Au = fem.apply_A(u, h, om, "neumann", elem=elem)
            Mu = fem.apply_1d(fem.apply_1d(u, 0, n, h[0], om, "M", "neumann", elem), 1, n, h[1], om, "M", "neumann",
                              elem)
            c = n // 2
            out.append(abs(Au[c, c] / Mu[c, c]) / om ** 2)
        defects[elem] = out
    r2 = [defects["q1"][i] / defects["q1"][i + 1] for i in range(2)]
    r4 = [defects["q1mod"][i] / defects["q1mod"][i + 1] for i in range(2)]
    assert all(3.8 < r < 4.2 for r in r2), defects
    assert all(15.0 < r < 17.0 for r in r4), defects
    assert defects["q1mod"][-1] < 1e-3 * defects["q1"][-1]


@pytest.mark.parametrize("n,h", [(9, 0.125), (16, 0.07)])
def test_modified_element_closed_form_eigenvalues(n, h):
    """Neumann pencil with the modified mass: the cosine closed form equals
    LAPACK's generalised symmetric eigenvalues."""
    K = fem.K1d(n, h, 0.0, "neumann").real
    M = fem.M1d(n, h, "q1mod")
    ref = np.sort(sl.eigh(K, M, eigvals_only=True))
    np.testing.assert_allclose(np.sort(fem.eig_neumann(n, h, "q1mod")), ref, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("shape,h,bc", [((9, 7), (0.11, 0.14), "abc"), ((6, 5, 7), (0.2, 0.25, 0.15), "abc"),
                                        ((8, 6), (0.12, 0.2), ("neumann", "abc"))])
def test_modified_element_solvers_and_residual(shape, h, bc):
    """O1 and O2 with the modified elements agree with dense LU of the
    element-assembled matrix; the C double-double residual equals the numpy
    one bit for bit."""
    om = 6.1
    f = random_rhs(shape, 21)
    u0 = solvers.solve_dense(f, h, om, bc, elem="q1mod")
    n0 = np.linalg.norm(u0)
    assert np.linalg.norm(solvers.solve_banded_lu(f, h, om, bc, elem="q1mod") - u0) / n0 < 1e-12
    for t in range(len(shape)):
        u3 = solvers.TensorSolver(shape, h, om, tri_axis=t, bc=bc, elem="q1mod").solve(f)
        assert np.linalg.norm(u3 - u0) / n0 < 1e-11
    # residual of a perturbed load (|r| ~ 1e-9: the two summation orders agree
    # after rounding to double)
    A = fem.assemble(shape, h, om, bc, elem="q1mod")
    f2 = (A @ u0.ravel()).reshape(shape) + 1e-9 * random_rhs(shape, 22)
    r1 = fem.residual_dd(f2, u0, h, om, bc, elem="q1mod")
    assert np.array_equal(r1, fem.residual_dd_c(f2, u0, h, om, bc, elem="q1mod"))
    np.testing.assert_allclose(r1.ravel(), f2.ravel() - A @ u0.ravel(), rtol=0, atol=1e-13)
