"""Plain, slow FP64 solvers for A u = f (test infrastructure only).

The fast solver of the paper is a *direct* method: it returns u = A^-1 f up to
rounding (Section 1; the three steps of Section 3.1 give u exactly once B is
invertible).  The oracle therefore computes that plain definition, never the
FFT algorithm:

* O1 ``solve_banded_lu``: the element-assembled A (oracle.fem.assemble) in
  band storage, LU with partial pivoting (LAPACK gbsv through scipy).
* O2 ``solve_tensor``: the tensor-product eigen-solve the paper builds on
  (Lynch-Rice-Thomas; the representation of eq. A2Dinv / A3Dinv applied on
  every axis but one): dense generalized eigen-decomposition of the absorbing
  1D pencil (K_j, M_j) with V^T M V = I (eq. EVPcondA), then one tridiagonal
  LU with partial pivoting per line along the remaining axis.
* ``refine``: iterative refinement with the double-double residual of
  oracle.fem.residual_dd.

Also the plain definitions of the intermediate quantities of Section 3.1:
v = B^-1 f (Step 1, eq. probB), w = A^-1 (B - A) v (Step 2, eq. probStep2), with
B the operator whose absorbing x1 matrices are replaced by the circulant ones
(eqs. B2D / B3D).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl
import scipy.sparse.linalg as spl
from scipy.linalg import lapack

from . import fem


# ---------------------------------------------------------------------------
# O1: assembled banded LU
# ---------------------------------------------------------------------------

def solve_banded_lu(f, h, omega, bc="abc", elem="q1"):
    """u = A^-1 f with A assembled element by element (fem.assemble) and
    factorised by banded LU with partial pivoting.  Axes are reordered so the
    longest axis is slowest, which minimises the bandwidth."""
    f = np.asarray(f, dtype=np.complex128)
    d = f.ndim
    order = sorted(range(d), key=lambda j: -f.shape[j])
    fp = np.ascontiguousarray(np.transpose(f, order))
    hp = tuple(h[j] for j in order)
    bcp = bc if isinstance(bc, str) else tuple(bc[j] for j in order)
    A = fem.assemble(fp.shape, hp, omega, bcp, elem).tocoo()
    bw = int(np.max(np.abs(A.row - A.col)))
    N = fp.size
    ab = np.zeros((2 * bw + 1, N), dtype=np.complex128)
    ab[bw + A.row - A.col, A.col] = A.data
    u = sl.solve_banded((bw, bw), ab, fp.ravel(), check_finite=False)
    u = u.reshape(fp.shape)
    inv = np.argsort(order)
    return np.ascontiguousarray(np.transpose(u, inv))


def solve_dense(f, h, omega, bc="abc", elem="q1"):
    """Brute force for tiny grids: dense LU of the assembled A."""
    f = np.asarray(f, dtype=np.complex128)
    A = fem.assemble(f.shape, h, omega, bc, elem).toarray()
    return np.linalg.solve(A, f.ravel()).reshape(f.shape)


# ---------------------------------------------------------------------------
# O2: tensor-product eigen-solve
# ---------------------------------------------------------------------------

def abc_pencil_eig(n, h, omega, bc="abc", elem="q1"):
    """Eigenpairs of K V = M V Lam (eq. EVP1a) normalised so V^T M V = I
    (eq. EVPcondA; transpose, not conjugate transpose).

    Computed densely: M = L L^T (Cholesky, M is SPD), C = L^-1 K L^-T is
    complex symmetric, C Y = Y Lam by LAPACK geev, V = L^-T Y, then each column
    is scaled by 1/sqrt(v^T M v) (eqs. sA, sAnorm)."""
    K = fem.K1d(n, h, omega, bc)
    M = fem.M1d(n, h, elem)
    L = np.linalg.cholesky(M)
    Li = sl.solve_triangular(L, np.eye(n), lower=True)
    C = Li @ K @ Li.T
    lam, Y = np.linalg.eig(C)
    V = Li.T @ Y
    s = np.sqrt(np.einsum("ij,ik,kj->j", V, M, V))
    V = V / s[None, :]
    return lam, V


def _tridiag_solve_lines(sub, diag, sup, rhs):
    """Solve many tridiagonal systems with LAPACK gtsv (LU, partial pivoting).

    sub/sup: (nlines, n-1); diag, rhs: (nlines, n)."""
    out = np.empty_like(rhs)
    for i in range(rhs.shape[0]):
        _, _, _, x, info = lapack.zgtsv(sub[i], diag[i], sup[i], rhs[i])
        if info != 0:
            raise np.linalg.LinAlgError(f"gtsv info={info} on line {i}")
        out[i] = x
    return out


class TensorSolver:
    """O2: A^-1 = (V_a (x) ... (x) I) H^-1 (V_a^T (x) ... (x) I) with one axis
    (`tri_axis`) kept as tridiagonal blocks (eqs. A2Dinv, HA2D, A3Dinv, HA3D)."""

    def __init__(self, shape, h, omega, tri_axis=None, bc="abc", elem="q1"):
        self.shape = tuple(shape)
        self.h = tuple(h)
        self.omega = float(omega)
        d = len(shape)
        self.bc = fem._bc_tuple(bc, d)
        self.elem = elem
        self.tri_axis = int(np.argmax(shape)) if tri_axis is None else tri_axis
        self.eig_axes = [j for j in range(d) if j != self.tri_axis]
        self.eigs = {j: abc_pencil_eig(shape[j], h[j], omega, self.bc[j], elem) for j in self.eig_axes}

    def _transform(self, x, transpose):
        for j in self.eig_axes:
            V = self.eigs[j][1]
            T = V.T if transpose else V
            x = np.moveaxis(np.tensordot(T, x, axes=([1], [j])), 0, j)
        return x

    def solve(self, f):
        f = np.asarray(f, dtype=np.complex128)
        d = f.ndim
        t = self.tri_axis
        g = self._transform(f, transpose=True)
        # sum of transverse eigenvalues for every line
        lam = np.zeros([f.shape[j] if j != t else 1 for j in range(d)], dtype=np.complex128)
        for j in self.eig_axes:
            shp = [1] * d
            shp[j] = f.shape[j]
            lam = lam + self.eigs[j][0].reshape(shp)
        n = f.shape[t]
        ht = self.h[t]
        g_lines = np.moveaxis(g, t, -1).reshape(-1, n)
        lam_lines = np.moveaxis(lam, t, -1).reshape(-1)
        s = lam_lines - self.omega ** 2
        # line matrix: K_t + (lam - w^2) M_t   (eq. HA2D block)
        subK, diagK, _ = fem._tri_coeffs(n, ht, self.omega, "K", self.bc[t])
        subM, diagM, _ = fem._tri_coeffs(n, ht, self.omega, "M", elem=self.elem)
        diag = diagK[None, :] + s[:, None] * diagM[None, :]
        off = subK[1:][None, :] + s[:, None] * subM[1:][None, :]
        x = _tridiag_solve_lines(off.copy(), diag, off.copy(), g_lines.copy())
        shp = list(np.moveaxis(g, t, -1).shape)
        x = np.moveaxis(x.reshape(shp), -1, t)
        return np.ascontiguousarray(self._transform(x, transpose=False))


def refine(f, u, solve, h, omega, iters=2, bc="abc", elem="q1"):
    """Iterative refinement u <- u + solve(f - A u) with the residual formed in
    double-double (fem.residual_dd).  Returns (u, [relative residuals])."""
    hist = []
    fn = np.linalg.norm(f)
    resid = fem.residual_dd_c if f.size > 4096 else fem.residual_dd
    for _ in range(iters):
        r = resid(f, u, h, omega, bc, elem)
        hist.append(float(np.linalg.norm(r) / fn))
        u = u + solve(r)
    r = resid(f, u, h, omega, bc, elem)
    hist.append(float(np.linalg.norm(r) / fn))
    return u, hist


def oracle_solve(f, h, omega, method="auto", iters=2, tri_axis=None, bc="abc", elem="q1"):
    """u = A^-1 f: O1 (banded LU) for small problems, O2 (tensor eigen-solve)
    otherwise, followed by double-double iterative refinement.  bc: "abc"
    (absorbing faces everywhere), or per axis "abc" / "neumann" (Section 2's
    Gamma_A / Gamma_N: both faces of an axis of the same kind).  elem: "q1"
    (the paper's elements) or "q1mod" (the modified elements, see
    oracle.fem)."""
    f = np.asarray(f, dtype=np.complex128)
    if method == "auto":
        srt = sorted(f.shape)
        bw = int(np.prod(srt[:-1])) if f.ndim > 1 else 1
        method = "banded" if bw * f.size <= 3e8 else "tensor"
    if method == "banded":
        solve = lambda r: solve_banded_lu(r, h, omega, bc, elem)
    elif method == "dense":
        solve = lambda r: solve_dense(r, h, omega, bc, elem)
    else:
        ts = TensorSolver(f.shape, h, omega, tri_axis, bc, elem)
        solve = ts.solve
    u = solve(f)
    u, hist = refine(f, u, solve, h, omega, iters=iters, bc=bc, elem=elem)
    return u, hist


# ---------------------------------------------------------------------------
# Plain definitions of the three-step solve's intermediates (Section 3.1)
# ---------------------------------------------------------------------------

def step_definitions(f, h, omega, axis, gamma=None):
    """Return (v, w, u): v = B^-1 f (Step 1), w = A^-1 (B - A) v (Step 2),
    u = A^-1 f, with B periodic along `axis` (eqs. probB, probStep2, B2D/B3D),
    or gamma-circulant when `gamma` is given.  Uses sparse LU on the Kronecker
    forms; meant for small grids."""
    f = np.asarray(f, dtype=np.complex128)
    A = fem.kron_operator(f.shape, h, omega).tocsc()
    B = fem.kron_operator(f.shape, h, omega, periodic_axis=axis, gamma=gamma).tocsc()
    v = spl.spsolve(B, f.ravel())
    w = spl.spsolve(A, (B - A) @ v)
    u = spl.spsolve(A, f.ravel())
    return v.reshape(f.shape), w.reshape(f.shape), u.reshape(f.shape)
