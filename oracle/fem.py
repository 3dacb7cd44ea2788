"""Discrete Helmholtz operator of Section 2, assembled from its definition.

Test infrastructure only (see oracle/__init__.py).

Model problem (Section 2, eqs. helmholtz, 1st-order-abc): -Lap u - w^2 u = f on
a box, with du/dn - i w u = 0 on absorbing faces and du/dn = 0 on Neumann
faces.  Weak form (eq. bf-1st-order-abc):
    a(u, v) = int grad u . grad v - w^2 u v  -  i w int_{boundary} u v ds.
Bilinear (2D) / trilinear (3D) elements on a uniform tensor mesh with n_j
nodes and spacing h_j per axis (Section 2; generalised to h_j = L_j/(n_j-1)).

Arrays are C-ordered with the last axis fastest.  The 1D matrices are those of
eqs. matrixK / matrixM; the Kronecker forms are eqs. A2D / A3D; the periodic
auxiliary operator uses the circulant matrices of eqs. matrixKper / matrixMper
(eq. B2D / B3D).

Elements (`elem`): "q1", the paper's bilinear / trilinear elements with every
element integral exact (2-point Gauss rule per axis); "q1mod", the modified
elements with reduced dispersion that the paper names as applicable (Section
1, the modified integration rules it cites): every element integral
(stiffness, mass, boundary mass) by the tensor-product 2-point rule at
+-sqrt(2/3) of the reference half-width.  Both keep the Kronecker form with
one 1D mass matrix per axis, h [(den-2)/den on the diagonal, 1/den off it,
half the diagonal at the ends]: den = 6 for "q1", 12 for "q1mod" (the mean of
the consistent and the lumped mass).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import dd as ddm

# 2-point Gauss-Legendre rule on [0, 1]: exact for the cubic integrands that
# appear in products of two linear (per-axis) shape functions.
_GAUSS_X = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
_GAUSS_W = np.array([0.5, 0.5])
# the modified rule: points at +-sqrt(2/3) of the half-width, equal weights
_MOD_X = np.array([0.5 - 0.5 * np.sqrt(2.0 / 3.0), 0.5 + 0.5 * np.sqrt(2.0 / 3.0)])

ELEMENTS = ("q1", "q1mod")


def _quad_x(elem):
    if elem not in ELEMENTS:
        raise ValueError(f"element must be one of {ELEMENTS}")
    return _GAUSS_X if elem == "q1" else _MOD_X


def mass_den(elem):
    """den of the 1D mass matrix h [(den-2)/den, 1/den] of the element."""
    if elem not in ELEMENTS:
        raise ValueError(f"element must be one of {ELEMENTS}")
    return 6.0 if elem == "q1" else 12.0


def _shape_1d(s):
    """Linear shape functions on the reference segment [0, 1] and derivatives."""
    return np.array([1.0 - s, s]), np.array([-1.0, 1.0])


def element_matrix(h, omega, elem="q1"):
    """Element matrix of int grad phi_a . grad phi_b - w^2 phi_a phi_b over one
    box element with edge lengths h (d = len(h)), by the element's tensor
    2-point quadrature of the multilinear shape functions (Section 2, weak
    form).  Local node a is the multi-index (a_1, ..., a_d) in {0,1}^d, in C
    order."""
    d = len(h)
    xq = _quad_x(elem)
    locs = list(itertools.product((0, 1), repeat=d))
    E = np.zeros((2 ** d, 2 ** d), dtype=np.complex128)
    for q in itertools.product(range(2), repeat=d):
        s = [xq[qi] for qi in q]
        wq = np.prod([_GAUSS_W[qi] * hj for qi, hj in zip(q, h)])
        vals, grads = [], []
        for a in locs:
            phis = [_shape_1d(s[j])[0][a[j]] for j in range(d)]
            dphis = [_shape_1d(s[j])[1][a[j]] / h[j] for j in range(d)]
            vals.append(np.prod(phis))
            g = []
            for j in range(d):
                g.append(dphis[j] * np.prod([phis[k] for k in range(d) if k != j]))
            grads.append(np.array(g))
        for ia in range(2 ** d):
            for ib in range(2 ** d):
                E[ia, ib] += wq * (grads[ia] @ grads[ib] - omega ** 2 * vals[ia] * vals[ib])
    return E, locs


def face_mass_matrix(h_face, elem="q1"):
    """int_face phi_a phi_b over a (d-1)-dimensional element face with edge
    lengths h_face, by the element's quadrature (boundary term of the weak
    form)."""
    m = len(h_face)
    xq = _quad_x(elem)
    locs = list(itertools.product((0, 1), repeat=m))
    F = np.zeros((2 ** m, 2 ** m))
    if m == 0:
        return np.ones((1, 1)), [()]
    for q in itertools.product(range(2), repeat=m):
        s = [xq[qi] for qi in q]
        wq = np.prod([_GAUSS_W[qi] * hj for qi, hj in zip(q, h_face)])
        vals = [np.prod([_shape_1d(s[j])[0][a[j]] for j in range(m)]) for a in locs]
        F += wq * np.outer(vals, vals)
    return F, locs


def assemble(shape, h, omega, bc="abc", elem="q1"):
    """Global sparse matrix A (CSR, complex128) assembled element by element.

    shape: node counts per axis; h: spacings; bc: "abc" on every face, or
    "neumann" on every face, or a tuple with one of those per axis.  This is
    the definition of A (Section 2); it deliberately does not use the
    Kronecker formula of eqs. A2D/A3D so that it can pin it.
    """
    shape = tuple(int(n) for n in shape)
    d = len(shape)
    if isinstance(bc, str):
        bc = (bc,) * d
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    rows, cols, vals = [], [], []
    E, locs = element_matrix(h, omega, elem)
    # element origin nodes
    origin = idx[tuple(slice(0, n - 1) for n in shape)].ravel()
    strides = [int(np.prod(shape[j + 1:])) for j in range(d)]
    loc_off = [sum(a[j] * strides[j] for j in range(d)) for a in locs]
    for ia in range(len(locs)):
        for ib in range(len(locs)):
            rows.append(origin + loc_off[ia])
            cols.append(origin + loc_off[ib])
            vals.append(np.full(origin.size, E[ia, ib]))
    # boundary faces: for each axis j with an absorbing condition, the two
    # faces x_j = 0 and x_j = L_j, each tiled by (d-1)-dimensional element faces.
    for j in range(d):
        if bc[j] != "abc":
            continue
        other = [k for k in range(d) if k != j]
        F, flocs = face_mass_matrix([h[k] for k in other], elem)
        for side in (0, shape[j] - 1):
            sl = [slice(0, n - 1) for n in shape]
            sl[j] = side
            o = idx[tuple(sl)].ravel()
            off = [sum(a[t] * strides[other[t]] for t in range(len(other))) for a in flocs]
            for ia in range(len(flocs)):
                for ib in range(len(flocs)):
                    rows.append(o + off[ia])
                    cols.append(o + off[ib])
                    vals.append(np.full(o.size, -1j * omega * F[ia, ib]))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A


# ---------------------------------------------------------------------------
# 1D matrices (eqs. matrixK, matrixM, matrixKper, matrixMper)
# ---------------------------------------------------------------------------

def K1d(n, h, omega, bc="abc"):
    """Dense 1D stiffness matrix (eq. matrixK): (1/h) tridiag(-1, 2, -1) with
    corner entries k11 = knn = 1 - i w h (absorbing) or 1 (Neumann)."""
    K = (2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)).astype(np.complex128) / h
    # corner (1 - i w h)/h written as 1/h - i w (same value, fewer roundings)
    K[0, 0] = K[-1, -1] = (1.0 / h - 1j * omega) if bc == "abc" else 1.0 / h
    return K


def M1d(n, h, elem="q1"):
    """Dense 1D mass matrix (eq. matrixM): (h/6) tridiag(1, 4, 1), corners 2;
    for the modified element (h/12) tridiag(1, 10, 1), corners 5."""
    den = mass_den(elem)
    M = (den - 2.0) * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    M[0, 0] = M[-1, -1] = (den - 2.0) / 2.0
    return M * (h / den)


def K1d_periodic(n, h, gamma=1.0):
    """Circulant stiffness matrix of eq. matrixKper.  With gamma != 1 the
    wrap-around entries become gamma * (-1/h) (last row, first column) and
    (-1/h) / gamma (first row, last column): a gamma-circulant, the damped
    periodic auxiliary (gamma = 1 is the paper's matrix)."""
    K = (2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)).astype(np.complex128)
    K[-1, 0] = -1.0 * gamma
    K[0, -1] = -1.0 / gamma
    return K / h


def M1d_periodic(n, h, gamma=1.0, elem="q1"):
    """Circulant mass matrix of eq. matrixMper (gamma-circulant as above)."""
    den = mass_den(elem)
    M = ((den - 2.0) * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)).astype(np.complex128)
    M[-1, 0] = 1.0 * gamma
    M[0, -1] = 1.0 / gamma
    return M * (h / den)


def kron_operator(shape, h, omega, periodic_axis=None, bc="abc", gamma=None, elem="q1"):
    """Sparse Kronecker-form operator: eq. A2D / A3D, or with `periodic_axis`
    replaced by the circulant matrices, eq. B2D / B3D.  `gamma` (a scalar,
    or a dict axis -> gamma; periodic_axis may then be a tuple) selects the
    gamma-circulant auxiliary on that axis.

    General d: sum_j (x)_k [K_k if k == j else M_k]  -  w^2 (x)_k M_k.
    """
    d = len(shape)
    if isinstance(bc, str):
        bc = (bc,) * d
    Ks, Ms = [], []
    paxes = periodic_axis if isinstance(periodic_axis, (tuple, list)) else (periodic_axis,)
    for j in range(d):
        if j in paxes:
            g = 1.0 if gamma is None else (gamma[j] if isinstance(gamma, dict) else gamma)
            Ks.append(sp.csr_matrix(K1d_periodic(shape[j], h[j], g)))
            Ms.append(sp.csr_matrix(M1d_periodic(shape[j], h[j], g, elem)))
        else:
            Ks.append(sp.csr_matrix(K1d(shape[j], h[j], omega, bc[j])))
            Ms.append(sp.csr_matrix(M1d(shape[j], h[j], elem)))

    def kron_all(mats):
        out = mats[0]
        for m in mats[1:]:
            out = sp.kron(out, m, format="csr")
        return out

    A = -omega ** 2 * kron_all(Ms)
    for j in range(d):
        A = A + kron_all([Ks[k] if k == j else Ms[k] for k in range(d)])
    return A.tocsr()


# ---------------------------------------------------------------------------
# Closed-form 1D eigenvalues of the linear-FEM pencils
# ---------------------------------------------------------------------------

def _ratio(theta, h, elem="q1"):
    if elem == "q1":
        return 6.0 / h ** 2 * (1.0 - np.cos(theta)) / (2.0 + np.cos(theta))
    den = mass_den(elem)
    return (2.0 - 2.0 * np.cos(theta)) / h / (h * ((den - 2.0) + 2.0 * np.cos(theta)) / den)


def eig_periodic(n, h):
    """Eigenvalues of the circulant pencil (K^B, M^B), eq. eigvaluesPer, in
    DFT order l = 1..n (theta = 2 pi (l-1) / n)."""
    th = 2.0 * np.pi * np.arange(n) / n
    num = 2.0 / h - (1.0 / h) * (np.exp(-1j * th) + np.exp(-1j * th * (n - 1)))
    den = 4.0 * h / 6 + (h / 6) * (np.exp(-1j * th) + np.exp(-1j * th * (n - 1)))
    return (num / den).real


def eig_periodic_closed(n, h):
    """Same eigenvalues from the closed form 6/h^2 (1 - cos t)/(2 + cos t)."""
    return _ratio(2.0 * np.pi * np.arange(n) / n, h)


def eig_neumann(n, h, elem="q1"):
    """Eigenvalues of the Neumann pencil (k11 = 1): theta_k = k pi/(n-1), k=0..n-1."""
    return _ratio(np.pi * np.arange(n) / (n - 1), h, elem)


def eig_dirichlet(n, h):
    """Eigenvalues of the pencil with both end nodes eliminated (Dirichlet):
    the (n-2)x(n-2) interior block, theta_k = k pi h / L = k pi/(n-1), k=1..n-2."""
    return _ratio(np.pi * np.arange(1, n - 1) / (n - 1), h)


# ---------------------------------------------------------------------------
# Separable operator application (for residuals), eqs. A2D / A3D
# ---------------------------------------------------------------------------

def _bc_tuple(bc, d):
    return (bc,) * d if isinstance(bc, str) else tuple(bc)


def _tri_coeffs(n, h, omega, kind, bc="abc", elem="q1"):
    """(sub, diag, super) coefficient vectors of a 1D matrix from eqs.
    matrixK / matrixM; sub[j] multiplies x[j-1], super[j] multiplies x[j+1].
    K's corners are 1/h - i w on an absorbing axis, 1/h on a Neumann one."""
    if kind == "K":
        diag = np.full(n, 2.0 / h, dtype=np.complex128)
        diag[0] = diag[-1] = (1.0 / h - 1j * omega) if bc == "abc" else 1.0 / h
        off = -1.0 / h
    else:
        den = mass_den(elem)
        diag = np.full(n, (den - 2.0) * h / den, dtype=np.complex128)
        diag[0] = diag[-1] = ((den - 2.0) / 2.0) * h / den
        off = h / den
    sub = np.full(n, off, dtype=np.complex128)
    sup = np.full(n, off, dtype=np.complex128)
    sub[0] = 0.0
    sup[-1] = 0.0
    return sub, diag, sup


def _bshape(n, axis, d):
    s = [1] * d
    s[axis] = n
    return s


def apply_1d(u, axis, n, h, omega, kind, bc="abc", elem="q1"):
    """y = T u along `axis`, T the 1D matrix K or M, complex128."""
    d = u.ndim
    sub, diag, sup = (c.reshape(_bshape(n, axis, d)) for c in _tri_coeffs(n, h, omega, kind, bc, elem))
    y = diag * u
    lo = [slice(None)] * d
    hi = [slice(None)] * d
    lo[axis] = slice(0, n - 1)
    hi[axis] = slice(1, n)
    y[tuple(hi)] += sub[tuple(hi)] * u[tuple(lo)]
    y[tuple(lo)] += sup[tuple(lo)] * u[tuple(hi)]
    return y


def apply_A(u, h, omega, bc="abc", elem="q1"):
    """A u for the Kronecker form of eqs. A2D / A3D, complex128 (bc: per
    axis "abc" or "neumann", or one of them for every axis)."""
    shape = u.shape
    d = len(shape)
    bc = _bc_tuple(bc, d)
    total = None
    for j in range(d + 1):
        t = u
        for k in range(d):
            kind = "K" if k == j else "M"
            t = apply_1d(t, k, shape[k], h[k], omega, kind, bc[k], elem)
        if j == d:
            t = -omega ** 2 * t
        total = t if total is None else total + t
    return total


def _apply_1d_dd(x: ddm.CDD, axis, n, h, omega, kind, bc="abc", elem="q1"):
    d = x.re[0].ndim
    sub, diag, sup = (c.reshape(_bshape(n, axis, d)) for c in _tri_coeffs(n, h, omega, kind, bc, elem))

    def shift(a, direction):
        # direction +1: out[j] = a[j-1]; -1: out[j] = a[j+1]; zero fill
        out = np.zeros_like(a)
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        if direction > 0:
            out[tuple(hi)] = a[tuple(lo)]
        else:
            out[tuple(lo)] = a[tuple(hi)]
        return out

    y = x.mul_c(diag)
    y = y + x.map(lambda a: shift(a, +1)).mul_c(sub)
    y = y + x.map(lambda a: shift(a, -1)).mul_c(sup)
    return y


def residual_dd(f, u, h, omega, bc="abc", elem="q1"):
    """r = f - A u with A of eqs. A2D / A3D, every operation in double-double,
    rounded to complex128 at the end."""
    shape = u.shape
    d = len(shape)
    bc = _bc_tuple(bc, d)
    U = ddm.CDD.from_complex(u)
    acc = ddm.CDD.from_complex(f)
    for j in range(d + 1):
        t = U
        for k in range(d):
            t = _apply_1d_dd(t, k, shape[k], h[k], omega, "K" if k == j else "M", bc[k], elem)
        if j == d:
            t = t.mul_c(-omega ** 2)
        acc = acc - t
    return acc.to_complex()


# ---------------------------------------------------------------------------
# Plane-wave manufactured solution with inhomogeneous absorbing data
# ---------------------------------------------------------------------------

def plane_wave_load(shape, h, omega, direction, elem="q1"):
    """Load vector and nodal exact solution for u* = exp(i w d.x), |d| = 1.

    u* solves -Lap u - w^2 u = 0 exactly.  On the face with outward normal n the
    absorbing data is g = du*/dn - i w u* = i w (d.n - 1) u*, so the weak form
    (eq. bf-1st-order-abc with data) gives the load f_i = sum over faces of
    int_face g phi_i ds, evaluated as face mass matrix times nodal g."""
    d = len(shape)
    direction = np.asarray(direction, dtype=float)
    direction = direction / np.linalg.norm(direction)
    coords = np.meshgrid(*[np.arange(n) * hj for n, hj in zip(shape, h)], indexing="ij")
    phase = sum(direction[j] * coords[j] for j in range(d))
    u_exact = np.exp(1j * omega * phase)
    f = np.zeros(shape, dtype=np.complex128)
    for j in range(d):
        for side, normal in ((0, -1.0), (shape[j] - 1, 1.0)):
            sl = [slice(None)] * d
            sl[j] = side
            sl = tuple(sl)
            g = 1j * omega * (normal * direction[j] - 1.0) * u_exact[sl]
            # apply the (d-1)-dimensional face mass: tensor product of 1D M's
            t = g
            ax = 0
            for k in range(d):
                if k == j:
                    continue
                t = apply_1d(t, ax, shape[k], h[k], omega, "M", elem=elem)
                ax += 1
            f[sl] += t
    return f, u_exact


def residual_dd_c(f, u, h, omega, bc="abc", elem="q1"):
    """Same double-double residual as `residual_dd`, computed by the oracle's
    C helper (oracle/c/dd_resid.c) for large grids."""
    from . import cbuild

    f = np.ascontiguousarray(f, dtype=np.complex128)
    u = np.ascontiguousarray(u, dtype=np.complex128)
    n = np.array(u.shape, dtype=np.int64)
    hh = np.array(h, dtype=np.float64)
    r = np.empty_like(u)
    if isinstance(bc, str) and bc == "abc" and elem == "q1":
        cbuild.lib().helm_oracle_dd_residual(u.ndim, n.ctypes.data, hh.ctypes.data, float(omega), f.ctypes.data,
                                             u.ctypes.data, r.ctypes.data)
        return r
    wc = np.array([float(omega) if b == "abc" else 0.0 for b in _bc_tuple(bc, u.ndim)], dtype=np.float64)
    cbuild.lib().helm_oracle_dd_residual_el(u.ndim, n.ctypes.data, hh.ctypes.data, float(omega), wc.ctypes.data,
                                            float(mass_den(elem)), f.ctypes.data, u.ctypes.data, r.ctypes.data)
    return r
