"""Seeded synthetic workloads for the Helmholtz fast direct solver.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.
It holds problem definitions (grid sizes, spacings, wave number) and seeded
right-hand-side generators only -- none of the solver's arithmetic.

Problems follow the paper's setting (Section 2): a rectangular domain with a
uniform tensor mesh of n_j nodes and spacing h_j = L_j / (n_j - 1) per axis,
first-order absorbing boundary conditions on every face, and a nodal load
vector f.  Arrays are C-ordered with the LAST axis fastest, shape (nx, ny) in
2D and (nx, ny, nz) in 3D, complex valued.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Problem:
    """One Helmholtz problem: node counts, spacings, wave number, seed."""

    name: str
    shape: tuple            # node counts, slowest axis first
    h: tuple                # spacing per axis
    omega: float            # wave number
    seed: int
    rhs: str = "gaussian"   # "gaussian" | "gaussian_bump" | "paper"
    bump_sigma: float = 0.1
    note: str = ""

    @property
    def dim(self) -> int:
        return len(self.shape)

    @property
    def N(self) -> int:
        return int(np.prod(self.shape))

    @property
    def lengths(self) -> tuple:
        return tuple((n - 1) * h for n, h in zip(self.shape, self.h))


def ppw_omega(h: float, ppw: float) -> float:
    """Wave number giving `ppw` nodes per wavelength at spacing h: 2*pi/(ppw*h)."""
    return 2.0 * math.pi / (ppw * h)


def box(shape, lengths, omega, seed, name="box", rhs="gaussian", **kw) -> Problem:
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    return Problem(name=name, shape=tuple(int(n) for n in shape), h=h,
                   omega=float(omega), seed=int(seed), rhs=rhs, **kw)


# The three single-GPU configurations of the benchmark suite.
def config_2d_small() -> Problem:
    """129 x 129 nodes on the unit square, omega = 16*pi (16 nodes/wavelength)."""
    return box((129, 129), (1.0, 1.0), 16.0 * math.pi, seed=1, name="2d_129x129")


def config_2d_large() -> Problem:
    """8192 x 4096 nodes on [0,2]x[0,1], 10 nodes/wavelength at h = max(hx, hy),
    f = complex Gaussian times a Gaussian bump centred at (1, 0.5), sigma 0.1."""
    hx, hy = 2.0 / 8191, 1.0 / 4095
    return box((8192, 4096), (2.0, 1.0), ppw_omega(max(hx, hy), 10.0), seed=2,
               name="2d_8192x4096", rhs="gaussian_bump", bump_sigma=0.1)


def config_3d() -> Problem:
    """512^3 nodes on the unit cube, 10 nodes per wavelength."""
    return box((512, 512, 512), (1.0, 1.0, 1.0), ppw_omega(1.0 / 511, 10.0), seed=3,
               name="3d_512cube")


def _max_prime_factor(n: int) -> int:
    m, p, big = n, 2, 1
    while p * p <= m:
        while m % p == 0:
            big, m = p, m // p
        p += 1
    return max(big, m) if m > 1 else big


def batch_2d(count: int = 512, seed: int = 1000) -> list:
    """Batched 2D workload: `count` independent problems.

    nx and ny (the x1 / transform length) uniform on {63..1023}; anisotropic
    spacings h_j = s_j / (n_j - 1) with s_j uniform on [0.5, 2]; omega for a
    uniform 6..20 nodes per wavelength at max(h).  Two problems in eight are
    moved next to a discrete resonance, omega^2 set to the nearest of
      (i)  (i % 8 == 7) a sum of closed-box (Neumann) eigenvalues of the
           linear-element pencils of the two axes,
           6/h^2 (1 - cos(k pi/(n-1))) / (2 + cos(k pi/(n-1))), and
      (ii) (i % 8 == 3) a periodic eigenvalue of the x1 axis,
           6/h^2 (1 - cos(2 pi l/n)) / (2 + cos(2 pi l/n)), plus a Neumann
           eigenvalue of the other axis -- the mode sums at which the periodic
           auxiliary's line matrices come close to singular.
    The absorbing boundary keeps every problem solvable.  Right-hand sides are
    seeded complex Gaussians (seed + 1 + index)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def closed(theta, h):
        return 6.0 / h ** 2 * (1.0 - np.cos(theta)) / (2.0 + np.cos(theta))

    out = []
    for i in range(count):
        nx = int(rng.integers(63, 1024))
        ny = int(rng.integers(63, 1024))
        hx = float(rng.uniform(0.5, 2.0)) / (nx - 1)
        hy = float(rng.uniform(0.5, 2.0)) / (ny - 1)
        ppw = float(rng.uniform(6.0, 20.0))
        omega = ppw_omega(max(hx, hy), ppw)
        note = ""
        if i % 8 in (3, 7):
            ex = closed(np.pi * np.arange(nx) / (nx - 1), hx)
            if i % 8 == 7:
                ey = closed(np.pi * np.arange(ny) / (ny - 1), hy)
                note = "near resonance"
            else:
                ey = closed(2.0 * np.pi * np.arange(ny) / ny, hy)
                note = "near periodic-mode resonance"
            sums = (ex[:, None] + ey[None, :]).ravel()
            omega = float(np.sqrt(sums[np.argmin(np.abs(sums - omega ** 2))]))
        out.append(Problem(name=f"batch2d_{i}", shape=(nx, ny), h=(hx, hy), omega=omega, seed=seed + 1 + i,
                           note=note))
    return out


def serve_3d(count: int = 32, operators: int = 12, rate_per_s: float = 4.0, seed: int = 2000) -> list:
    """Serving workload: a Poisson stream of `count` 3D requests over a pool of
    `operators` box problems (domain-decomposition sweeps reuse one operator
    for many right-hand sides).

    Per operator: nx, ny, nz uniform on {31..255}; side lengths uniform on
    [0.5, 2] per axis; omega for a uniform 8..12 nodes per wavelength at
    max(h).  Per request: an operator drawn uniformly from the
    pool, nrhs uniform on {1..64}, arrival after an exponential gap of mean
    1 / rate_per_s (rate_per_s <= 0: every request arrives at time 0, the
    saturated stream).  Returns [(Problem, nrhs, arrival_s)]; the right-hand
    sides are seeded complex Gaussians (Problem.seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ops = []
    for k in range(operators):
        nx = int(rng.integers(31, 256))
        ny = int(rng.integers(31, 256))
        nz = int(rng.integers(31, 256))
        h = tuple(float(rng.uniform(0.5, 2.0)) / (n - 1) for n in (nx, ny, nz))
        omega = ppw_omega(max(h), float(rng.uniform(8.0, 12.0)))
        ops.append(((nx, ny, nz), h, omega))
    out, t = [], 0.0
    for i in range(count):
        shape, h, omega = ops[int(rng.integers(0, operators))]
        nrhs = int(rng.integers(1, 65))
        gap = float(rng.exponential(1.0))  # drawn in both modes: the same requests
        t += gap / rate_per_s if rate_per_s > 0 else 0.0
        out.append((Problem(name=f"serve3d_{i}", shape=shape, h=h, omega=omega, seed=seed + 1 + i), nrhs, t))
    return out


def scaled(p: Problem, shape, seed=None, name=None) -> Problem:
    """Same spacing and wave number as `p` on a smaller node grid (bounded samples)."""
    return Problem(name=name or f"{p.name}_sample{'x'.join(map(str, shape))}",
                   shape=tuple(shape), h=p.h, omega=p.omega,
                   seed=p.seed if seed is None else seed, rhs=p.rhs,
                   bump_sigma=p.bump_sigma)


def rhs(p: Problem, dtype=np.complex128) -> np.ndarray:
    """Seeded nodal load vector f for problem p (numpy PCG64).

    gaussian: real and imaginary parts i.i.d. N(0, 1).
    gaussian_bump: the same times exp(-|x - c|^2 / (2 sigma^2)), c = domain centre.
    paper: 0.01 on the first n_last entries, 1 elsewhere (the paper's timing RHS,
           Section 6), in this module's C order.
    """
    rng = np.random.Generator(np.random.PCG64(p.seed))
    if p.rhs == "paper":
        f = np.ones(p.shape, dtype=np.complex128)
        f.reshape(-1)[: p.shape[-1]] = 0.01
        return f.astype(dtype)
    re = rng.standard_normal(p.shape)
    im = rng.standard_normal(p.shape)
    f = re + 1j * im
    if p.rhs == "gaussian_bump":
        coords = np.meshgrid(*[np.arange(n) * h for n, h in zip(p.shape, p.h)], indexing="ij")
        centre = [L / 2 for L in p.lengths]
        r2 = sum((c - c0) ** 2 for c, c0 in zip(coords, centre))
        f *= np.exp(-r2 / (2.0 * p.bump_sigma ** 2))
    return np.ascontiguousarray(f.astype(dtype))


def random_rhs(shape, seed, dtype=np.complex128) -> np.ndarray:
    """Complex Gaussian array of the given shape from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype))
