"""The seeded workload generators: deterministic and inside the stated
ranges (every length in range, including those with large prime factors,
which the transforms take by Bluestein's method)."""
import numpy as np

import workloads


def _max_prime(n):
    m, p, big = n, 2, 1
    while p * p <= m:
        while m % p == 0:
            big, m = p, m // p
        p += 1
    return max(big, m) if m > 1 else big


def test_batch_2d_ranges_and_determinism():
    a = workloads.batch_2d(64)
    assert a == workloads.batch_2d(64)
    for i, q in enumerate(a):
        nx, ny = q.shape
        assert 63 <= nx <= 1023 and 63 <= ny <= 1023
        assert all(0.5 - 1e-12 <= n_h <= 2.0 + 1e-12 for n_h in (q.h[0] * (nx - 1), q.h[1] * (ny - 1)))
        ppw = 2 * np.pi / (q.omega * max(q.h))
        if q.note:
            assert i % 8 in (3, 7)
        else:
            assert 6.0 - 1e-9 <= ppw <= 20.0 + 1e-9
    assert sum(1 for q in a if q.note) == 16
    # large prime factors are drawn too
    assert any(_max_prime(q.shape[1]) > 64 for q in a)


def test_batch_2d_near_resonance_is_an_eigenvalue_sum():
    """omega^2 of the resonant problems is a Neumann + Neumann (i % 8 == 7)
    or Neumann + periodic (i % 8 == 3) sum of the oracle's closed-form 1D
    eigenvalues (pinned against LAPACK in test_oracle_pins)."""
    from oracle import fem

    for i, q in enumerate(workloads.batch_2d(16)):
        if not q.note:
            continue
        nx, ny = q.shape
        ey = fem.eig_neumann(ny, q.h[1]) if i % 8 == 7 else fem.eig_periodic_closed(ny, q.h[1])
        sums = fem.eig_neumann(nx, q.h[0])[:, None] + ey[None, :]
        assert np.min(np.abs(sums - q.omega ** 2)) <= 1e-9 * q.omega ** 2


def test_serve_3d_stream():
    r = workloads.serve_3d(48, operators=12, rate_per_s=4.0)
    sat = workloads.serve_3d(48, operators=12, rate_per_s=0.0)
    assert [(q, n) for q, n, _ in r] == [(q, n) for q, n, _ in sat]
    times = [t for _, _, t in r]
    assert all(b > a for a, b in zip(times, times[1:])) and all(t == 0.0 for _, _, t in sat)
    ops = {(q.shape, q.h, q.omega) for q, _, _ in r}
    assert len(ops) <= 12
    for q, nrhs, _ in r:
        nx, ny, nz = q.shape
        assert 31 <= min(q.shape) and max(q.shape) <= 255 and 1 <= nrhs <= 64
        ppw = 2 * np.pi / (q.omega * max(q.h))
        assert 8.0 - 1e-9 <= ppw <= 12.0 + 1e-9
    assert len({q.seed for q, _, _ in r}) == len(r)


def test_rhs_is_seeded():
    p = workloads.config_2d_small()
    assert np.array_equal(workloads.rhs(p), workloads.rhs(p))
    assert not np.array_equal(workloads.random_rhs((9, 7), 1), workloads.random_rhs((9, 7), 2))
