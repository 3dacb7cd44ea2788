"""2D parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative 2-norm error against the oracle's refined FP64
solution): 1e-10 for complex128 and for refined complex64; raw complex64 is
reported and bounded loosely (its error is the FP32 solve error amplified by
the conditioning of the periodic auxiliary problem).
"""
import math

import numpy as np
import pytest

from oracle import solvers
from workloads import ppw_omega, random_rhs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1809_03808_gb300 as helm

    return helm, torch


def _case(shape, lengths, ppw=None, omega=None):
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    if omega is None:
        omega = ppw_omega(max(h), ppw)
    return shape, h, omega


CASES = {
    "tiny_9x7": _case((9, 7), (1.0, 1.0), ppw=4),
    "c1_129x129_16pi": _case((129, 129), (1.0, 1.0), omega=16 * math.pi),
    "aniso_40x24": _case((40, 24), (1.3, 0.7), ppw=8),
    "ragged_65x100": _case((65, 100), (0.64, 1.0), ppw=10),
    "primes_31x37": _case((31, 37), (1.0, 1.2), ppw=7),
    "tall_300x64": _case((300, 64), (3.0, 0.63), ppw=12),
    "wide_17x512": _case((17, 512), (0.1, 3.0), ppw=10),
    "pow2_256x128_x1_3x43": _case((256, 129), (2.0, 1.0), ppw=10),
    # power-of-two x1 lengths: compile-time-radix transforms with 1..3 passes
    "pow2_6x32": _case((6, 32), (0.5, 1.0), ppw=8),
    "pow2_5x256": _case((5, 256), (0.1, 2.0), ppw=10),
    "pow2_7x2048": _case((7, 2048), (0.1, 8.0), ppw=10),
    "pow2_4x4096": _case((4, 4096), (0.05, 10.0), ppw=12),
    # x1 lengths with a prime factor above 64: Bluestein's chirp-z transform
    "bluestein_40x67": _case((40, 67), (0.6, 1.0), ppw=8),
    "bluestein_33x257": _case((33, 257), (0.2, 1.6), ppw=10),
    "bluestein_6x1021": _case((6, 1021), (0.05, 6.0), ppw=10),
    "bluestein_20x586": _case((20, 586), (0.3, 4.0), ppw=9),  # 2 x 293
}


def _oracle(shape, h, omega, seed):
    f = random_rhs(shape, seed)
    u, hist = solvers.oracle_solve(f, h, omega, method="banded")
    assert hist[-1] < 1e-13
    return f, u


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("dtype", ["c128", "c64_refined", "c64_ff", "c64_raw"])
@pytest.mark.parametrize("aux", ["damped", "periodic"])
def test_solve_matches_oracle(env, name, dtype, aux):
    helm, torch = env
    shape, h, omega = CASES[name]
    f, u_ref = _oracle(shape, h, omega, seed=sum(map(ord, name)) % 1000)
    code = {"c128": helm.HELM_C128, "c64_refined": helm.HELM_C64_REFINED, "c64_ff": helm.HELM_C64_REFINED,
            "c64_raw": helm.HELM_C64_RAW}[dtype]
    plan = helm.Plan(shape, h, omega, code)
    if dtype == "c64_ff":
        # float-float residual: floor near 1e-13 relative, so a tolerance above it
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 15)
    if aux == "periodic":
        helm.helm_set_auxiliary(plan.handle, 0.0, 0)
    tdt = torch.complex64 if dtype == "c64_raw" else torch.complex128
    fd = torch.from_numpy(f).to("cuda").to(tdt)
    u = plan.solve(fd)
    info, st = plan.info()
    plan.close()
    un = u.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
    errmax = np.abs(un - u_ref).max() / np.abs(u_ref).max()
    print(f"{name} {dtype} {aux}: rel_err={err:.3e} max={errmax:.3e} iters={info.iterations} "
          f"resid={list(info.residual[:info.iterations + 1])}")
    assert np.all(np.isfinite(un))
    if dtype == "c64_raw":
        assert err < 5e-2
    else:
        assert err <= TOL and errmax <= TOL
        if dtype in ("c64_refined", "c64_ff"):
            assert st == helm.HELM_OK and info.converged == 1


AUX = [(0.0, 0), (1.0, 1), (0.5, 2)]


@pytest.mark.parametrize("name", ["tiny_9x7", "aniso_40x24", "c1_129x129_16pi"])
@pytest.mark.parametrize("rho,q", AUX)
def test_stepwise_intermediates(env, name, rho, q):
    """Each step of Section 4.2 against its plain definition: f_hat = DFT of f
    along x1 (eq. step1FFTfcoeff; with the gamma-circulant auxiliary, of
    e^{-t j} f), v_b = boundary rows of B^-1 f (eq. 2dBs1), w_b = boundary rows
    of A^-1 (B - A) v (eq. step2-3), for the paper's periodic B (rho = q = 0)
    and damped ones."""
    helm, torch = env
    shape, h, omega = CASES[name]
    f = random_rhs(shape, 77)
    g = np.exp(rho + 0.5j * np.pi * q)
    t = (rho + 0.5j * np.pi * q) / shape[1]
    v, w, u_ref = solvers.step_definitions(f, h, omega, axis=1, gamma=g)
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    helm.helm_set_auxiliary(plan.handle, rho, q)
    fd = torch.from_numpy(f).cuda()
    u = torch.empty_like(fd)
    fhat = torch.empty_like(fd)
    vb = torch.empty((2, shape[0]), dtype=torch.complex128, device="cuda")
    wb = torch.empty_like(vb)
    helm.helm_set_stream(plan.handle, torch.cuda.current_stream().cuda_stream)
    helm.helm_solve_debug(plan.handle, fd, u, fhat, vb, wb)
    torch.cuda.synchronize()
    plan.close()
    fh_ref = np.fft.fft(f * np.exp(-t * np.arange(shape[1]))[None, :], axis=1)
    assert np.linalg.norm(fhat.cpu().numpy() - fh_ref) / np.linalg.norm(fh_ref) < 1e-13
    vb_ref = np.stack([v[:, 0], v[:, -1]])
    wb_ref = np.stack([w[:, 0], w[:, -1]])
    ev = np.linalg.norm(vb.cpu().numpy() - vb_ref) / np.linalg.norm(vb_ref)
    ew = np.linalg.norm(wb.cpu().numpy() - wb_ref) / np.linalg.norm(wb_ref)
    eu = np.linalg.norm(u.cpu().numpy() - u_ref) / np.linalg.norm(u_ref)
    print(name, ev, ew, eu)
    assert ev < 1e-10 and ew < 1e-10 and eu < 1e-10


def test_repeated_solves_and_host_api(env):
    helm, torch = env
    shape, h, omega = CASES["ragged_65x100"]
    f, u_ref = _oracle(shape, h, omega, seed=5)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    fd = torch.from_numpy(f).cuda()
    u1 = plan.solve(fd)
    u2 = plan.solve(fd)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)
    uh = np.empty_like(f)
    helm.helm_solve_host(plan.handle, f, uh)
    plan.close()
    assert np.linalg.norm(uh - u_ref) / np.linalg.norm(u_ref) <= TOL
    assert np.array_equal(uh, u1.cpu().numpy())


@pytest.mark.parametrize("shape,lengths", [((65, 100), (0.64, 1.0)), ((20, 24, 18), (0.8, 1.0, 0.7))])
@pytest.mark.parametrize("tol", [1e-8, 2e-11, 1e-12, 3e-13])
def test_host_api_fp64_sweep_by_sweep(env, shape, lengths, tol):
    """helm_solve_host with the FP64 residual runs the refinement sweep by
    sweep and starts the copy of u to the host beside the test that the last
    two residuals predict to converge.  Over tolerances where that copy is
    taken early, where the prediction misses and where one sweep or none is
    needed, the host result (page-locked buffers) equals the device-buffer
    solve bit for bit with the same sweeps and residual history."""
    helm, torch = env
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    omega = ppw_omega(max(h), 8)
    f = random_rhs(shape, 19)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    helm.helm_set_refinement(plan.handle, tol, 12)
    u1 = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    i1, s1 = plan.info()
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.full(f.shape, float("nan"), dtype=torch.complex128).pin_memory()
    helm.helm_solve_host(plan.handle, fh, uh)
    i2, s2 = plan.info()
    plan.close()
    print(f"HOST {shape} tol {tol:g}: sweeps {i2.iterations}, residuals {list(i2.residual[:i2.iterations + 1])}")
    assert s1 == s2 == helm.HELM_OK
    assert i1.iterations == i2.iterations
    assert list(i1.residual[:i1.iterations + 1]) == list(i2.residual[:i2.iterations + 1])
    assert np.array_equal(uh.numpy(), u1)


def test_host_api_float_float_mapped_and_pageable(env):
    """helm_solve_host with the float-float residual: page-locked host buffers
    (split and join work on them directly) and pageable ones (staged copies)
    give the device-buffer solve bit for bit."""
    helm, torch = env
    shape, h, omega = CASES["ragged_65x100"]
    f, u_ref = _oracle(shape, h, omega, seed=7)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
    helm.helm_set_refinement(plan.handle, 1e-12, 12)
    u1 = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.full(f.shape, float("nan"), dtype=torch.complex128).pin_memory()
    helm.helm_solve_host(plan.handle, fh, uh)
    up = np.empty_like(f)
    helm.helm_solve_host(plan.handle, f, up)
    plan.close()
    assert np.array_equal(uh.numpy(), u1) and np.array_equal(up, u1)
    assert np.linalg.norm(u1 - u_ref) / np.linalg.norm(u_ref) <= TOL


def test_unsupported_and_invalid(env):
    helm, torch = env
    with pytest.raises(helm.HelmError) as e:
        helm.helm_plan_2d(64, 16384, 0.01, 0.01, 10.0, helm.HELM_C128)
    assert e.value.status == helm.HELM_EUNSUPPORTED
    plan = helm.Plan((9, 9), (0.125, 0.125), 5.0)
    x = torch.zeros(81, dtype=torch.complex128, device="cuda")
    with pytest.raises(helm.HelmError):
        helm.helm_solve(plan.handle, x, x)  # aliasing f and u is rejected
    plan.close()


def test_overlapping_buffers_rejected(env):
    """f and u whose byte ranges share even one element are rejected with
    HELM_EINVAL by every solve entry point, before any kernel runs."""
    helm, torch = env
    shape, h, omega = CASES["tiny_9x7"]
    N = shape[0] * shape[1]
    buf = torch.zeros(2 * N, dtype=torch.complex128, device="cuda")
    f, u = buf.data_ptr(), buf.data_ptr() + (N - 1) * 16  # one shared element
    for code in (helm.HELM_C128, helm.HELM_C64_REFINED):
        plan = helm.Plan(shape, h, omega, code)
        assert helm.lib.helm_solve(plan.handle, f, u) == helm.HELM_EINVAL
        assert helm.lib.helm_solve(plan.handle, u, f) == helm.HELM_EINVAL
        assert helm.lib.helm_solve_debug(plan.handle, f, u, None, None, None) == helm.HELM_EINVAL
        # adjacent, disjoint ranges are fine
        assert helm.lib.helm_solve(plan.handle, buf.data_ptr(), buf.data_ptr() + N * 16) == helm.HELM_OK
        torch.cuda.synchronize()
        plan.close()
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_RAW)
    b32 = torch.zeros(2 * N, dtype=torch.complex64, device="cuda")
    assert helm.lib.helm_solve(plan.handle, b32.data_ptr(), b32.data_ptr() + (N - 1) * 8) == helm.HELM_EINVAL
    plan.close()
    fh = np.zeros(2 * N, dtype=np.complex128)
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    assert helm.lib.helm_solve_host(plan.handle, fh.ctypes.data, fh.ctypes.data + (N - 1) * 16) == helm.HELM_EINVAL
    plan.close()


def test_misaligned_buffers_rejected(env):
    """f or u not on a multiple of the element size (16 B complex128, 8 B
    complex64) is rejected with HELM_EINVAL by every solve entry point, before
    any kernel runs."""
    helm, torch = env
    shape, h, omega = CASES["tiny_9x7"]
    N = shape[0] * shape[1]
    buf = torch.zeros(4 * N, dtype=torch.complex128, device="cuda")
    p = buf.data_ptr()
    for code, es in ((helm.HELM_C128, 16), (helm.HELM_C64_REFINED, 16), (helm.HELM_C64_RAW, 8)):
        plan = helm.Plan(shape, h, omega, code)
        f, u = p, p + 2 * N * 16
        for ff, uu in ((f + es // 2, u), (f, u + es // 2), (f + 4, u + 4)):
            assert helm.lib.helm_solve(plan.handle, ff, uu) == helm.HELM_EINVAL
            assert helm.lib.helm_solve_debug(plan.handle, ff, uu, None, None, None) == helm.HELM_EINVAL
            assert helm.lib.helm_solve_many(plan.handle, 2, ff, uu) == helm.HELM_EINVAL
        # a multiple of the element size is fine
        assert helm.lib.helm_solve(plan.handle, f + es, u + es) == helm.HELM_OK
        torch.cuda.synchronize()
        plan.close()
    fh = np.zeros(4 * N, dtype=np.complex128)
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    assert helm.lib.helm_solve_host(plan.handle, fh.ctypes.data + 8, fh.ctypes.data + 2 * N * 16) == helm.HELM_EINVAL
    plan.close()


def test_set_residual_validation(env):
    helm, torch = env
    shape, h, omega = CASES["tiny_9x7"]
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    assert helm.lib.helm_set_residual(plan.handle, helm.HELM_RESID_FF) == helm.HELM_EINVAL  # not refined
    plan.close()
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    assert helm.lib.helm_set_residual(plan.handle, 7) == helm.HELM_EINVAL
    assert helm.lib.helm_set_residual(plan.handle, helm.HELM_RESID_FF) == helm.HELM_OK
    info, st = plan.info()
    assert info.residual_kind == helm.HELM_RESID_FF
    plan.close()


def test_ff_and_fp64_residuals_agree(env):
    """Both refinement residuals converge to the same solution.  The first
    residual is of the same u0 (the FP32 solve of f) in both and agrees to
    FP32 rounding; later iterates differ by FP32-solve rounding of slightly
    different residuals, so only the converged solutions are compared."""
    helm, torch = env
    shape, h, omega = CASES["c1_129x129_16pi"]
    f = torch.from_numpy(random_rhs(shape, 5)).cuda()
    out = {}
    for kind in (helm.HELM_RESID_FP64, helm.HELM_RESID_FF):
        plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
        helm.helm_set_residual(plan.handle, kind)
        helm.helm_set_refinement(plan.handle, 1e-12, 15)
        u = plan.solve(f)
        info, st = plan.info()
        assert st == helm.HELM_OK and info.converged == 1
        out[kind] = (u.cpu().numpy(), list(info.residual[:info.iterations + 1]))
        plan.close()
    (u64, r64), (uff, rff) = out[helm.HELM_RESID_FP64], out[helm.HELM_RESID_FF]
    print("fp64", r64, "ff", rff)
    assert abs(r64[0] - rff[0]) <= 1e-5 * r64[0]
    assert abs(len(r64) - len(rff)) <= 1
    assert np.linalg.norm(u64 - uff) / np.linalg.norm(u64) < 1e-10


@pytest.mark.parametrize("kind", ["fp64", "ff"])
def test_graph_and_eager_refinement_agree(env, kind):
    """The refinement loop captured as a CUDA graph (device-side while node)
    runs the same kernels as the kernel-by-kernel loop: identical results and
    residual histories, also when the graph is reused and when u moves."""
    helm, torch = env
    shape, h, omega = CASES["ragged_65x100"]
    f = torch.from_numpy(random_rhs(shape, 11)).cuda()
    res = {}
    for graphs in (0, 1):
        plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF if kind == "ff" else helm.HELM_RESID_FP64)
        helm.helm_set_refinement(plan.handle, 1e-12, 10)
        helm.helm_set_graphs(plan.handle, graphs)
        outs = []
        for rep in range(3):
            u = plan.solve(f)  # a fresh u every time: the FP64 graph is recaptured
            info, st = plan.info()
            assert st == helm.HELM_OK and info.converged == 1
            outs.append((u.cpu().numpy(), list(info.residual[:info.iterations + 1])))
        u2 = torch.empty_like(f)
        plan.solve(f, u2)
        plan.solve(f, u2)  # same buffers: the captured graph is reused
        outs.append((u2.cpu().numpy(), None))
        plan.close()
        res[graphs] = outs
    for (a, ra), (b, rb) in zip(res[0], res[1]):
        assert np.array_equal(a, b)
        if ra is not None:
            assert ra == rb


@pytest.mark.parametrize("dtype", ["c64_refined", "c64_ff", "c64_raw"])
def test_long_x1_complex64(env, dtype):
    """x1 length 8192 (complex64 plans only): the persistent bulk-copy fed
    transform of 8192-point lines against the oracle."""
    helm, torch = env
    shape, h, omega = _case((4, 8192), (0.05, 16.0), ppw=12)
    f, u_ref = _oracle(shape, h, omega, seed=8192)
    code = helm.HELM_C64_RAW if dtype == "c64_raw" else helm.HELM_C64_REFINED
    plan = helm.Plan(shape, h, omega, code)
    if dtype == "c64_ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 15)
    tdt = torch.complex64 if dtype == "c64_raw" else torch.complex128
    u = plan.solve(torch.from_numpy(f).to("cuda").to(tdt))
    info, st = plan.info()
    plan.close()
    un = u.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
    print(f"8192 {dtype}: rel_err={err:.3e} iters={info.iterations}")
    if dtype == "c64_raw":
        assert err < 5e-2
    else:
        assert err <= TOL and st == helm.HELM_OK
