"""The tensor-core transform variant (HELM_VARIANT_DFT = 1): the transforms
along the contiguous axis (x1 in 2D, the inner axis in 3D) of complex64
plans as dense products with the scaled DFT matrix on the tcgen05 tensor
cores (TF32 with high/low operand splitting, FP32 accumulation).

* Refined solves with the variant meet the parity bound against the CPU
  oracle (2-norm and max-norm), for lengths 31..128 including primes (61, 67,
  97, 127) that the FFT path takes through radix-61 or Bluestein passes.
* The raw complex64 solve with the variant stays within a factor 30 of the
  FFT path's error (measured 1.5-14x: the TF32 high and low parts carry 22
  bits, and a dense DFT's rounding grows like sqrt(n) where an FFT's grows
  like log n); refinement removes the difference.
* Timing: the tensor-core transforms against the FFT kernels, per line
  length, on grids of batch and serving sizes (recorded; the autotuner keeps
  the faster per plan).
* The tables follow the auxiliary (rebuilt by helm_set_auxiliary).
* Complex128 plans and lines longer than 128 nodes reject the variant.
"""
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


def _problem(shape, lengths, ppw):
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    return shape, h, ppw_omega(max(h), ppw)


CASES = {
    "2d_40x64": _problem((40, 64), (1.0, 1.6), 10),
    "2d_33x61": _problem((33, 61), (0.8, 1.5), 8),
    "2d_50x97": _problem((50, 97), (0.5, 1.0), 12),
    "2d_24x128": _problem((24, 128), (0.3, 1.6), 10),
    "3d_20x24x67": _problem((20, 24, 67), (0.6, 0.7, 2.0), 8),
    "3d_16x18x128": _problem((16, 18, 128), (0.4, 0.5, 3.0), 8),
    "3d_30x20x31": _problem((30, 20, 31), (1.0, 0.7, 1.0), 8),
    "3d_12x40x127": _problem((12, 40, 127), (0.3, 1.0, 3.2), 8),
}


def _oracle(f, h, omega):
    u, _ = solvers.oracle_solve(f, h, omega, method="tensor" if f.ndim == 3 else "banded")
    return u


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("resid", ["fp64", "ff"])
def test_tensor_core_transform_meets_parity(env, name, resid):
    helm, torch = env
    shape, h, omega = CASES[name]
    f = random_rhs(shape, 77)
    u_ref = _oracle(f, h, omega)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    if resid == "ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 12)
    else:
        helm.helm_set_refinement(plan.handle, 1e-13, 12)
    helm.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, 1)
    assert helm.helm_get_variant(plan.handle, helm.HELM_VARIANT_DFT) == 1
    u = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    info, st = plan.info()
    plan.close()
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    errmax = np.abs(u - u_ref).max() / np.abs(u_ref).max()
    print(f"TC {name} {resid}: err {err:.3e} max {errmax:.3e} sweeps {info.iterations}")
    assert st == helm.HELM_OK and info.converged == 1
    assert err <= TOL and errmax <= TOL


@pytest.mark.parametrize("name", ["2d_33x61", "2d_50x97", "3d_20x24x67", "3d_16x18x128"])
def test_tensor_core_raw_solve_keeps_fp32_accuracy(env, name):
    helm, torch = env
    shape, h, omega = CASES[name]
    f = random_rhs(shape, 78)
    u_ref = _oracle(f, h, omega)
    fd = torch.from_numpy(f).cuda().to(torch.complex64)
    errs = {}
    for v in (0, 1):
        plan = helm.Plan(shape, h, omega, helm.HELM_C64_RAW)
        helm.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, v)
        u = plan.solve(fd).cpu().numpy().astype(np.complex128)
        plan.close()
        errs[v] = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    print(f"TC raw {name}: FFT {errs[0]:.3e}, tensor cores {errs[1]:.3e}")
    assert errs[1] <= 30 * errs[0] + 1e-6


def test_tables_follow_the_auxiliary(env):
    helm, torch = env
    shape, h, omega = CASES["3d_30x20x31"]
    f = random_rhs(shape, 79)
    u_ref = _oracle(f, h, omega)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    helm.helm_set_refinement(plan.handle, 1e-13, 12)
    helm.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, 1)
    for rho, q in ((0.0, 0), (0.5, 1), (1.0, 0)):
        helm.helm_set_auxiliary(plan.handle, rho, q)
        u = plan.solve(torch.from_numpy(f).cuda()).cpu().numpy()
        err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
        print(f"TC aux ({rho}, {q}): err {err:.3e}")
        assert err <= TOL
    plan.close()


def test_variant_validation(env):
    helm, torch = env
    shape, h, omega = CASES["2d_40x64"]
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    assert helm.lib.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, 1) == helm.HELM_EUNSUPPORTED
    plan.close()
    shape, h, omega = _problem((20, 130), (0.5, 1.0), 10)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    assert helm.lib.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, 1) == helm.HELM_EUNSUPPORTED
    assert helm.lib.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, 2) == helm.HELM_EINVAL
    assert helm.lib.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, 0) == helm.HELM_OK
    plan.close()


@pytest.mark.parametrize("shape", [(1024, 61), (1024, 64), (1024, 67), (1024, 97), (1024, 127), (1024, 128),
                                   (64, 64, 61), (64, 64, 67), (64, 64, 127), (64, 64, 128)])
def test_tensor_core_vs_fft_timing(env, shape):
    """Device time of one complex64 solve (helm_time_solve) with the FFT
    kernels and with the tensor-core transforms; the autotuner keeps the
    faster."""
    from paper_1809_03808_gb300 import tuning

    helm, torch = env
    h = tuple(1.0 / (n - 1) for n in shape)
    plan = helm.Plan(shape, h, ppw_omega(max(h), 10), helm.HELM_C64_REFINED)
    t = {}
    for v in (0, 1):
        helm.helm_set_variant(plan.handle, helm.HELM_VARIANT_DFT, v)
        t[v] = helm.helm_time_solve(plan.handle, 5)
    best, timings = tuning.autotune(plan, reps=3)
    chosen = helm.helm_get_variant(plan.handle, helm.HELM_VARIANT_DFT)
    plan.close()
    print(f"TC time {shape}: FFT {t[0]:.3f} ms, tensor cores {t[1]:.3f} ms ({t[1] / t[0]:.2f}x); autotuner keeps "
          f"{'tensor cores' if chosen else 'FFT'}")
    assert "dft_tensor_cores" in timings
    assert chosen == (1 if timings["dft_tensor_cores"] < timings[best] else 0)
