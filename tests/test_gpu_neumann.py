"""Neumann faces (Section 2's Gamma_N, du/dn = 0: the corner entries of eq.
matrixK are 1 instead of 1 - i w h) on some axes, absorbing faces on the
others: the CUDA path (helm_plan_2d_bc / helm_plan_3d_bc through the C ABI)
against the CPU oracle assembled with the same per-axis conditions.

A Neumann x1 axis uses the closed-form cosine eigen-data in place of the
absorbing pencil's, and C_bb's corner 1/h - w^2 h/3; a Neumann tridiagonal
axis changes the end entries of every line matrix.  Tolerance 1e-10 in the
2-norm and the max-norm, as for the absorbing-only parity tests.
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


def _case(shape, lengths, ppw, bc):
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    return shape, h, ppw_omega(max(h), ppw), bc


CASES = {
    "2d_neumann_x": _case((65, 48), (1.0, 0.75), 10, ("neumann", "abc")),
    "2d_neumann_x1": _case((65, 48), (1.0, 0.75), 10, ("abc", "neumann")),
    "2d_aniso_neumann_x1": _case((40, 100), (0.6, 1.7), 8, ("abc", "neumann")),
    "3d_neumann_x": _case((14, 16, 12), (1.0, 1.1, 0.9), 6, ("neumann", "abc", "abc")),
    "3d_neumann_y": _case((14, 16, 12), (1.0, 1.1, 0.9), 6, ("abc", "neumann", "abc")),
    "3d_neumann_z": _case((14, 16, 12), (1.0, 1.1, 0.9), 6, ("abc", "abc", "neumann")),
    "3d_neumann_yz": _case((20, 9, 15), (1.5, 0.6, 1.1), 6, ("abc", "neumann", "neumann")),
    "3d_neumann_xz": _case((12, 18, 10), (0.9, 1.4, 0.8), 7, ("neumann", "abc", "neumann")),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("dtype", ["c128", "c64_refined", "c64_ff"])
@pytest.mark.parametrize("aux", ["damped", "periodic"])
def test_mixed_boundaries_match_oracle(env, name, dtype, aux):
    helm, torch = env
    shape, h, omega, bc = CASES[name]
    f = random_rhs(shape, 900 + len(name))
    u_ref, hist = solvers.oracle_solve(f, h, omega, method="banded", bc=bc)
    assert hist[-1] < 1e-13
    code = helm.HELM_C128 if dtype == "c128" else helm.HELM_C64_REFINED
    plan = helm.Plan(shape, h, omega, code, bc=bc)
    if dtype == "c64_ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 15)
    if aux == "periodic":
        helm.helm_set_auxiliary(plan.handle, 0.0, 0)
    u = plan.solve(torch.from_numpy(f).cuda())
    info, st = plan.info()
    plan.close()
    assert list(info.axis_bc[:len(shape)]) == [1 if b == "neumann" else 0 for b in bc]
    un = u.cpu().numpy()
    err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
    errmax = np.abs(un - u_ref).max() / np.abs(u_ref).max()
    print(f"NEUMANN {name} {dtype} {aux}: err={err:.3e} max={errmax:.3e} sweeps={info.iterations}")
    assert err <= TOL and errmax <= TOL
    if dtype != "c128":
        assert st == helm.HELM_OK and info.converged == 1


def test_boundary_kind_validation(env):
    helm, torch = env
    import ctypes

    out = ctypes.c_void_p(1)
    bad = [(ctypes.c_int32 * 2)(1, 1), (ctypes.c_int32 * 2)(0, 2)]  # no absorbing axis; unknown kind
    for bc in bad:
        assert helm.lib.helm_plan_2d_bc(ctypes.byref(out), 9, 9, 0.1, 0.1, 5.0, 0, bc) == helm.HELM_EINVAL
        assert out.value is None
    assert helm.lib.helm_plan_2d_bc(ctypes.byref(out), 9, 9, 0.1, 0.1, 5.0, 0, None) == helm.HELM_EINVAL
    bc3 = (ctypes.c_int32 * 3)(1, 1, 1)
    assert helm.lib.helm_plan_3d_bc(ctypes.byref(out), 5, 5, 5, 0.1, 0.1, 0.1, 5.0, 0, bc3) == helm.HELM_EINVAL
