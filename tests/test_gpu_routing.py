"""Precision routing (spec: FP64 for the tridiagonal solves of
near-resonant modes): 3D complex64 plans can solve the inner lines whose line
matrix is close to singular with FP64 arithmetic (helm_set_precision_routing).

* On a grid with the 512^3 workload's spacing and wave number, the raw
  complex64 solve's error, resolved over the inner lines, sits almost wholly
  in the near-singular lines.  Routing those lines to FP64 leaves it where it
  is: the error is the complex64 rounding of those modes' inputs (the
  transformed load), which a near-singular line amplifies whatever the
  precision of its own sweeps, not the sweeps' FP32 arithmetic (whose pivots
  are FP64 already).  The test records both facts; routing is therefore off
  by default.
* Routed and unrouted refinements both converge to the parity bound against
  the CPU oracle; tau = 0 routes nothing; 2D and complex128 plans reject the
  setting.
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


def _case(shape, lengths, ppw):
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    return shape, h, ppw_omega(max(h), ppw)


CASES = {
    "cube64_10ppw": _case((64, 64, 64), (1.0, 1.0, 1.0), 10),
    "box96x64x48": _case((96, 64, 48), (1.5, 1.0, 0.75), 8),
}


def _lamB(n, h, rho, q):
    """Eigenvalues of the gamma-circulant auxiliary (closed form of the
    pencil the oracle pins in test_gamma_circulant_is_diagonalised_by_scaled_dft)."""
    t = (rho + 0.5j * np.pi * q) / n
    s = np.sinh((t + 1j * 2 * np.pi * np.arange(n) / n) / 2)
    return (-4 * s * s / h) / (h * (1 + 2 / 3 * s * s))


def test_error_sits_in_near_singular_lines_and_routing_keeps_it(env):
    """On a 160^3 grid with the 512^3 workload's spacing and wave number, the
    error of the raw complex64 solve (against complex128, same auxiliary),
    resolved over the inner lines (l, m) by the DFT over y and z, lies mostly
    in the lines within 2e-2 w^2 of singular; routing exactly those lines to
    FP64 changes neither their share nor the total error by more than a few
    per cent."""
    import workloads

    helm, torch = env
    p = workloads.scaled(workloads.config_3d(), (160, 160, 160))
    f = torch.from_numpy(workloads.rhs(p)).cuda()
    pl64 = helm.Plan(p.shape, p.h, p.omega, helm.HELM_C128)
    out = {}
    for tau in (0.0, 2e-2):
        pl = helm.Plan(p.shape, p.h, p.omega, helm.HELM_C64_RAW)
        info, _ = pl.info()
        rho, q = info.aux_rho, info.aux_q
        helm.helm_set_precision_routing(pl.handle, tau)
        out[tau] = (pl.solve(f.to(torch.complex64)).to(torch.complex128), pl.info()[0].fp64_lines)
        pl.close()
    helm.helm_set_auxiliary(pl64.handle, rho, q)
    u64 = pl64.solve(f)
    pl64.close()
    # inner lines within 2e-2 w^2 of singular, for the outer-B / inner-B type
    lamx = solvers.abc_pencil_eig(p.shape[0], p.h[0], p.omega)[0]
    s = _lamB(p.shape[1], p.h[1], rho, q)[:, None] + _lamB(p.shape[2], p.h[2], rho, q)[None, :] - p.omega ** 2
    dist = np.min(np.abs(s[..., None] + lamx[None, None, :]), axis=-1) / p.omega ** 2
    near = dist < 2e-2
    nrm = torch.linalg.norm(u64).item()
    res = {}
    for tau, (u, nl) in out.items():
        E = (torch.fft.fft2(u - u64, dim=(1, 2)).abs() ** 2).sum(0).cpu().numpy()
        res[tau] = (torch.linalg.norm(u - u64).item() / nrm, E[near].sum() / E.sum(), E[near].sum(), nl)
    print(f"ROUTING 160^3: {near.sum()} near-singular B lines; total err {res[0.0][0]:.3e} -> {res[2e-2][0]:.3e}; "
          f"their error energy {res[0.0][2]:.3e} ({res[0.0][1]*100:.1f}% of all) -> {res[2e-2][2]:.3e}; "
          f"{res[2e-2][3]} FP64 lines")
    assert res[0.0][3] == 0 and res[2e-2][3] > 0
    assert res[0.0][1] > 0.5  # most of the error sits in the near-singular lines
    assert 0.8 * res[0.0][2] < res[2e-2][2] < 1.2 * res[0.0][2]  # FP64 sweeps do not remove it
    assert res[2e-2][0] <= 1.05 * res[0.0][0]


@pytest.mark.parametrize("tau", [0.0, 2e-2, 0.1])
def test_routed_refinement_meets_parity(env, tau):
    helm, torch = env
    shape, h, omega = CASES["box96x64x48"]
    f = random_rhs(shape, 62)
    u_ref, hist = solvers.oracle_solve(f, h, omega, method="tensor")
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    helm.helm_set_precision_routing(plan.handle, tau)
    helm.helm_set_refinement(plan.handle, 2e-11, 10)
    u = plan.solve(torch.from_numpy(f).cuda())
    info, st = plan.info()
    plan.close()
    un = u.cpu().numpy()
    err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
    errmax = np.abs(un - u_ref).max() / np.abs(u_ref).max()
    print(f"tau={tau}: {info.fp64_lines} FP64 lines, sweeps {info.iterations}, err {err:.3e}")
    assert st == helm.HELM_OK and info.converged == 1
    assert err <= TOL and errmax <= TOL
    assert (info.fp64_lines > 0) == (tau > 0)


def test_routing_setting_validation(env):
    helm, torch = env
    shape, h, omega = _case((9, 12), (1.0, 1.2), 8)
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    assert helm.lib.helm_set_precision_routing(plan.handle, 1e-2) == helm.HELM_EUNSUPPORTED
    plan.close()
    shape, h, omega = _case((9, 12, 10), (1.0, 1.2, 0.9), 8)
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    assert helm.lib.helm_set_precision_routing(plan.handle, 1e-2) == helm.HELM_EUNSUPPORTED
    plan.close()
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    assert helm.lib.helm_set_precision_routing(plan.handle, -1.0) == helm.HELM_EINVAL
    assert helm.lib.helm_set_precision_routing(plan.handle, 0.0) == helm.HELM_OK
    info, st = plan.info()
    assert info.fp64_lines == 0
    plan.close()
