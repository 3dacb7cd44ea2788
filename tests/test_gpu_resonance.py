"""Near-resonant parity: wave numbers placed next to a discrete resonance,
the worst case for the conditioning of the per-mode problems (Section 4.1.2:
every T_l is solved by LU without pivoting).

Two kinds of resonance, both located with the oracle's own eigenvalues:

* "neumann": w^2 at a sum of closed-box (Neumann) eigenvalues of the 1D
  pencils, lam^N_k = 6/h^2 (1 - cos(k pi/(n-1))) / (2 + cos(k pi/(n-1))), one
  per axis -- a physical resonance of the box, damped only by the absorbing
  faces;
* "periodic_mode": w^2 at Lam^B_l + Re Lam^A_m -- a periodic eigenvalue of
  the auxiliary axis (eq. eigvaluesPer) plus the real part of an absorbing
  pencil eigenvalue (eq. EVP1a) of the tridiagonal axis (in 3D plus one more
  periodic eigenvalue), so that the line matrix T_l = K + (Lam^B_l - w^2) M of
  the paper's periodic auxiliary is nearly singular.  Lam^A depends on w
  through the absorbing corner, so the placement is iterated.

Every case runs complex128, complex64 refined on the FP64 residual and on the
float-float residual, each with the plan's own auxiliary and with the paper's
periodic one (rho = q = 0).  Refined plans stop at the benchmark's rule
||r||/||f|| <= 2e-11, so these cases also check that the stop rule keeps the
error within 1e-10 near resonance; each prints its error / residual ratio.
Errors are asserted in the 2-norm and in the max-norm.

One combination is held to a looser bound on purpose: plain complex128 with
the paper's periodic auxiliary at a "periodic_mode" resonance.  There the
auxiliary's own line matrix T_l is nearly singular, and the FP64 rounding of
Steps 1-3 is amplified by its conditioning (measured 3.0e-10 at a relative
distance of 1e-4 from singularity).  The library's default auxiliary (chosen
per plan by trial solves) and every refined path stay within 1e-10 on the
same problems; these cases check that, and bound the paper's periodic
auxiliary by 1e-8.
"""
import numpy as np
import pytest

from oracle import fem, solvers
from workloads import ppw_omega, random_rhs

pytestmark = pytest.mark.gpu

TOL = 1e-10
REFINE_TOL = 2e-11  # the benchmark's stop rule
PAPER_AUX_TOL = 1e-8  # complex128 with the paper's periodic auxiliary at its own resonance


def _tol(dtype, aux, kind):
    return PAPER_AUX_TOL if (dtype == "c128" and aux == "periodic" and kind == "periodic_mode") else TOL


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1809_03808_gb300 as helm

    return helm, torch


def _sum_grid(*vecs):
    out = np.zeros(1)
    for v in vecs:
        out = (out[..., None] + np.asarray(v)[None, :]).ravel()
    return out


def place_resonance(shape, h, omega0, kind):
    """Wave number next to omega0 whose square is a resonance of `kind`.
    Axis 0 is the tridiagonal axis (absorbing pencil), the others periodic."""
    if kind == "neumann":
        sums = _sum_grid(*[fem.eig_neumann(n, hh) for n, hh in zip(shape, h)])
        return float(np.sqrt(sums[np.argmin(np.abs(sums - omega0 ** 2))]))
    # among the pairs within 5 % of omega0^2, the one whose absorbing
    # eigenvalue is least damped (smallest |Im Lam^A_m|) comes closest to a
    # singular T_l; w^2 is set to its real part
    per = _sum_grid(*[fem.eig_periodic_closed(n, hh) for n, hh in zip(shape[1:], h[1:])])
    lamA = solvers.abc_pencil_eig(shape[0], h[0], omega0)[0]
    re = per[:, None] + lamA.real[None, :]
    damp = np.broadcast_to(np.abs(lamA.imag)[None, :], re.shape)
    ok = np.abs(re - omega0 ** 2) <= 0.05 * omega0 ** 2
    l, m = divmod(int(np.argmin(np.where(ok, damp, np.inf))), lamA.size)
    lam_m = lamA[m]
    w = float(np.sqrt(per[l] + lam_m.real))
    for _ in range(6):  # Lam^A depends on w through the absorbing corner
        lamA = solvers.abc_pencil_eig(shape[0], h[0], w)[0]
        lam_m = lamA[int(np.argmin(np.abs(lamA - lam_m)))]  # the same mode, moved
        w = float(np.sqrt(per[l] + lam_m.real))
    return w


def resonance_distance(shape, h, omega):
    """min over periodic modes l and absorbing modes m of
    |Lam^B_l + Lam^A_m - w^2| / w^2 (the periodic auxiliary's nearest line)."""
    per = _sum_grid(*[fem.eig_periodic_closed(n, hh) for n, hh in zip(shape[1:], h[1:])])
    lamA = solvers.abc_pencil_eig(shape[0], h[0], omega)[0]
    return float(np.abs(per[:, None] + lamA[None, :] - omega ** 2).min() / omega ** 2)


CASES_2D = {
    "sq129": ((129, 129), (1.0, 1.0), 10),
    "aniso96x150": ((96, 150), (1.0, 1.4), 8),
    "wide64x252": ((64, 252), (0.5, 2.0), 12),
}
CASES_3D = {
    "cube17": ((17, 17, 17), (1.0, 1.0, 1.0), 8),
    "long48x12x16": ((48, 12, 16), (3.0, 0.7, 1.0), 8),
    "box33x17x9": ((33, 17, 9), (1.6, 0.8, 0.4), 6),
}


def _run(helm, torch, shape, h, omega, dtype, aux, seed):
    f = random_rhs(shape, seed)
    u_ref, hist = solvers.oracle_solve(f, h, omega, method="banded")
    assert hist[-1] < 1e-13
    code = helm.HELM_C128 if dtype == "c128" else helm.HELM_C64_REFINED
    plan = helm.Plan(shape, h, omega, code)
    if dtype == "c64_ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
    if dtype != "c128":
        helm.helm_set_refinement(plan.handle, REFINE_TOL, 15)
    if aux == "periodic":
        helm.helm_set_auxiliary(plan.handle, 0.0, 0)
    u = plan.solve(torch.from_numpy(f).cuda())
    info, st = plan.info()
    plan.close()
    un = u.cpu().numpy()
    err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
    errmax = np.abs(un - u_ref).max() / np.abs(u_ref).max()
    res = float(info.residual[info.iterations]) if dtype != "c128" else float("nan")
    return err, errmax, res, info, st


@pytest.mark.parametrize("name", list(CASES_2D))
@pytest.mark.parametrize("kind", ["neumann", "periodic_mode"])
@pytest.mark.parametrize("dtype", ["c128", "c64_refined", "c64_ff"])
@pytest.mark.parametrize("aux", ["damped", "periodic"])
def test_resonant_2d(env, name, kind, dtype, aux):
    helm, torch = env
    shape, lengths, ppw = CASES_2D[name]
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    omega = place_resonance(shape, h, ppw_omega(max(h), ppw), kind)
    dist = resonance_distance(shape, h, omega)
    err, errmax, res, info, st = _run(helm, torch, shape, h, omega, dtype, aux, seed=400 + len(name))
    ratio = err / res if res == res and res > 0 else float("nan")
    print(f"RESONANT2D {name} {kind} {dtype} {aux}: omega={omega:.6f} dist={dist:.2e} err={err:.3e} "
          f"errmax={errmax:.3e} sweeps={info.iterations} resid={res:.3e} err/resid={ratio:.2f}")
    assert err <= _tol(dtype, aux, kind) and errmax <= _tol(dtype, aux, kind)
    if dtype != "c128":
        assert st == helm.HELM_OK and info.converged == 1


@pytest.mark.parametrize("name", list(CASES_3D))
@pytest.mark.parametrize("kind", ["neumann", "periodic_mode"])
@pytest.mark.parametrize("dtype", ["c128", "c64_refined", "c64_ff"])
@pytest.mark.parametrize("aux", ["damped", "periodic"])
def test_resonant_3d(env, name, kind, dtype, aux):
    helm, torch = env
    shape, lengths, ppw = CASES_3D[name]
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    omega = place_resonance(shape, h, ppw_omega(max(h), ppw), kind)
    dist = resonance_distance(shape, h, omega)
    err, errmax, res, info, st = _run(helm, torch, shape, h, omega, dtype, aux, seed=700 + len(name))
    ratio = err / res if res == res and res > 0 else float("nan")
    print(f"RESONANT3D {name} {kind} {dtype} {aux}: omega={omega:.6f} dist={dist:.2e} err={err:.3e} "
          f"errmax={errmax:.3e} sweeps={info.iterations} resid={res:.3e} err/resid={ratio:.2f}")
    assert err <= _tol(dtype, aux, kind) and errmax <= _tol(dtype, aux, kind)
    if dtype != "c128":
        assert st == helm.HELM_OK and info.converged == 1
