"""helm_solve_many: many right-hand sides of one operator (the paper's
domain-decomposition motivation, Section 1).  Each right-hand side's result is
bit-identical to helm_solve of that right-hand side alone, for 2D and 3D
plans of every mode, with more right-hand sides than workspaces, after the
plan's settings change (workspaces rebuilt), and one of them is checked
against the CPU oracle.
"""
import ctypes

import numpy as np
import pytest

from oracle import solvers
from workloads import ppw_omega, random_rhs

pytestmark = pytest.mark.gpu


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


CASES = [((65, 100), (0.64, 1.0), 10, "c64_ff"), ((65, 100), (0.64, 1.0), 10, "c64_refined"),
         ((130, 64), (1.3, 0.63), 12, "c128"), ((20, 24, 18), (1.9, 1.2, 1.0), 8, "c64_ff"),
         ((20, 24, 18), (1.9, 1.2, 1.0), 8, "c64_refined"), ((12, 17, 10), (1.1, 1.6, 0.9), 6, "c128"),
         ((31, 40), (1.0, 1.3), 7, "c64_raw")]


def _plan(helm, shape, h, omega, mode):
    code = {"c128": helm.HELM_C128, "c64_raw": helm.HELM_C64_RAW}.get(mode, helm.HELM_C64_REFINED)
    plan = helm.Plan(shape, h, omega, code)
    if mode == "c64_ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 12)
    elif mode == "c64_refined":
        helm.helm_set_refinement(plan.handle, 1e-13, 12)
    return plan


@pytest.mark.parametrize("case", CASES)
def test_many_equals_single_solves(env, case):
    helm, torch = env
    shape, lengths, ppw, mode = case
    shape, h, omega = _problem(shape, lengths, ppw)
    nrhs = 7
    tdt = torch.complex64 if mode == "c64_raw" else torch.complex128
    f = torch.from_numpy(np.stack([random_rhs(shape, 300 + j) for j in range(nrhs)])).cuda().to(tdt)
    plan = _plan(helm, shape, h, omega, mode)
    helm.helm_set_rhs_concurrency(plan.handle, 3)
    single = torch.stack([plan.solve(f[j].contiguous()).clone() for j in range(nrhs)])
    for rep in range(2):
        if rep == 1 and mode in ("c64_ff", "c64_refined"):
            helm.helm_set_refinement(plan.handle, 1e-12, 11)  # a setting change: workspaces rebuilt
            single = torch.stack([plan.solve(f[j].contiguous()).clone() for j in range(nrhs)])
        u = torch.full_like(f, complex(float("nan"), float("nan")))
        helm.helm_set_stream(plan.handle, torch.cuda.current_stream().cuda_stream)
        helm.helm_solve_many(plan.handle, nrhs, f, u)
        info, st = plan.info()
        torch.cuda.synchronize()
        for j in range(nrhs):
            assert torch.equal(u[j], single[j]), f"rhs {j} differs from its single solve"
        if mode in ("c64_ff", "c64_refined"):
            assert st == helm.HELM_OK and info.converged == 1
    if mode != "c64_raw":
        u_ref, _ = solvers.oracle_solve(f[4].cpu().numpy(), h, omega)
        err = np.linalg.norm(u[4].cpu().numpy() - u_ref) / np.linalg.norm(u_ref)
        assert err <= 1e-10
    plan.close()


def test_many_argument_checks(env):
    helm, torch = env
    shape, h, omega = _problem((9, 7), (1.0, 1.0), 4)
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    N = 63
    buf = torch.zeros(8 * N, dtype=torch.complex128, device="cuda")
    p = buf.data_ptr()
    # 3 right-hand sides of f overlap the last one of u by one element
    assert helm.lib.helm_solve_many(plan.handle, 3, p, p + (3 * N - 1) * 16) == helm.HELM_EINVAL
    assert helm.lib.helm_solve_many(plan.handle, 0, p, p + 4 * N * 16) == helm.HELM_EINVAL
    assert helm.lib.helm_set_rhs_concurrency(plan.handle, 0) == helm.HELM_EINVAL
    assert helm.lib.helm_set_rhs_concurrency(plan.handle, 17) == helm.HELM_EINVAL
    assert helm.lib.helm_solve_many(plan.handle, 3, p, p + 3 * N * 16) == helm.HELM_OK
    torch.cuda.synchronize()
    plan.close()


MANY_TIMING = [((64, 64, 64), (1.0, 1.0, 1.0), 10, "c64_refined"), ((96, 80, 72), (1.2, 1.0, 0.9), 10, "c64_ff"),
               ((257, 257), (1.0, 1.0), 10, "c64_refined"), ((48, 48, 48), (1.0, 1.0, 1.0), 8, "c128")]


@pytest.mark.parametrize("case", MANY_TIMING)
def test_many_cheaper_than_single_solves(env, case):
    """64 right-hand sides of one serving-size operator: helm_solve_many
    (right-hand sides spread over concurrent workspaces) against 64
    helm_solve calls one after another, both timed with CUDA events on the
    caller's stream after a warm-up."""
    helm, torch = env
    shape, lengths, ppw, mode = case
    shape, h, omega = _problem(shape, lengths, ppw)
    nrhs = 64
    f = torch.from_numpy(np.stack([random_rhs(shape, 500 + j) for j in range(nrhs)])).cuda()
    u = torch.empty_like(f)
    plan = _plan(helm, shape, h, omega, mode)
    if mode != "c128":
        helm.helm_set_refinement(plan.handle, 2e-11, 10)
    s = torch.cuda.current_stream()
    helm.helm_set_stream(plan.handle, s.cuda_stream)

    def singles():
        for j in range(nrhs):
            helm.helm_solve(plan.handle, f[j], u[j])

    def many():
        helm.helm_solve_many(plan.handle, nrhs, f, u)

    times = {}
    for name, fn in (("single", singles), ("many", many)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(2):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / 2
    info, st = plan.info()
    assert st == helm.HELM_OK
    print(f"MANY {shape} {mode}: 64 single solves {times['single']:.2f} ms, helm_solve_many {times['many']:.2f} ms "
          f"({times['many'] / times['single']:.2f}x)")
    plan.close()
    assert times["many"] < times["single"]
