"""Failure detection without a GPU fault.

* A bounded device wait that runs out: helm_debug_wait_timeout enqueues a
  kernel whose mbarrier wait (the wait the bulk-copy kernels use) can never
  complete, with a short poll limit.  The kernel gives up and returns, the
  plan's error word is set, helm_get_info reports HELM_ETIMEOUT, and the
  CUDA context stays usable (a new plan solves correctly afterwards).
* Host-side allocation-failure injection: every device allocation a plan
  makes is made to fail in turn (helm_debug_fail_alloc).  Each plan either
  fails with HELM_ENOMEM and *out = NULL, or -- when the failed allocation was
  optional memory the plan works around -- still solves to the parity bound;
  either way no device allocation is left behind once it is destroyed.
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


def test_bounded_wait_times_out_and_context_survives(env):
    helm, torch = env
    shape, h, omega = _problem((33, 40), (1.0, 1.2), 10)
    plan = helm.Plan(shape, h, omega, helm.HELM_C128)
    info, st = plan.info()
    assert st == helm.HELM_OK
    assert helm.lib.helm_debug_wait_timeout(plan.handle, 0) == helm.HELM_EINVAL
    assert helm.lib.helm_debug_wait_timeout(plan.handle, 64) == helm.HELM_OK
    torch.cuda.synchronize()  # the kernel returned
    info = helm.helm_info()
    assert helm.lib.helm_get_info(plan.handle, ctypes.byref(info)) == helm.HELM_ETIMEOUT
    assert helm.lib.helm_get_info(plan.handle, ctypes.byref(info)) == helm.HELM_ETIMEOUT  # sticky
    plan.close()
    # the context is still usable: a fresh plan solves to the parity bound
    f = random_rhs(shape, 3)
    u_ref, _ = solvers.oracle_solve(f, h, omega, method="banded")
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    u = plan.solve(torch.from_numpy(f).cuda())
    info, st = plan.info()
    plan.close()
    assert st == helm.HELM_OK
    err = np.linalg.norm(u.cpu().numpy() - u_ref) / np.linalg.norm(u_ref)
    assert err <= 1e-10


def _live(helm):
    b = ctypes.c_size_t(0)
    n = helm.lib.helm_debug_live_allocations(ctypes.byref(b))
    return n, b.value


@pytest.mark.parametrize("case", [((24, 30), (1.0, 1.1), "c128"), ((24, 30), (1.0, 1.1), "c64_ff"),
                                  ((9, 12, 10), (1.0, 1.2, 0.9), "c64_ff"), ((9, 12, 10), (1.0, 1.2, 0.9), "c128")])
def test_every_allocation_failure_is_clean(env, case):
    helm, torch = env
    shape, lengths, mode = case
    shape, h, omega = _problem(shape, lengths, 8)
    f = random_rhs(shape, 11)
    u_ref, _ = solvers.oracle_solve(f, h, omega, method="banded")
    fd = torch.from_numpy(f).cuda()
    torch.cuda.synchronize()
    base = _live(helm)
    code = helm.HELM_C128 if mode == "c128" else helm.HELM_C64_REFINED
    fired_any = False
    for k in range(1, 400):
        before = helm.lib.helm_debug_fail_alloc(0)
        helm.lib.helm_debug_fail_alloc(k)
        out = ctypes.c_void_p(1)
        if len(shape) == 2:
            st = helm.lib.helm_plan_2d(ctypes.byref(out), shape[0], shape[1], h[0], h[1], omega, code)
        else:
            st = helm.lib.helm_plan_3d(ctypes.byref(out), shape[0], shape[1], shape[2], h[0], h[1], h[2], omega,
                                       code)
        if st == helm.HELM_OK and mode == "c64_ff":
            st2 = helm.lib.helm_set_residual(out, helm.HELM_RESID_FF)
        else:
            st2 = helm.HELM_OK
        fired = helm.lib.helm_debug_fail_alloc(0) > before
        if fired:
            fired_any = True
        if st != helm.HELM_OK:
            assert fired and st == helm.HELM_ENOMEM and out.value is None, (k, st)
        else:
            if st2 != helm.HELM_OK:
                assert fired and st2 == helm.HELM_ENOMEM
            else:
                # optional memory missing (or nothing failed): the plan still solves
                u = torch.empty_like(fd)
                helm.lib.helm_set_refinement(out, 1e-12, 15)
                assert helm.lib.helm_solve(out, fd.data_ptr(), u.data_ptr()) == helm.HELM_OK
                info = helm.helm_info()
                assert helm.lib.helm_get_info(out, ctypes.byref(info)) == helm.HELM_OK
                err = np.linalg.norm(u.cpu().numpy() - u_ref) / np.linalg.norm(u_ref)
                assert err <= 1e-10, (k, err)
            assert helm.lib.helm_destroy(out) == helm.HELM_OK
        torch.cuda.synchronize()
        assert _live(helm) == base, f"allocation {k}: device memory left behind"
        if not fired:
            break  # k is past the last allocation of this plan
    else:
        pytest.fail("more than 400 allocations")
    assert fired_any
    print(f"{mode} {shape}: every one of {k - 1} allocations failed once, cleanly")
