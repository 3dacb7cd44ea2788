"""Batches of independent problems (helm_batch_*): every plan's result in the
batch equals its own helm_solve, bit for bit (the same kernels on the same
data, launched as branches of one CUDA graph), for mixed sizes, wave numbers,
2D and 3D, and all modes; the graph is reused while the buffers stay and
captured again when they move."""
import numpy as np
import pytest

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


MIX = [
    ((9, 7), (1.0, 1.0), 4, "c128"),
    ((40, 24), (1.3, 0.7), 8, "c64_ff"),
    ((65, 100), (0.64, 1.0), 10, "c64_refined"),
    ((31, 37), (1.0, 1.2), 7, "c64_raw"),
    ((17, 512), (0.1, 3.0), 10, "c64_ff"),
    ((130, 64), (1.3, 0.63), 12, "c128"),
    ((200, 256), (2.0, 2.5), 6, "c64_ff"),
    ((5, 6, 7), (1.0, 1.0, 1.0), 4, "c64_ff"),
    ((12, 17, 10), (1.1, 1.6, 0.9), 6, "c128"),
    ((20, 9, 33), (1.9, 0.8, 3.2), 8, "c64_refined"),
]


def _make(helm, shape, lengths, ppw, mode):
    shape, h, omega = _problem(shape, lengths, ppw)
    code = {"c128": helm.HELM_C128, "c64_raw": helm.HELM_C64_RAW}.get(mode, helm.HELM_C64_REFINED)
    plan = helm.Plan(shape, h, omega, code)
    if mode == "c64_ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 12)
    elif mode == "c64_refined":
        helm.helm_set_refinement(plan.handle, 1e-13, 12)
    return plan


def test_batch_equals_single_solves(env):
    helm, torch = env
    plans = [_make(helm, *m) for m in MIX]
    fs = []
    for i, (plan, m) in enumerate(zip(plans, MIX)):
        f = torch.from_numpy(random_rhs(plan.shape, 500 + i)).cuda().to(plan.tensor_dtype)
        fs.append(f)
    alone = []
    for plan, f in zip(plans, fs):
        alone.append(plan.solve(f).clone())
    torch.cuda.synchronize()
    batch = helm.Batch(plans)
    try:
        for rep in range(3):
            # reps 0 and 1 reuse the buffers (graph reused); rep 2 moves u
            if rep != 1:
                us = [torch.full_like(f, float("nan")) for f in fs]
            batch.solve(fs, us)
            torch.cuda.synchronize()
            for i, (plan, u, ua, m) in enumerate(zip(plans, us, alone, MIX)):
                assert torch.equal(u, ua), f"problem {i} {m}: batch differs from its single solve"
                if m[3] in ("c64_ff", "c64_refined"):
                    info, st = plan.info()
                    assert st == helm.HELM_OK and info.converged == 1
    finally:
        batch.close()
        for p in plans:
            p.close()


def test_batch_rejects_bad_arguments(env):
    helm, torch = env
    import ctypes

    h = ctypes.c_void_p(1)
    assert helm.lib.helm_batch_create(ctypes.byref(h), 0, None) == helm.HELM_EINVAL
    assert h.value is None
    plan = _make(helm, (9, 7), (1.0, 1.0), 4, "c128")
    arr = (ctypes.c_void_p * 1)(plan.handle)
    assert helm.lib.helm_batch_create(ctypes.byref(h), 1, arr) == helm.HELM_OK
    f = torch.zeros(plan.shape, dtype=torch.complex128, device="cuda")
    fa = (ctypes.c_void_p * 1)(f.data_ptr())
    assert helm.lib.helm_batch_solve(h, fa, fa) == helm.HELM_EINVAL  # f aliases u
    helm.helm_set_profiling(plan.handle, True)
    u = torch.empty_like(f)
    ua = (ctypes.c_void_p * 1)(u.data_ptr())
    assert helm.lib.helm_batch_solve(h, fa, ua) == helm.HELM_EINVAL  # profiling on
    helm.helm_set_profiling(plan.handle, False)
    assert helm.lib.helm_batch_solve(h, fa, ua) == helm.HELM_OK
    torch.cuda.synchronize()
    assert helm.lib.helm_batch_destroy(h) == helm.HELM_OK
    assert helm.lib.helm_batch_destroy(None) == helm.HELM_OK
    plan.close()


def _oracle_method(q):
    return "banded" if q.N <= 40000 else "tensor"


@pytest.mark.parametrize("residual", ["ff", "fp64"])
def test_batch_workload_sample_matches_oracle(env, residual):
    """A seeded sample of the 512-problem batch workload (mixed sizes up to
    1004 x 1023, anisotropic spacings, 6-20 nodes per wavelength, three of
    the near-resonant problems), solved as one batch with the benchmark's
    settings (complex64 refined to ||r||/||f|| <= 2e-11) and checked problem
    by problem against the CPU oracle (banded LU below 4e4 unknowns, the
    tensor eigen-solve above) in the 2-norm and the max-norm."""
    import numpy as np

    import workloads
    from oracle import solvers

    helm, torch = env
    probs = workloads.batch_2d(512)
    resonant = sorted((i for i, q in enumerate(probs) if q.note), key=lambda i: probs[i].N)[:3]
    rest = sorted((i for i, q in enumerate(probs) if not q.note), key=lambda i: probs[i].N)
    rng = np.random.default_rng(7)
    pick = resonant + [int(i) for i in rng.choice(rest[:256], 3, replace=False)] + [rest[-1]]
    plans, fs, refs = [], [], []
    for i in pick:
        q = probs[i]
        f = workloads.rhs(q)
        u_ref, hist = solvers.oracle_solve(f, q.h, q.omega, method=_oracle_method(q))
        assert hist[-1] < 1e-13
        plan = helm.Plan(q.shape, q.h, q.omega, helm.HELM_C64_REFINED)
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF if residual == "ff" else helm.HELM_RESID_FP64)
        helm.helm_set_refinement(plan.handle, 2e-11, 10)
        plans.append(plan)
        fs.append(torch.from_numpy(f).cuda())
        refs.append(u_ref)
    us = [torch.empty_like(f) for f in fs]
    batch = helm.Batch(plans)
    try:
        batch.solve(fs, us)
        torch.cuda.synchronize()
        for i, plan, u, u_ref in zip(pick, plans, us, refs):
            info, st = plan.info()
            un = u.cpu().numpy()
            err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
            errmax = np.abs(un - u_ref).max() / np.abs(u_ref).max()
            res = float(info.residual[info.iterations])
            print(f"BATCHSAMPLE {residual} #{i} {probs[i].shape} {probs[i].note or 'random'}: err={err:.3e} "
                  f"max={errmax:.3e} sweeps={info.iterations} resid={res:.3e} err/resid={err / res:.2f}")
            assert st == helm.HELM_OK and info.converged == 1
            assert err <= 1e-10 and errmax <= 1e-10
    finally:
        batch.close()
        for p in plans:
            p.close()
