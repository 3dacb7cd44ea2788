"""Request server (helm_server_*): every request's result equals the same
request solved alone by its own plan, bit for bit, when it runs in a mix of
2D and 3D requests of all modes that overlap on several streams and share
cached plans; the plan cache evicts under a small device budget; a request
that can never fit the budget fails with HELM_ENOMEM."""
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


MODES = {
    "c128": dict(dtype=0, residual=0, tol=0.0, max_iter=1),
    "c64_ff": dict(dtype=1, residual=1, tol=1e-11, max_iter=12),  # above the float-float floor
    "c64_fp64": dict(dtype=1, residual=0, tol=1e-13, max_iter=12),
}


def _problem(shape, lengths, ppw):
    h = tuple(L / (n - 1) for n, L in zip(shape, lengths))
    return shape, h, ppw_omega(max(h), ppw)


# (shape, side lengths, nodes per wavelength, mode, nrhs); repeated operators share a plan
MIX = [
    ((40, 24), (1.3, 0.7), 8, "c64_ff", 2),
    ((65, 100), (0.64, 1.0), 10, "c64_fp64", 1),
    ((40, 24), (1.3, 0.7), 8, "c64_ff", 3),
    ((9, 7), (1.0, 1.0), 4, "c128", 1),
    ((12, 17, 10), (1.1, 1.6, 0.9), 6, "c64_ff", 2),
    ((130, 64), (1.3, 0.63), 12, "c128", 2),
    ((40, 24), (1.3, 0.7), 8, "c64_ff", 1),
    ((5, 6, 7), (1.0, 1.0, 1.0), 4, "c128", 1),
    ((12, 17, 10), (1.1, 1.6, 0.9), 6, "c64_ff", 1),
    ((200, 256), (2.0, 2.5), 6, "c64_ff", 2),
]


def _alone(helm, torch, shape, h, omega, mode, f):
    m = MODES[mode]
    plan = helm.Plan(shape, h, omega, m["dtype"])
    try:
        if m["dtype"] == helm.HELM_C64_REFINED:
            helm.helm_set_residual(plan.handle, m["residual"])
            helm.helm_set_refinement(plan.handle, m["tol"], m["max_iter"])
        out = torch.stack([plan.solve(f[j].contiguous()).clone() for j in range(f.shape[0])])
        torch.cuda.synchronize()
        return out
    finally:
        plan.close()


def _inputs(torch, shape, nrhs, seed):
    import numpy as np

    f = np.stack([random_rhs(shape, seed + 17 * j) for j in range(nrhs)])
    return torch.from_numpy(f).cuda()


def _submit(srv, shape, h, omega, mode, f, u):
    m = MODES[mode]
    return srv.submit(shape, h, omega, f, u, dtype=m["dtype"], residual=m["residual"], tol=m["tol"],
                      max_iter=m["max_iter"], nrhs=f.shape[0])


def test_server_mix_equals_alone(env):
    helm, torch = env
    cases = []
    for i, (shape, lengths, ppw, mode, nrhs) in enumerate(MIX):
        shape, h, omega = _problem(shape, lengths, ppw)
        f = _inputs(torch, shape, nrhs, 700 + 31 * i)
        cases.append((shape, h, omega, mode, f, _alone(helm, torch, shape, h, omega, mode, f)))
    srv = helm.Server(nslots=4, device_budget_bytes=8 << 30)
    try:
        us = [torch.full_like(f, float("nan")) for _, _, _, _, f, _ in cases]
        torch.cuda.synchronize()  # the server's streams do not wait on torch's
        tickets = [_submit(srv, shape, h, omega, mode, f, u) for (shape, h, omega, mode, f, _), u in zip(cases, us)]
        results = [srv.wait(t, 120.0) for t in tickets]
        torch.cuda.synchronize()
        for i, ((shape, h, omega, mode, f, ua), u, res) in enumerate(zip(cases, us, results)):
            assert res.done == 1 and res.status == helm.HELM_OK, (i, res.status, srv.error(tickets[i]))
            assert srv.error(tickets[i]) == ""
            if mode != "c128":
                assert res.converged == 1 and res.residual <= MODES[mode]["tol"]
            assert torch.equal(u, ua), f"request {i} ({shape}, {mode}) differs from its solve alone"
        st = srv.stats()
        keys = {(s, h, o, m) for s, h, o, m, _, _ in cases}
        assert st.completed == len(cases) and st.failed == 0
        assert st.plans_built == len(keys) and st.plans_reused == len(cases) - len(keys)
        assert st.plans_evicted == 0
        assert 0 < st.latency_p50_s <= st.latency_p99_s
        assert st.unknowns_solved == sum(f.numel() for *_, f, _ in cases)
    finally:
        srv.close()


def _estimate(shape):
    """The server's admission estimate of a 2D complex64 plan (helm.h)."""
    return 100 * shape[0] * shape[1] + (64 << 20)


def test_server_evicts_under_budget(env):
    helm, torch = env
    ops = [_problem((40, 24), (1.3, 0.7), 8), _problem((30, 32), (1.0, 0.9), 7), _problem((9, 7), (1.0, 1.0), 4)]
    sizes = []
    for shape, h, omega in ops:
        p = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
        helm.helm_set_residual(p.handle, helm.HELM_RESID_FF)
        sizes.append(p.info()[0].device_bytes)
        p.close()
    # any cached plan plus any new plan's estimate exceeds the budget: every
    # change of operator evicts; every single plan fits
    budget = max(_estimate(s) for s, _, _ in ops) + min(sizes) - 1
    order = [0, 1, 0, 2, 2, 1]
    srv = helm.Server(nslots=2, device_budget_bytes=budget)
    try:
        jobs = []
        for i, k in enumerate(order):
            shape, h, omega = ops[k]
            f = _inputs(torch, shape, 1, 900 + i)
            u = torch.empty_like(f)
            torch.cuda.synchronize()
            jobs.append((k, f, u, _submit(srv, shape, h, omega, "c64_ff", f, u)))
        srv.drain(120.0)
        for k, f, u, t in jobs:
            res = srv.wait(t, 0.0)
            assert res.done == 1 and res.status == helm.HELM_OK, (res.status, srv.error(t))
            shape, h, omega = ops[k]
            assert torch.equal(u, _alone(helm, torch, shape, h, omega, "c64_ff", f))
        st = srv.stats()
        assert st.completed == len(order) and st.plans_built == 5 and st.plans_evicted == 4
        assert st.plans_reused == 1 and st.device_bytes_peak <= budget
        # a request whose plan can never fit the budget
        shape, h, omega = _problem((512, 512), (1.0, 1.0), 10)
        f = _inputs(torch, shape, 1, 1)
        u = torch.empty_like(f)
        torch.cuda.synchronize()
        t = _submit(srv, shape, h, omega, "c64_ff", f, u)
        res = srv.wait(t, 60.0)
        assert res.done == 1 and res.status == helm.HELM_ENOMEM
        assert "budget" in srv.error(t)
    finally:
        srv.close()


def test_server_builds_plans_off_the_scheduler(env):
    """While the plan of a large 3D request is being built, a later request
    whose plan is cached starts and finishes: its whole latency is shorter
    than the large request's wait for its plan.  Both results equal their
    solves alone."""
    helm, torch = env
    small = _problem((40, 24), (1.3, 0.7), 8)
    big = _problem((192, 160, 128), (1.0, 0.9, 0.7), 10)
    srv = helm.Server(nslots=2, device_budget_bytes=8 << 30)
    try:
        f0 = _inputs(torch, small[0], 1, 5)
        u0 = torch.empty_like(f0)
        torch.cuda.synchronize()
        assert srv.wait(_submit(srv, *small, "c64_ff", f0, u0), 60.0).status == helm.HELM_OK  # caches its plan
        fb = _inputs(torch, big[0], 1, 6)
        fs = _inputs(torch, small[0], 1, 7)
        ub, us = torch.empty_like(fb), torch.empty_like(fs)
        torch.cuda.synchronize()
        tb = _submit(srv, *big, "c64_fp64", fb, ub)
        ts = _submit(srv, *small, "c64_ff", fs, us)
        rs = srv.wait(ts, 60.0)
        rb = srv.wait(tb, 120.0)
        torch.cuda.synchronize()
        assert rs.status == helm.HELM_OK and rb.status == helm.HELM_OK, (srv.error(ts), srv.error(tb))
        assert rs.plan_reused == 1 and rb.plan_reused == 0
        print(f"SERVER small request latency {rs.latency_s * 1e3:.2f} ms, large request's wait for its plan "
              f"{rb.queue_s * 1e3:.2f} ms")
        assert rs.latency_s < rb.queue_s
        assert torch.equal(us, _alone(helm, torch, *small, "c64_ff", fs))
        assert torch.equal(ub, _alone(helm, torch, *big, "c64_fp64", fb))
        st = srv.stats()
        assert st.plans_built == 2 and st.plans_reused == 1 and st.completed == 3
    finally:
        srv.close()


def test_server_rejects_bad_requests(env):
    helm, torch = env
    import ctypes

    h = ctypes.c_void_p(1)
    assert helm.lib.helm_server_create(ctypes.byref(h), 0, 1 << 30) == helm.HELM_EINVAL
    assert h.value is None
    assert helm.lib.helm_server_create(ctypes.byref(h), 2, 0) == helm.HELM_EINVAL
    srv = helm.Server(nslots=1, device_budget_bytes=1 << 30)
    try:
        shape, hh, omega = _problem((9, 7), (1.0, 1.0), 4)
        f = _inputs(torch, shape, 1, 3)
        with pytest.raises(helm.HelmError):  # f aliases u
            srv.submit(shape, hh, omega, f, f)
        with pytest.raises(helm.HelmError):  # bad tolerance settings
            srv.submit(shape, hh, omega, f, torch.empty_like(f), max_iter=0)
        with pytest.raises(helm.HelmError):  # omega <= 0
            srv.submit(shape, hh, -1.0, f, torch.empty_like(f))
        assert helm.lib.helm_server_wait(srv.handle, 12345, 0.0, None) == helm.HELM_EINVAL
    finally:
        srv.close()
    assert helm.lib.helm_server_destroy(None) == helm.HELM_OK


def test_serving_workload_sample_matches_oracle(env):
    """The three smallest operators of the 3D serving workload (0.6-0.8 M
    unknowns, anisotropic, 8-12 nodes per wavelength), two right-hand sides
    each, served with the benchmark's settings (complex64 refined on the
    float-float residual to ||r||/||f|| <= 2e-11) through one server with two
    streams, each result checked against the CPU oracle's tensor eigen-solve
    in the 2-norm and the max-norm."""
    import numpy as np

    import workloads
    from oracle import solvers

    helm, torch = env
    reqs = workloads.serve_3d(32)
    ops = sorted({(q.shape, q.h, q.omega) for q, _, _ in reqs}, key=lambda o: int(np.prod(o[0])))[:3]
    srv = helm.Server(nslots=2, device_budget_bytes=8 << 30)
    try:
        jobs = []
        for k, (shape, h, omega) in enumerate(ops):
            f = np.stack([workloads.random_rhs(shape, 900 + 10 * k + j) for j in range(2)])
            fd = torch.from_numpy(f).cuda()
            u = torch.empty_like(fd)
            torch.cuda.synchronize()
            t = srv.submit(shape, h, omega, fd, u, dtype=helm.HELM_C64_REFINED, residual=helm.HELM_RESID_FF,
                           tol=2e-11, max_iter=10, nrhs=2)
            jobs.append((t, shape, h, omega, f, fd, u))
        for t, shape, h, omega, f, fd, u in jobs:
            r = srv.wait(t, -1.0)
            assert r.status == helm.HELM_OK and r.converged == 1
            for j in range(2):
                u_ref, hist = solvers.oracle_solve(f[j], h, omega, method="tensor")
                un = u[j].cpu().numpy()
                err = np.linalg.norm(un - u_ref) / np.linalg.norm(u_ref)
                errmax = np.abs(un - u_ref).max() / np.abs(u_ref).max()
                print(f"SERVESAMPLE {shape} rhs {j}: err={err:.3e} max={errmax:.3e} resid={r.residual:.3e}")
                assert err <= 1e-10 and errmax <= 1e-10
    finally:
        srv.close()
