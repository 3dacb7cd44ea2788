"""Full-size parity in the launch configuration bench.py times.

The oracle cannot rerun at 33.5M (2D) / 134M (3D) unknowns inside a test, so
its solution was computed once by tests/golden/make_golden.py (oracle only)
and stored at seeded sample indices.  The CUDA result is checked on those
samples (relative 2-norm error <= 1e-10) and, at every node, through the
oracle's double-double residual ||f - A u|| / ||f||.
"""
import os
import sys

import numpy as np
import pytest

import workloads
from oracle import fem

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
from make_golden import load  # noqa: E402

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


CONFIGS = {"2d_large": workloads.config_2d_large, "3d": workloads.config_3d}


@pytest.mark.parametrize("name", ["2d_large", "3d"])
@pytest.mark.parametrize("dtype", ["c128", "c64_refined", "c64_ff"])
def test_fullsize_sampled_parity(env, name, dtype):
    helm, torch = env
    path = os.path.join(HERE, "golden", f"{name}_samples.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    d, idx, vals = load(name)
    p = CONFIGS[name]()
    assert list(p.shape) == d["shape"] and abs(p.omega - d["omega"]) < 1e-9 * p.omega
    f = workloads.rhs(p)
    fd = torch.from_numpy(f).cuda()
    code = helm.HELM_C128 if dtype == "c128" else helm.HELM_C64_REFINED
    plan = helm.Plan(p.shape, p.h, p.omega, code)
    if dtype == "c64_ff":
        helm.helm_set_residual(plan.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(plan.handle, 1e-12, 15)
    u = plan.solve(fd)
    info, st = plan.info()
    plan.close()
    got = u.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    err = np.linalg.norm(got - vals) / np.linalg.norm(vals)
    un = u.cpu().numpy()
    del u, fd
    r = fem.residual_dd_c(f, un, p.h, p.omega)
    rel_res = np.linalg.norm(r) / np.linalg.norm(f)
    print(f"{name} {dtype}: sampled rel err {err:.3e}, rel residual {rel_res:.3e}, iters {info.iterations}")
    assert err <= TOL
    assert rel_res < 1e-9
