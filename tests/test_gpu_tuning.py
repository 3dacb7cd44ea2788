"""The autotuner and its learned cost model (spec: the learned part,
trained on the GPU by the project's own forward and backward kernels; the
paper has no learned component).

* The GPU gradient of the cost-model network (helm_mlp_gradient: the
  library's backward kernels) equals the CPU oracle's backprop
  (oracle/mlp.py, pinned by finite differences) to FP32 rounding.
* Training by helm_mlp_train (Adam, the library's kernels) fits a smooth
  function.
* The gain: on 3D grids of the serving workload's sizes, every variant of
  the tiled inner sweeps is timed (helm_time_solve); a model trained on part
  of the grids picks variants for the held-out grids, and its picks are
  compared, by their measured times, with the fixed default variant and with
  the best measured one.
* Every variant gives the same solution (parity is variant-independent).
"""
import ctypes
import math

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


def _mlp(helm, n_in, n_h, seed):
    h = ctypes.c_void_p()
    assert helm.lib.helm_mlp_create(ctypes.byref(h), n_in, n_h, seed) == helm.HELM_OK
    return h


@pytest.mark.parametrize("n_in,n_h,B", [(9, 32, 64), (3, 5, 7), (16, 48, 200)])
def test_mlp_gradient_matches_oracle(env, n_in, n_h, B):
    from oracle import mlp

    helm, torch = env
    rng = np.random.default_rng(n_in * 100 + n_h)
    h = _mlp(helm, n_in, n_h, 7)
    n = helm.lib.helm_mlp_num_params(h)
    assert n == mlp.num_params(n_in, n_h)
    p = (rng.standard_normal(n) * 0.4).astype(np.float32)
    assert helm.lib.helm_mlp_set_params(h, p.ctypes.data, n) == helm.HELM_OK
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    T = rng.standard_normal(B).astype(np.float32)
    xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    g = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    assert helm.lib.helm_mlp_gradient(h, xd.data_ptr(), td.data_ptr(), B, g.data_ptr(), loss.data_ptr()) == 0
    L_ref, g_ref = mlp.loss_and_gradient(p.astype(np.float64), X, T, n_in, n_h)
    gg = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref)
    print(f"MLP grad {n_in}-{n_h}-{n_h}-1 batch {B}: rel err {rel:.2e}, loss {loss.item():.6f} vs {L_ref:.6f}")
    assert rel < 1e-4
    assert abs(loss.item() - L_ref) <= 1e-5 * max(1.0, abs(L_ref))
    y = torch.empty(B, dtype=torch.float32, device="cuda")
    assert helm.lib.helm_mlp_forward(h, xd.data_ptr(), B, y.data_ptr()) == 0
    y_ref, _ = mlp.forward(p.astype(np.float64), X, n_in, n_h)
    assert np.abs(y.cpu().numpy() - y_ref).max() < 1e-4 * max(1.0, np.abs(y_ref).max())
    # bit-reproducible: the same gradient again
    g2 = torch.empty_like(g)
    assert helm.lib.helm_mlp_gradient(h, xd.data_ptr(), td.data_ptr(), B, g2.data_ptr(), None) == 0
    assert torch.equal(g, g2)
    helm.lib.helm_mlp_destroy(h)


def test_mlp_training_fits(env):
    helm, torch = env
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (256, 2)).astype(np.float32)
    T = (np.sin(2 * X[:, 0]) + X[:, 1] ** 2).astype(np.float32)
    h = _mlp(helm, 2, 16, 3)
    xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    l0 = ctypes.c_float()
    l1 = ctypes.c_float()
    assert helm.lib.helm_mlp_train(h, xd.data_ptr(), td.data_ptr(), 256, 0, ctypes.c_float(1e-2), ctypes.byref(l0)) == 0
    assert helm.lib.helm_mlp_train(h, xd.data_ptr(), td.data_ptr(), 256, 2000, ctypes.c_float(1e-2),
                                   ctypes.byref(l1)) == 0
    print(f"MLP fit: loss {l0.value:.4f} -> {l1.value:.5f}")
    assert l1.value < 0.02 * l0.value
    helm.lib.helm_mlp_destroy(h)


def _grids():
    """3D grids of the serving workload's sizes (nodes per axis in 31..255,
    transform axes 64-smooth), seeded."""
    import workloads

    rng = np.random.default_rng(11)
    smooth = [n for n in range(31, 256) if workloads._max_prime_factor(n) <= 64]
    out = []
    while len(out) < 24:
        nx = int(rng.integers(31, 256))
        ny, nz = int(rng.choice(smooth)), int(rng.choice(smooth))
        if nx * ny * nz <= 6_000_000:
            out.append((nx, ny, nz))
    return out


def test_learned_variant_choice_gains(env):
    from paper_1809_03808_gb300 import tuning

    helm, torch = env
    data = {}
    defaults = {}
    for shape in _grids():
        h = tuple(1.0 / (n - 1) for n in shape)
        plan = helm.Plan(shape, h, ppw_omega(max(h), 10), helm.HELM_C64_REFINED)
        defaults[shape] = tuning.get_variant(plan)
        data[shape] = tuning.measure(plan, reps=3)
        plan.close()
    shapes = list(data)
    train, test = shapes[: 2 * len(shapes) // 3], shapes[2 * len(shapes) // 3:]
    model = tuning.CostModel(hidden=32, seed=2)
    loss = model.train([(s, v, ms) for s in train for v, ms in data[s].items()], steps=4000, lr=3e-3)
    ratios_default, ratios_best = [], []
    for s in test:
        pick = model.choose(s, list(data[s]))
        t_pick, t_def, t_best = data[s][pick], data[s][defaults[s]], min(data[s].values())
        ratios_default.append(t_pick / t_def)
        ratios_best.append(t_pick / t_best)
        print(f"TUNE {s}: default {defaults[s]} {t_def:.3f} ms, model {pick} {t_pick:.3f} ms, best {t_best:.3f} ms")
    gm = lambda r: math.exp(sum(math.log(x) for x in r) / len(r))
    print(f"TUNE summary: training loss {loss:.4f}; held-out geometric mean time model/default "
          f"{gm(ratios_default):.3f}, model/best {gm(ratios_best):.3f}")
    model.close()
    assert gm(ratios_best) < 1.15       # the model's picks are close to the measured best
    assert gm(ratios_default) < 1.0     # and faster than the fixed default, on held-out grids


def test_variants_give_the_same_solution(env):
    from paper_1809_03808_gb300 import tuning
    from oracle import solvers

    helm, torch = env
    shape = (40, 36, 30)
    h = tuple(1.0 / (n - 1) for n in shape)
    omega = ppw_omega(max(h), 8)
    f = random_rhs(shape, 81)
    u_ref, _ = solvers.oracle_solve(f, h, omega, method="tensor")
    plan = helm.Plan(shape, h, omega, helm.HELM_C64_REFINED)
    helm.helm_set_refinement(plan.handle, 2e-11, 10)
    fd = torch.from_numpy(f).cuda()
    for v in tuning.VARIANTS_3D:
        tuning.set_variant(plan, v)
        u = plan.solve(fd).cpu().numpy()
        err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
        assert err <= 1e-10, (v, err)
    plan.close()
