"""Autotuner of the kernel variants, with a learned cost model.

Every variant (helm_set_variant) computes the same solution; their speed
depends on the grid.  Two ways to pick one for a plan:

* ``autotune(plan)`` -- exhaustive: time every variant of the plan with
  helm_time_solve (one solve of the plan's compute path each) and keep the
  fastest.  Costs a few solves per variant at plan time.
* ``CostModel`` -- learned: a small MLP (libhelm's helm_mlp_*, trained on the
  GPU by the library's own forward and backward kernels) maps grid features
  and a variant to the predicted log solve time, so a new plan takes the
  predicted-best variant without timing each.  Trained on measurements made
  with ``measure``.

The paper has no learned part; this serves the autotuner only.  Host-side
argument marshalling and bookkeeping only: measurements, training and
prediction run in libhelm.
"""
from __future__ import annotations

import ctypes
import math

from . import (HELM_C128, HELM_OK, HELM_VARIANT_DFT, HELM_VARIANT_INNER_CHUNK, HELM_VARIANT_INNER_TILES,
               HELM_VARIANT_TRI2D, _check, helm_get_variant, helm_set_variant, helm_time_solve, lib)

# variants of 3D plans: (rows per chunk, tiles per CTA) of the tiled inner sweeps
VARIANTS_3D = tuple((ch, nmb) for ch in (8, 16, 32) for nmb in (1, 2, 4))
# variants of 2D complex64 plans: bulk-copy fed (0) or register-tile (1) passes
VARIANTS_2D = ((0,), (1,))


def plan_variants(plan):
    return VARIANTS_3D if len(plan.shape) == 3 else VARIANTS_2D


def set_variant(plan, v):
    if len(plan.shape) == 3:
        helm_set_variant(plan.handle, HELM_VARIANT_INNER_CHUNK, v[0])
        helm_set_variant(plan.handle, HELM_VARIANT_INNER_TILES, v[1])
    else:
        helm_set_variant(plan.handle, HELM_VARIANT_TRI2D, v[0])


def get_variant(plan):
    if len(plan.shape) == 3:
        return (helm_get_variant(plan.handle, HELM_VARIANT_INNER_CHUNK),
                helm_get_variant(plan.handle, HELM_VARIANT_INNER_TILES))
    return (helm_get_variant(plan.handle, HELM_VARIANT_TRI2D),)


def measure(plan, variants=None, reps=3):
    """{variant: device ms per solve} for every variant the plan accepts
    (variants whose tile does not fit are skipped).  The plan is left on its
    original variant."""
    from . import HelmError

    orig = get_variant(plan)
    out = {}
    for v in variants or plan_variants(plan):
        try:
            set_variant(plan, v)
        except HelmError:
            continue
        out[v] = helm_time_solve(plan.handle, reps)
    set_variant(plan, orig)
    return out


def dft_variant_possible(plan):
    """Complex64 plans whose contiguous transformed axis has at most 128
    nodes can take their transforms on the tensor cores (HELM_VARIANT_DFT)."""
    return plan.dtype != HELM_C128 and plan.shape[-1] <= 128


def autotune(plan, reps=3):
    """Time every variant and keep the fastest; then, where the plan allows
    it, the tensor-core transforms against the FFT kernels with that variant
    (kept only if faster).  Returns (variant, timings); timings has the key
    "dft_tensor_cores" when that was tried."""
    dft = dft_variant_possible(plan)
    if dft:
        helm_set_variant(plan.handle, HELM_VARIANT_DFT, 0)  # the variants are timed with the FFT kernels
    t = measure(plan, reps=reps)
    best = min(t, key=t.get)
    set_variant(plan, best)
    if dft and lib.helm_set_variant(plan.handle, HELM_VARIANT_DFT, 1) == HELM_OK:
        t["dft_tensor_cores"] = helm_time_solve(plan.handle, reps)
        if t["dft_tensor_cores"] >= t[best]:
            helm_set_variant(plan.handle, HELM_VARIANT_DFT, 0)
    return best, t


def features(shape, variant):
    """Inputs of the cost model: log2 of the node counts and of the unknowns,
    the variant's parameters and the derived launch shape of the tiled
    sweeps (chunks per line, CTAs), scaled to O(1)."""
    nx, ny, nz = shape
    ch, nmb = variant
    tiles = math.ceil(nz / 16)
    ctas = ny * math.ceil(tiles / min(nmb, tiles))
    return [math.log2(nx) / 10, math.log2(ny) / 10, math.log2(nz) / 10, math.log2(nx * ny * nz) / 30,
            math.log2(ch) / 5, math.log2(nmb) / 2, math.log2(math.ceil(nx / ch)) / 6, math.log2(ctas) / 17,
            math.log2(max(1, nx * ny * nz // (16 * ch))) / 25]


N_FEATURES = 9


class CostModel:
    """log(ms) = MLP(features(shape, variant)), trained on measurements."""

    def __init__(self, hidden=32, seed=1):
        import torch

        self.torch = torch
        self.handle = ctypes.c_void_p()
        _check(lib.helm_mlp_create(ctypes.byref(self.handle), N_FEATURES, int(hidden), int(seed)), "helm_mlp_create")

    def close(self):
        if self.handle:
            lib.helm_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _x(self, rows):
        t = self.torch
        return t.tensor(rows, dtype=t.float32, device="cuda").contiguous()

    def train(self, samples, steps=3000, lr=3e-3):
        """samples: [(shape, variant, ms)].  Returns the final training loss
        (mean squared error of log ms)."""
        x = self._x([features(s, v) for s, v, _ in samples])
        y = self._x([math.log(ms) for _, _, ms in samples])
        loss = ctypes.c_float(0.0)
        _check(lib.helm_mlp_train(self.handle, x.data_ptr(), y.data_ptr(), x.shape[0], int(steps), float(lr),
                                  ctypes.byref(loss)), "helm_mlp_train")
        return float(loss.value)

    def predict(self, shape, variants):
        """Predicted ms of each variant on `shape`."""
        x = self._x([features(shape, v) for v in variants])
        y = self.torch.empty(x.shape[0], dtype=self.torch.float32, device="cuda")
        _check(lib.helm_mlp_forward(self.handle, x.data_ptr(), x.shape[0], y.data_ptr()), "helm_mlp_forward")
        return {v: math.exp(float(t)) for v, t in zip(variants, y.cpu().tolist())}

    def choose(self, shape, variants=VARIANTS_3D):
        p = self.predict(shape, list(variants))
        return min(p, key=p.get)
