"""Write the stored oracle samples for the full-size workloads.

Calls only oracle/ (and the seeded input module): the O2 tensor eigen-solve
with double-double iterative refinement, at the full problem size.  Stores,
as JSON text, the solution at seeded sample indices plus norms, so the GPU
parity tests and bench.py can check full-size results without rerunning the
oracle.  Usage: python tests/golden/make_golden.py 2d_large|3d
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solvers  # noqa: E402
import workloads  # noqa: E402

CONFIGS = {"2d_large": workloads.config_2d_large, "3d": workloads.config_3d, "2d_small": workloads.config_2d_small}
NSAMPLES = 1024


def sample_indices(N, seed=20240531):
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.unique(np.concatenate([rng.integers(0, N, NSAMPLES), [0, N - 1]]))
    return idx


def main(name):
    p = CONFIGS[name]()
    f = workloads.rhs(p)
    t0 = time.time()
    u, hist = solvers.oracle_solve(f, p.h, p.omega, method="tensor", iters=2)
    secs = time.time() - t0
    idx = sample_indices(p.N)
    flat = u.reshape(-1)
    out = {
        "workload": p.name,
        "shape": list(p.shape),
        "h": list(p.h),
        "omega": p.omega,
        "seed": p.seed,
        "rhs": p.rhs,
        "oracle": "O2 tensor eigen-solve + 2 double-double refinement sweeps",
        "oracle_residual_history": hist,
        "oracle_seconds": secs,
        "norm2": float(np.linalg.norm(flat)),
        "norm_inf": float(np.abs(flat).max()),
        "index": [int(i) for i in idx],
        "re": [repr(float(flat[i].real)) for i in idx],
        "im": [repr(float(flat[i].imag)) for i in idx],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_samples.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print(path, "residuals", hist, "seconds", secs)


def load(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_samples.json")
    with open(path) as fh:
        d = json.load(fh)
    vals = np.array([float(a) + 1j * float(b) for a, b in zip(d["re"], d["im"])])
    return d, np.array(d["index"], dtype=np.int64), vals


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "2d_large")
