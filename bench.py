"""Benchmark: complex unknowns solved per second by the GB300 fast Helmholtz
solver at relative error <= 1e-10 against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Default workload: the 512^3-node 3D problem (unit cube, ABC on all six faces,
10 nodes per wavelength, seeded complex Gaussian load), the largest
single-GPU configuration.  One step = one full solve (outer Steps 1-3 of the
paper's Section 5.2 with the inner 2D solves of Section 5.1.2, the forward
and inverse transforms) of the whole workload with inputs resident in HBM.
The main line (`--path`, default c64_refined) is the mixed-precision solve:
complex64 transforms and tridiagonal solves with per-plan FP64-built pivot
tables, iterative refinement on an FP64 residual (27-point stencil in FP64)
to ||r||/||f|| <= 2e-11, the loop launched as one CUDA graph.  Its sampled
error against the stored oracle solution is checked in the run.  The plain
complex128 solve, the float-float-residual refinement and the 8192 x 4096 2D
workload in plain complex128 are reported under "variants".  Under torchrun
every rank solves its own replica of the workload (replicas only).

The JSON line on stdout is kept short (per-kernel milliseconds, compact
variants); the full per-kernel roofline table goes to stderr as a second
JSON object.

--impl reference times the CPU oracle (test infrastructure) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "complex unknowns solved/s at rel. err <=1e-10 vs FP64 oracle"
UNIT = "unknowns/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA throughput: 2 DFMA per clock per SM (measured on this GB300 with an
# FMA-chain probe: 1.197 TFLOP/s at 1.995 GHz over 152 SMs), at the 2.07 GHz
# maximum clock.
# The FP64 pipe issues 2 FP64 operations (add, multiply or fused
# multiply-add, one element each) per clock per SM; ALU-bound kernels are
# quoted in FP64 operations per second against that rate.
FP64_PEAK_TFLOPS = 152 * 2 * 2.070e9 / 1e12  # T FP64-op/s
FP64_PEAK_NOTE = "derived: 152 SMs x 2 FP64 ops/clk x 2.07 GHz (issue rate measured by an FMA-chain probe)"

# Solve paths: (helm dtype, refinement residual kind or None).  dtype codes of
# include/helm.h: HELM_C128 = 0, HELM_C64_REFINED = 1; residual kinds
# HELM_RESID_FP64 = 0, HELM_RESID_FF = 1.
PATHS = {"c128": (0, None), "c64_refined": (1, 0), "c64_ff": (1, 1)}
PATHS_NAMES = tuple(PATHS)
PATH_DTYPE = {"c128": "f64", "c64_refined": "f32 solves + f64 residual",
              "c64_ff": "f32 solves + float-float residual"}
PATH_PRECISION = {"c128": "complex128 plain",
                  "c64_refined": "complex64 solves, FP64 residual, refined to ||r||/||f|| <= 2e-11",
                  "c64_ff": "complex64 solves, float-float residual, refined to ||r||/||f|| <= 2e-11"}
# Refinement stop: with the error/residual ratio measured on the 2D and 3D
# workloads (<= 3.1), ||r||/||f|| <= 2e-11 keeps the error below 6.2e-11;
# every run also checks the sampled error against the oracle's solution and
# fails above 1e-10.
REFINE_TOL = 2e-11
# solves run under the library's per-kernel event profiler after the timed
# region (the per-kernel breakdown; never part of `value`)
PROFILE_SOLVES = 2


def sample_shape(workload="3d"):
    """Bounded CPU sample with the workload's spacing and wave number (about
    10-30 s of oracle work on the host cores): 128^3 nodes in 3D, 2048 x 1024
    in 2D."""
    return (128, 128, 128) if workload == "3d" else (2048, 1024)


def workload_problem(name):
    return workloads.config_3d() if name == "3d" else workloads.config_2d_large()


def sig(x, d=4):
    """Round to d significant digits (compact JSON)."""
    if x is None or isinstance(x, (bool, str)):
        return x
    return float(f"{x:.{d}g}")


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# Algorithmic traffic and arithmetic per unknown of each 2D kernel, per
# launch (multiply by N = nx * n1).  Bytes: the kernel's own minimum reads and
# writes, e = bytes per complex value of the compute precision (16 FP64, 8
# FP32); the first solve reads f as complex128, refinement sweeps read the
# complex64 residual, the last transform writes (or updates) complex128 u.
# Flops: real operations of the algorithm as written (complex multiply 6,
# complex add 2, complex reciprocal 5 counting each division as 1).
def kernel_model(name, e, n1, accum=False, first=True, tables=False, ff=False, per_solve=1.0, n1_dim=2):
    import math

    log2n = math.log2(n1)
    # forward-transform input, averaged over the per_solve launches of a
    # refined solve: the first reads f (complex128; with the float-float
    # residual the complex64 hi parts the split wrote), the sweeps read r
    f0 = e if ff else 16
    fin = (f0 + (per_solve - 1.0) * e) / per_solve if first else e
    if tables:
        # FP64 with per-plan line tables: pass 1 reads rhs, m_j, w_j; pass 2
        # reads rhs, m_j, 1/u_j (and step 3 writes x)
        tri = {"tri_step1_pass1": (3 * e, 22.0), "tri_step2_pass1": (2 * e, 18.0),
               "tri_step3_pass1": (3 * e, 24.0), "tri_step1_pass2": (3 * e, 34.0),
               "tri_step2_pass2": (2 * e, 36.0), "tri_step3_pass2": (4 * e, 30.0)}
    else:
        # complex64: the rhs (f_hat; Step 2 only face vectors) and, in Step 3,
        # the solution; the per-plan 1/u_j table is read only for rows before
        # the pivots settle, so it is not counted
        tri = {"tri_step1_pass1": (e, 67.0), "tri_step2_pass1": (0.0, 61.0), "tri_step3_pass1": (e, 75.0),
               "tri_step1_pass2": (e, 53.0), "tri_step2_pass2": (0.0, 47.0), "tri_step3_pass2": (2 * e, 55.0)}
    # 3D (n1 = the y / z length): z transforms on rows, y transforms in place
    # on columns; k_plane3d per outer step: per inner step the forward sweep
    # reads 1/den and writes d, the backward sweep reads both (4e), x3 steps,
    # plus f_hat read in inner Steps 1 and 3 (outer Steps 1, 3) and y3 written
    c128 = e == 16
    # tiled inner sweeps (3D): the rhs read from f_hat in outer Steps 1, 3
    # (inner Steps 1, 3), y3 written in inner Step 3; inner Step 2 and outer
    # Step 2 generate their right-hand sides from face vectors (no bulk bytes)
    if name.startswith("inner_o") and len(name) == 11:
        o, i = int(name[7]), int(name[10])
        byts = (e if (o != 2 and i != 2) else 0.0) + (e if i == 3 else 0.0)
        return (byts, 80.0) if byts > 0 else None
    tab3 = {
        "dft_z_fwd": ((16 if c128 else 8) + e, 5.0 * log2n),
        "dft_y_fwd": (2 * e, 5.0 * log2n),
        "dft_y_inv": (2 * e, 5.0 * log2n),
        "dft_z_inv": (e + (16 if c128 else 32), 5.0 * log2n),
        "plane3d_step1": (15 * e, 100.0),
        "plane3d_step2": (13 * e, 90.0),
        "plane3d_step3": (15 * e, 100.0),
        "reduce_outer": (e, 8.0),
    }
    if name in tab3:
        return tab3[name]
    tab = {
        "dft_fwd": (fin + e, 5.0 * log2n),
        # refined paths: the first solve writes u (16 B), the sweeps update it (32 B)
        "dft_inv": (e + ((16.0 + (per_solve - 1.0) * 32.0) / per_solve if accum else 16 if e == 16 else 8),
                    5.0 * log2n),
        # f, u complex128 in, r complex64 out; FP64 instructions per unknown of
        # the monomial form (2D: 3 sums, 4 multiply-adds, ... = 14; 3D: 26)
        "residual_fp64": (40.0, 14.0 if n1_dim == 2 else 26.0),
        # f, u float-float (16 B each) in, r complex64 out
        "residual_ff": (40.0, 40.0),
        "split_ff": (40.0, 4.0),  # f in, float-float f and its hi parts out
        "join_ff": (32.0, 2.0),
    }
    tab.update(tri)
    return tab.get(name)


# DRAM bytes (read + write) per unknown of one launch, from an ncu capture of
# the same kernel on a smaller grid with the workload's spacing and wave
# number (the traffic of these kernels grows with the number of unknowns);
# kept only while the kernel is unchanged since the capture.
NCU_TRAFFIC_PER_UNKNOWN = {
    ("2d", "c64_ff", "residual_ff"): (
        (546.5e6 + 118.0e6 + 2.5e6) / (4096 * 4096),
        "ncu --set full, 4096 x 4096: k_residual2d_ff + k_perimeter2d_ff "
        "(profiles/ncu_2d_kernels_4096x4096.md)"),
    # DRAM bytes of one k_residual3d_tma launch on 256^3 (same spacing and wave
    # number), per unknown; the traffic of a launch is proportional to them
    ("3d", "c64_refined", "residual_fp64"): (
        (569.948416e6 + 118.337536e6) / 256 ** 3,
        "ncu --set full, 256^3: k_residual3d_tma (profiles/ncu_residual3d_tma_256cube.md), scaled by unknowns"),
}


def roofline_entry(name, launches, tot_ms, steps, N, e, n1, peaks, fp64, accum=False, tables=False, ff=False, dim=2):
    per_launch_ms = tot_ms / launches
    model = kernel_model(name, e, n1, accum=accum, tables=tables, ff=ff, per_solve=max(1.0, launches / steps),
                         n1_dim=dim)
    out = {"kernel": name, "launches_per_step": launches / steps, "ms_per_launch": per_launch_ms}
    if model is None or model[0] == 0:  # no bulk bytes: timed only
        return out
    byts, flops = model[0] * N, model[1] * N
    gbs = byts / (per_launch_ms * 1e-3) / 1e9
    tfl = flops / (per_launch_ms * 1e-3) / 1e12
    hbm = peaks.get("hbm_gbs")
    alu_frac = tfl / FP64_PEAK_TFLOPS
    hbm_frac = gbs / hbm if hbm else None
    # the binding resource: FP64 arithmetic for FP64 kernels unless the HBM
    # fraction is the larger one
    if (fp64 or name == "residual_fp64") and (hbm_frac is None or alu_frac >= hbm_frac):
        out.update({"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "T FP64-op/s",
                    "frac": alu_frac, "peak_source": FP64_PEAK_NOTE,
                    "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": byts,
                    "hbm_GBps": gbs, "hbm_frac_of_measured": hbm_frac})
    else:
        out.update({"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                    "frac": hbm_frac, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                    "algorithmic_bytes_per_launch": byts, "algorithmic_flops_per_launch": flops,
                    "fp64_frac": alu_frac if fp64 else None})
    out["traffic"] = None
    return out


def run_gb300(args):
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    try:
        import paper_1809_03808_gb300 as helm
    except ImportError:
        import __graft_entry__

        __graft_entry__.build()
        import paper_1809_03808_gb300 as helm

    if args.workload == "batch2d":
        return run_batch(args, helm, torch, dev, world, rank, local)
    if args.workload == "serve3d":
        return run_serve(args, helm, torch, dev, world, rank, local)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        import torch.distributed as dist

        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def load_problem(wl):
        p = workload_problem(wl)
        if args.shape and wl == args.workload:
            p = workloads.scaled(p, tuple(int(x) for x in args.shape.split(",")))
        f_host = workloads.rhs(p)
        return p, f_host, torch.from_numpy(f_host).to(dev)

    def timed(plan, f, u):
        """K solves, CUDA events on the launching stream, no profiler."""
        helm.helm_set_stream(plan.handle, stream.cuda_stream)
        for _ in range(args.warmup):
            helm.helm_solve(plan.handle, f, u)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            helm.helm_solve(plan.handle, f, u)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = clk.stop()
        return max_over_ranks(e0.elapsed_time(e1)), clocks

    def profiled(plan, f, u, path, sweeps):
        """Per-kernel device times from the library's event profiler (kernel by
        kernel), over PROFILE_SOLVES solves.  Refined paths run exactly the
        sweeps the timed solves took, so no skipped launch enters an average."""
        if PATHS[path][1] is not None:
            helm.helm_set_refinement(plan.handle, REFINE_TOL, max(1, sweeps))
        helm.helm_set_profiling(plan.handle, True)
        # an NVTX range around exactly these solves, so that an ncu launch
        # list can take them alone (--nvtx --nvtx-include "profiled_solves/")
        torch.cuda.nvtx.range_push("profiled_solves")
        for _ in range(PROFILE_SOLVES):
            helm.helm_solve(plan.handle, f, u)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        prof = helm.helm_get_profile(plan.handle)
        helm.helm_set_profiling(plan.handle, False)
        if PATHS[path][1] is not None:
            helm.helm_set_refinement(plan.handle, REFINE_TOL, 10)
        return prof

    def sampled_error(wl, u):
        if args.shape:
            return None
        try:
            sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
            from make_golden import load

            d, idx, vals = load("3d" if wl == "3d" else "2d_large")
            got = u.reshape(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy()
            return float(np.linalg.norm(got - vals) / np.linalg.norm(vals))
        except FileNotFoundError:
            return None

    def make_plan(p, path):
        code, kind = PATHS[path]
        plan = helm.Plan(p.shape, p.h, p.omega, code)
        if kind is not None:
            helm.helm_set_residual(plan.handle, kind)
            helm.helm_set_refinement(plan.handle, REFINE_TOL, 10)
        plan.variant = None
        if len(p.shape) == 3 and args.variant:
            from paper_1809_03808_gb300 import tuning

            plan.variant = [int(x) for x in args.variant.split(",")]
            tuning.set_variant(plan, tuple(plan.variant))
        elif len(p.shape) == 3 and not args.no_autotune:
            # the exhaustive autotuner: every variant of the tiled inner sweeps
            # timed on this plan, the fastest kept (plan time, not timed)
            from paper_1809_03808_gb300 import tuning

            best, _ = tuning.autotune(plan, reps=2)
            plan.variant = list(best)
        return plan

    def kernels_of(p, path, pr):
        f64 = path == "c128"
        return {k: roofline_entry(k, v[0], v[1], PROFILE_SOLVES, p.N, 16 if f64 else 8, p.shape[-1], peaks, fp64=f64,
                                  accum=(k in ("dft_inv", "dft_z_inv") and not f64), tables=f64,
                                  ff=(path == "c64_ff"), dim=len(p.shape))
                for k, v in pr.items()}

    def run_path(wl, p, f, path):
        """Time one path on one workload; returns (summary, details)."""
        plan = make_plan(p, path)
        u = torch.empty_like(f)
        ms, clocks = timed(plan, f, u)
        info, _ = plan.info()
        err = sampled_error(wl, u)
        sweeps = int(info.iterations)
        prof = profiled(plan, f, u, path, sweeps)
        plan_s = info.plan_seconds
        aux = {"rho": info.aux_rho, "q": info.aux_q, "trial_rel_residual": sig(info.aux_trial_residual)}
        refine = None
        if PATHS[path][1] is not None:
            refine = {"sweeps": sweeps, "tol": REFINE_TOL, "converged": bool(info.converged),
                      "history": [sig(float(x), 3) for x in info.residual[:sweeps + 1]]}
            if err is not None and err > 1e-10:
                raise RuntimeError(f"{wl} {path}: sampled error {err:.3e} above the 1e-10 bar")
        return plan, u, {"ms": ms / args.steps, "clocks": clocks, "err": err, "prof": prof, "refine": refine,
                         "plan_s": plan_s, "aux": aux, "device_bytes": int(info.device_bytes),
                         "variant": plan.variant}

    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    wl = args.workload
    p, f_host, f = load_problem(wl)
    N = p.N

    # --- the timed path (the headline) ---
    plan, u, main = run_path(wl, p, f, args.path)
    ms_step = main["ms"]
    value = world * N / (ms_step * 1e-3)

    # e2e through the host-buffer entry point (H2D of f, solve, D2H of u)
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(f_host).pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        helm.helm_set_stream(plan.handle, stream.cuda_stream)
        helm.lib.helm_solve_host(plan.handle, fh.data_ptr(), uh.data_ptr())
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st = helm.lib.helm_solve_host(plan.handle, fh.data_ptr(), uh.data_ptr())
            if st != 0:
                raise RuntimeError(helm.lib.helm_status_string(st))
        t1 = time.perf_counter()
        dt = max_over_ranks((t1 - t0) / args.steps)
        e2e = {"value": sig(world * N / dt), "unit": UNIT, "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16,
               "ms_per_step": sig(dt * 1e3), "api": "helm_solve_host (pinned host buffers)"}
        del fh, uh
    plan.close()
    del u

    # --- the other paths, and the 2D workload in plain complex128 ---
    variants, details = {}, {}
    todo = [] if args.no_variants else [(wl, q) for q in PATHS if q != args.path]
    if not args.no_variants and not args.shape and wl == "3d":
        todo.append(("2d_large", "c128"))
    cur_wl, cur_p, cur_f = wl, p, f
    for vwl, vpath in todo:
        if vwl != cur_wl:
            cur_f = f = None  # free the previous workload's load vector first
            torch.cuda.empty_cache()
            cur_p, _, cur_f = load_problem(vwl)
            cur_wl = vwl
        vp = cur_p
        vplan, vu, r = run_path(vwl, vp, cur_f, vpath)
        vplan.close()
        del vu
        key = vpath if vwl == wl else f"{workload_problem(vwl).name}/{vpath}"
        variants[key] = {"value": sig(world * vp.N / (r["ms"] * 1e-3)), "ms": sig(r["ms"]),
                         "err": sig(r["err"], 2), "dtype": PATH_DTYPE[vpath]}
        if r["refine"]:
            variants[key]["sweeps"] = r["refine"]["sweeps"]
        variants[key]["kernels_ms"] = {k: sig(v[1] / PROFILE_SOLVES, 3) for k, v in r["prof"].items()}
        details[key] = kernels_of(vp, vpath, r["prof"])

    # --- roofline of the dominant kernel of the timed step ---
    prof = main["prof"]
    name, (launches, tot_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    kernels_main = kernels_of(p, args.path, prof)
    tkey = ("3d" if len(p.shape) == 3 else "2d", args.path, name)
    if tkey in NCU_TRAFFIC_PER_UNKNOWN and "achieved" in kernels_main[name]:
        per_u, src = NCU_TRAFFIC_PER_UNKNOWN[tkey]
        kernels_main[name]["traffic"] = per_u * N
        kernels_main[name]["traffic_source"] = src
    rk = kernels_main[name]
    roof = {"kernel": name, "bound": rk.get("bound"), "achieved": sig(rk.get("achieved")), "peak": rk.get("peak"),
            "unit": rk.get("unit"), "frac": sig(rk.get("frac"), 3), "traffic": sig(rk.get("traffic")),
            "launches_per_step": rk.get("launches_per_step"), "ms_per_launch": sig(rk.get("ms_per_launch")),
            "peak_source": "measured" if rk.get("bound") == "hbm" else "derived FP64 FMA peak"}
    # kernels of one solve (the profiled solves launch exactly the timed ones)
    gpu_launches = int(round(sum(v[0] for v in prof.values()) / PROFILE_SOLVES)) * args.steps

    # --- CPU oracle baseline (rank 0, N = 1 only) ---
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_run(wl, p, 1)

    line = {
        "metric": METRIC, "value": sig(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sig(ms_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PATH_DTYPE[args.path], "data": "synthetic (seeded complex Gaussian"
        + (" x Gaussian bump)" if p.rhs == "gaussian_bump" else ")"),
        "config": {"workload": p.name, "nodes": list(p.shape), "omega": sig(p.omega, 8),
                   "precision": PATH_PRECISION[args.path], "rhs_per_step": 1,
                   "l2": f"inputs larger than L2 ({N * 16 / 1e6:.0f} MB each)", "parallelism": f"replicas x{world}",
                   "variant": main["variant"]},
        "gpu_launches": gpu_launches, "rel_err_sampled": sig(main["err"], 3), "refinement": main["refine"],
        "roofline": roof, "clocks": main["clocks"], "e2e": e2e, "cpu_baseline": cpu,
        "kernels_ms_per_step": {k: sig(v[1] / PROFILE_SOLVES, 3) for k, v in prof.items()},
        "variants": {k: {a: b for a, b in v.items() if a != "kernels_ms"} for k, v in variants.items()},
        "plan_seconds": sig(main["plan_s"], 3),
    }
    if rank == 0:
        full = {"kernels": kernels_main, "variants": variants, "variant_kernels": details, "auxiliary": main["aux"],
                "device_bytes": main["device_bytes"]}
        print(json.dumps(full), file=sys.stderr)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_batch(args, helm, torch, dev, world, rank, local):
    """The batched 2D workload (workloads.batch_2d): every problem refined in
    complex64 with the float-float residual to ||r||/||f|| <= REFINE_TOL, all
    solved by one helm_batch_solve (one CUDA graph launch) per step.  The same
    plans solved one helm_solve after another are reported beside it."""
    probs = workloads.batch_2d(args.batch_count)
    t0 = time.perf_counter()
    plans = []
    for q in probs:
        pl = helm.Plan(q.shape, q.h, q.omega, helm.HELM_C64_REFINED)
        helm.helm_set_residual(pl.handle, helm.HELM_RESID_FF)
        helm.helm_set_refinement(pl.handle, REFINE_TOL, 10)
        plans.append(pl)
    plan_s = time.perf_counter() - t0
    fs = [torch.from_numpy(workloads.rhs(q)).to(dev) for q in probs]
    us = [torch.empty_like(f) for f in fs]
    N = sum(q.N for q in probs)
    stream = torch.cuda.current_stream(dev)
    batch = helm.Batch(plans)

    def timed(step):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, clk.stop()

    ms_b, clocks = timed(lambda: batch.solve(fs, us))
    sweeps, conv, worst = [], 0, 0.0
    for pl in plans:
        info, st = pl.info()
        sweeps.append(int(info.iterations))
        conv += int(info.converged)
        worst = max(worst, float(info.residual[info.iterations]))

    def one_by_one():
        for pl, f, u in zip(plans, fs, us):
            pl.solve(f, u)

    ms_s, _ = timed(one_by_one)
    batch.close()
    line = {
        "metric": METRIC, "value": world * N / (ms_b * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PATH_DTYPE["c64_ff"], "data": "synthetic (seeded complex Gaussians)",
        "config": {"workload": f"batch2d_{len(probs)}", "problems": len(probs), "unknowns": N,
                   "nodes_range": [min(min(q.shape) for q in probs), max(max(q.shape) for q in probs)],
                   "near_resonance": sum(1 for q in probs if q.note), "precision": PATH_PRECISION["c64_ff"],
                   "launch": "one CUDA graph per step (helm_batch_solve)", "parallelism": f"replicas x{world}"},
        "refinement": {"converged": conv, "problems": len(probs), "sweeps_min": min(sweeps),
                       "sweeps_max": max(sweeps), "worst_final_rel_residual": worst, "tol": REFINE_TOL},
        "variants": {"one_by_one": {"value": world * N / (ms_s * 1e-3), "unit": UNIT, "ms_per_step": ms_s,
                                    "launch": "helm_solve per problem (each refinement loop one graph)"}},
        "plan_seconds": plan_s, "clocks": clocks,
    }
    for pl in plans:
        pl.close()
    if rank == 0:
        print(json.dumps(line))


def run_serve(args, helm, torch, dev, world, rank, local):
    """The serving workload (workloads.serve_3d): a Poisson stream of 3D
    requests, 1-64 right-hand sides each, over a pool of operators, submitted
    at their arrival times to one helm_server (plan cache under a device
    budget, several streams).  Complex64 solves refined on the float-float
    residual to ||r||/||f|| <= REFINE_TOL.  value = unknowns x right-hand
    sides solved / wall time from the first arrival to the last completion
    (plan builds included); latency percentiles from submit to completion."""
    reqs = workloads.serve_3d(args.serve_count, rate_per_s=args.serve_rate)
    budget = int(args.serve_budget_gb * (1 << 30))
    gen = torch.Generator(device=dev)

    def make_rhs(q, nrhs):
        gen.manual_seed(q.seed)
        re = torch.randn((nrhs, *q.shape), dtype=torch.float64, device=dev, generator=gen)
        im = torch.randn((nrhs, *q.shape), dtype=torch.float64, device=dev, generator=gen)
        return torch.complex(re, im)

    # warm-up: library load and one small request on a separate server
    q0, _, _ = reqs[0]
    w = helm.Server(nslots=1, device_budget_bytes=budget)
    f0 = make_rhs(workloads.scaled(q0, (31, 32, 32)), 1)
    u0 = torch.empty_like(f0)
    torch.cuda.synchronize()
    w.wait(w.submit((31, 32, 32), q0.h, q0.omega, f0, u0, tol=REFINE_TOL, max_iter=10), -1.0)
    w.close()
    del f0, u0

    srv = helm.Server(nslots=args.serve_slots, device_budget_bytes=budget)
    clk = ClockSampler(local)
    clk.start()
    t0 = time.perf_counter()
    tickets, results = [], {}

    def collect(block):
        for t in tickets:
            if t not in results:
                r = srv.wait(t, -1.0 if block else 0.0)
                if r.done:
                    results[t] = r  # the server drops its references to f, u

    for q, nrhs, at in reqs:
        delay = at - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        f = make_rhs(q, nrhs)
        u = torch.empty_like(f)
        torch.cuda.current_stream(dev).synchronize()  # the server's streams do not wait on torch's
        tickets.append(srv.submit(q.shape, q.h, q.omega, f, u, tol=REFINE_TOL, max_iter=10, nrhs=nrhs))
        del f, u
        collect(False)
    collect(True)
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    ok = [r for r in results.values() if r.status == helm.HELM_OK]
    line = {
        "metric": METRIC, "value": world * st.unknowns_solved / wall, "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PATH_DTYPE["c64_ff"],
        "data": "synthetic (complex Gaussians from a seeded torch CUDA generator)",
        "config": {"workload": f"serve3d_{len(reqs)}", "requests": len(reqs),
                   "operators": len({q.shape for q, _, _ in reqs}), "arrival_rate_per_s": args.serve_rate,
                   "slots": args.serve_slots, "device_budget_bytes": budget,
                   "unknowns_x_rhs": sum(q.N * n for q, n, _ in reqs),
                   "nodes_range": [min(min(q.shape) for q, _, _ in reqs), max(max(q.shape) for q, _, _ in reqs)],
                   "nrhs_range": [min(n for _, n, _ in reqs), max(n for _, n, _ in reqs)],
                   "precision": PATH_PRECISION["c64_ff"], "launch": "helm_server (plan cache, FIFO admission)",
                   "parallelism": f"replicas x{world}"},
        "latency": {"p50_s": st.latency_p50_s, "p99_s": st.latency_p99_s, "mean_s": st.latency_mean_s,
                    "queue_p50_s": sorted(r.queue_s for r in results.values())[len(results) // 2]},
        "server": {"completed": st.completed, "failed": st.failed, "plans_built": st.plans_built,
                   "plans_reused": st.plans_reused, "plans_evicted": st.plans_evicted,
                   "device_bytes_peak": st.device_bytes_peak},
        "refinement": {"converged": len(ok), "requests": len(reqs),
                       "worst_final_rel_residual": max((r.residual for r in results.values()), default=None),
                       "tol": REFINE_TOL},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))


def cpu_baseline_run(wl, p, steps):
    from oracle import solvers

    shape = sample_shape(wl)
    sp = workloads.scaled(p, shape)
    f = workloads.rhs(sp)
    t0 = time.perf_counter()
    for _ in range(steps):
        solvers.oracle_solve(f, sp.h, sp.omega, method="tensor", iters=2)
    dt = (time.perf_counter() - t0) / steps
    cores = len(os.sched_getaffinity(0))
    return {"value": sig(sp.N / dt), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{'x'.join(map(str, shape))} nodes, same h and omega (O2 tensor eigen-solve + 2 double-double "
                      f"refinement sweeps), {dt:.2f} s per solve; BLAS threads = host cores"}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    wl = args.workload if args.workload in ("3d", "2d_large") else "3d"
    p = workload_problem(wl)
    from oracle import solvers

    shape = sample_shape(wl)
    sp = workloads.scaled(p, shape)
    f = workloads.rhs(sp)
    for _ in range(args.warmup):
        solvers.oracle_solve(f, sp.h, sp.omega, method="tensor", iters=2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solvers.oracle_solve(f, sp.h, sp.omega, method="tensor", iters=2)
    dt = (time.perf_counter() - t0) / args.steps
    value = sp.N / dt
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded complex Gaussian"
        + (" x Gaussian bump)" if p.rhs == "gaussian_bump" else ")"),
        "config": {"workload": p.name, "nodes": list(p.shape), "h": list(p.h), "omega": p.omega,
                   "sample": f"{'x'.join(map(str, shape))} nodes, same spacing and wave number"},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores,
                         "sample": f"{'x'.join(map(str, shape))} nodes per step, O2 + 2 dd refinement sweeps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def summarize_launches(path, top=40):
    """Per-kernel table of an ncu launch list (``ncu --metrics
    gpu__time_duration.sum --csv --log-file PATH``): launches, total device
    time and share of each kernel, template arguments kept, parameters
    dropped.  Per-launch times under ncu are cold-cache and serialised, so
    the shares are the comparable figure."""
    import csv

    scale = {"nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0, "second": 1e3}
    with open(path, newline="") as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    rows = list(csv.reader(lines))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Value" in r)
    col = {h: i for i, h in enumerate(rows[hdr])}
    agg = {}
    for r in rows[hdr + 1:]:
        if len(r) < len(col) or r[col["Metric Name"]] != "gpu__time_duration.sum":
            continue
        name = r[col["Kernel Name"]]
        name = name[5:] if name.startswith("void ") else name
        for ns in ("(anonymous namespace)::", "<unnamed>::", "unnamed>::"):
            name = name.replace(ns, "")
        name = name.replace("(int)", "")
        depth, cut = 0, len(name)
        for i, ch in enumerate(name):  # drop the parameter list, keep template arguments
            depth += ch == "<"
            depth -= ch == ">"
            if ch == "(" and depth == 0:
                cut = i
                break
        name = name[:cut]
        ms = float(r[col["Metric Value"]].replace(",", "")) * scale.get(r[col["Metric Unit"]], 1e-6)
        n, t = agg.get(name, (0, 0.0))
        agg[name] = (n + 1, t + ms)
    total = sum(t for _, t in agg.values())
    print(f"{'kernel':<58} {'launches':>8} {'total ms':>10} {'share':>7}")
    for name, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1])[:top]:
        print(f"{name[:58]:<58} {n:>8} {t:>10.3f} {100 * t / total:>6.1f}%")
    print(f"{'all kernels':<58} {sum(n for n, _ in agg.values()):>8} {total:>10.3f} {100.0:>6.1f}%")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", default="", help="nx,ny: same spacing and wave number on a smaller grid "
                    "(profiling cases; not a benchmark line)")
    ap.add_argument("--minimal", action="store_true", help="timed solves only (no e2e, variants, CPU baseline)")
    ap.add_argument("--no-autotune", action="store_true", help="3D: keep the default kernel variant")
    ap.add_argument("--variant", default="", metavar="CH,NMB",
                    help="3D: take this variant of the tiled inner sweeps (rows per chunk, tiles per CTA) "
                    "instead of autotuning")
    ap.add_argument("--batch-count", type=int, default=512, help="problems of --workload batch2d")
    ap.add_argument("--workload", default="3d", choices=["2d_large", "3d", "batch2d", "serve3d"],
                    help="3d: the 512^3 workload (the bench line); 2d_large: the 8192 x 4096 workload; "
                    "batch2d: 512 independent 2D "
                    "problems in one graph launch; serve3d: a Poisson stream of 3D requests through "
                    "helm_server (measurements, not the bench line)")
    ap.add_argument("--serve-count", type=int, default=32, help="requests of --workload serve3d")
    ap.add_argument("--serve-rate", type=float, default=4.0,
                    help="mean arrivals per second (serve3d); <= 0: all requests at once (capacity)")
    ap.add_argument("--serve-slots", type=int, default=4, help="server streams (serve3d)")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0, help="plan-cache device budget (serve3d)")
    ap.add_argument("--path", default="c64_refined", choices=list(PATHS_NAMES),
                    help="path timed as the main line (the others are reported as variants)")
    ap.add_argument("--summarize-launches", default="", metavar="CSV",
                    help="print the per-kernel table of an ncu launch list and exit (no GPU needed)")
    args = ap.parse_args()
    if args.summarize_launches:
        summarize_launches(args.summarize_launches)
        return
    if args.minimal:
        args.no_e2e = args.no_variants = args.no_cpu_baseline = True
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        if args.steps > 3:
            args.steps = 3
        args.warmup = min(args.warmup, 1)
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
