"""Python binding of libhelm (include/helm.h): a GB300 (sm_103a) fast direct
solver for the FEM Helmholtz problem with first-order absorbing boundaries
(Toivanen & Wolfmayr, arXiv 1809.03808).

Argument marshalling only: every step of a solve runs in the CUDA kernels of
libhelm.so.  Device buffers are torch tensors (complex128 / complex64, C
contiguous, on the current CUDA device); their data pointers and the current
torch CUDA stream are passed through the C ABI.  If the library has not been
built this module raises ImportError -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhelm.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libhelm.so not found at {_LIB_PATH}; run __graft_entry__.build() "
                      "(or python -m paper_1809_03808_gb300._build)")

lib = ctypes.CDLL(_LIB_PATH)

HELM_C128, HELM_C64_REFINED, HELM_C64_RAW = 0, 1, 2
HELM_RESID_FP64, HELM_RESID_FF = 0, 1
HELM_BC_ABC, HELM_BC_NEUMANN = 0, 1
HELM_ELEMENT_Q1, HELM_ELEMENT_Q1_MODIFIED = 0, 1
HELM_VARIANT_INNER_CHUNK, HELM_VARIANT_INNER_TILES, HELM_VARIANT_TRI2D, HELM_VARIANT_DFT = 0, 1, 2, 3
HELM_OK, HELM_EINVAL, HELM_ENOMEM, HELM_ECUDA, HELM_ENOTCONV, HELM_ETIMEOUT, HELM_EUNSUPPORTED, HELM_ENUMERIC = \
    0, -1, -2, -3, -4, -5, -6, -7

_i64, _dbl, _vp, _i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int


class helm_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("residual", ctypes.c_double * 16), ("plan_seconds", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("n_dft_stages", ctypes.c_int32),
                ("device_bytes", ctypes.c_size_t), ("residual_kind", ctypes.c_int32),
                ("aux_q", ctypes.c_int32), ("aux_rho", ctypes.c_double), ("aux_trial_residual", ctypes.c_double),
                ("axis_bc", ctypes.c_int32 * 3), ("fp64_lines", ctypes.c_int32), ("element", ctypes.c_int32)]


class helm_plan_opts(ctypes.Structure):
    _fields_ = [("axis_bc", ctypes.c_int32 * 3), ("element", ctypes.c_int32)]


class helm_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int32), ("total_ms", ctypes.c_double)]


class helm_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double * 3),
                ("omega", ctypes.c_double), ("dtype", ctypes.c_int32), ("residual", ctypes.c_int32),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("f", ctypes.c_void_p), ("u", ctypes.c_void_p)]


class helm_request_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("plan_reused", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("residual", ctypes.c_double)]


class helm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("plans_built", ctypes.c_int64), ("plans_reused", ctypes.c_int64),
                ("plans_evicted", ctypes.c_int64), ("unknowns_solved", ctypes.c_double),
                ("elapsed_s", ctypes.c_double), ("latency_p50_s", ctypes.c_double),
                ("latency_p99_s", ctypes.c_double), ("latency_mean_s", ctypes.c_double),
                ("device_bytes_in_use", ctypes.c_size_t), ("device_bytes_peak", ctypes.c_size_t)]


_SIGS = {
    "helm_plan_2d": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _dbl, _dbl, _dbl, _i32]),
    "helm_plan_3d": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _i64, _dbl, _dbl, _dbl, _dbl, _i32]),
    "helm_plan_2d_bc": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _dbl, _dbl, _dbl, _i32, ctypes.POINTER(_i32)]),
    "helm_plan_2d_ex": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _dbl, _dbl, _dbl, _i32, _vp]),
    "helm_plan_3d_ex": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _i64, _dbl, _dbl, _dbl, _dbl, _i32, _vp]),
    "helm_plan_3d_bc": (_i32, [ctypes.POINTER(_vp), _i64, _i64, _i64, _dbl, _dbl, _dbl, _dbl, _i32,
                               ctypes.POINTER(_i32)]),
    "helm_set_precision_routing": (_i32, [_vp, _dbl]),
    "helm_set_variant": (_i32, [_vp, _i32, _i32]),
    "helm_get_variant": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
    "helm_time_solve": (_i32, [_vp, _i32, ctypes.POINTER(_dbl)]),
    "helm_set_stream": (_i32, [_vp, _vp]),
    "helm_set_refinement": (_i32, [_vp, _dbl, _i32]),
    "helm_set_auxiliary": (_i32, [_vp, _dbl, _i32]),
    "helm_set_residual": (_i32, [_vp, _i32]),
    "helm_set_graphs": (_i32, [_vp, _i32]),
    "helm_solve": (_i32, [_vp, _vp, _vp]),
    "helm_solve_host": (_i32, [_vp, _vp, _vp]),
    "helm_solve_many": (_i32, [_vp, _i64, _vp, _vp]),
    "helm_set_rhs_concurrency": (_i32, [_vp, _i32]),
    "helm_solve_debug": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "helm_get_info": (_i32, [_vp, ctypes.POINTER(helm_info)]),
    "helm_destroy": (_i32, [_vp]),
    "helm_status_string": (ctypes.c_char_p, [_i32]),
    "helm_last_error": (ctypes.c_char_p, [_vp]),
    "helm_abc_eigen": (_i32, [_i64, _dbl, _dbl, _vp, _vp, _vp]),
    "helm_dft_factor": (_i32, [_i64, _vp, _i32]),
    "helm_set_profiling": (_i32, [_vp, _i32]),
    "helm_solve_2d_static": (_i32, [_i64, _i64, _dbl, _dbl, _dbl, _vp, _vp, _vp]),
    "helm_get_profile": (_i32, [_vp, ctypes.POINTER(helm_profile_entry), _i32]),
    "helm_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp)]),
    "helm_batch_set_stream": (_i32, [_vp, _vp]),
    "helm_batch_solve": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "helm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "helm_batch_destroy": (_i32, [_vp]),
    "helm_server_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.c_size_t]),
    "helm_server_submit": (_i32, [_vp, ctypes.POINTER(helm_request), ctypes.POINTER(_i64)]),
    "helm_server_wait": (_i32, [_vp, _i64, _dbl, ctypes.POINTER(helm_request_result)]),
    "helm_server_drain": (_i32, [_vp, _dbl]),
    "helm_server_error": (ctypes.c_char_p, [_vp, _i64]),
    "helm_server_get_stats": (_i32, [_vp, ctypes.POINTER(helm_server_stats)]),
    "helm_server_destroy": (_i32, [_vp]),
    "helm_mlp_create": (_i32, [ctypes.POINTER(_vp), _i32, _i32, ctypes.c_uint64]),
    "helm_mlp_num_params": (_i32, [_vp]),
    "helm_mlp_get_params": (_i32, [_vp, _vp, _i32]),
    "helm_mlp_set_params": (_i32, [_vp, _vp, _i32]),
    "helm_mlp_forward": (_i32, [_vp, _vp, _i64, _vp]),
    "helm_mlp_gradient": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "helm_mlp_train": (_i32, [_vp, _vp, _vp, _i64, _i32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "helm_mlp_destroy": (_i32, [_vp]),
    "helm_debug_fail_alloc": (_i32, [_i32]),
    "helm_debug_live_allocations": (_i64, [ctypes.POINTER(ctypes.c_size_t)]),
    "helm_debug_wait_timeout": (_i32, [_vp, _i64]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class HelmError(RuntimeError):
    def __init__(self, status, where, detail=""):
        msg = f"{where}: {lib.helm_status_string(status).decode()}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)
        self.status = status


def _check(status, where, plan=None):
    if status != HELM_OK:
        detail = lib.helm_last_error(plan).decode() if plan else ""
        raise HelmError(status, where, detail)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# ---- names of the C ABI (marshalling only) ---------------------------------

def helm_plan_2d(nx, ny, hx, hy, omega, dtype=HELM_C128):
    h = _vp()
    _check(lib.helm_plan_2d(ctypes.byref(h), int(nx), int(ny), float(hx), float(hy), float(omega), int(dtype)),
           "helm_plan_2d")
    return h


def helm_plan_3d(nx, ny, nz, hx, hy, hz, omega, dtype=HELM_C128):
    h = _vp()
    _check(lib.helm_plan_3d(ctypes.byref(h), int(nx), int(ny), int(nz), float(hx), float(hy), float(hz),
                            float(omega), int(dtype)), "helm_plan_3d")
    return h


def helm_plan_2d_bc(nx, ny, hx, hy, omega, dtype, axis_bc):
    h = _vp()
    bc = (_i32 * 2)(*[int(b) for b in axis_bc])
    _check(lib.helm_plan_2d_bc(ctypes.byref(h), int(nx), int(ny), float(hx), float(hy), float(omega), int(dtype), bc),
           "helm_plan_2d_bc")
    return h


def plan_opts(axis_bc=None, element=HELM_ELEMENT_Q1):
    """helm_plan_opts: per-axis helm_bc values (default absorbing) and the
    element."""
    o = helm_plan_opts()
    for k, b in enumerate(axis_bc or ()):
        o.axis_bc[k] = int(b)
    o.element = int(element)
    return o


def helm_plan_2d_ex(nx, ny, hx, hy, omega, dtype, opts):
    h = _vp()
    _check(lib.helm_plan_2d_ex(ctypes.byref(h), int(nx), int(ny), float(hx), float(hy), float(omega), int(dtype),
                               ctypes.byref(opts)), "helm_plan_2d_ex")
    return h


def helm_plan_3d_ex(nx, ny, nz, hx, hy, hz, omega, dtype, opts):
    h = _vp()
    _check(lib.helm_plan_3d_ex(ctypes.byref(h), int(nx), int(ny), int(nz), float(hx), float(hy), float(hz),
                               float(omega), int(dtype), ctypes.byref(opts)), "helm_plan_3d_ex")
    return h


def helm_plan_3d_bc(nx, ny, nz, hx, hy, hz, omega, dtype, axis_bc):
    h = _vp()
    bc = (_i32 * 3)(*[int(b) for b in axis_bc])
    _check(lib.helm_plan_3d_bc(ctypes.byref(h), int(nx), int(ny), int(nz), float(hx), float(hy), float(hz),
                               float(omega), int(dtype), bc), "helm_plan_3d_bc")
    return h


def helm_set_precision_routing(plan, tau):
    _check(lib.helm_set_precision_routing(plan, float(tau)), "helm_set_precision_routing", plan)


def helm_set_variant(plan, knob, value):
    _check(lib.helm_set_variant(plan, int(knob), int(value)), "helm_set_variant", plan)


def helm_get_variant(plan, knob):
    v = _i32(0)
    _check(lib.helm_get_variant(plan, int(knob), ctypes.byref(v)), "helm_get_variant", plan)
    return int(v.value)


def helm_time_solve(plan, reps=3):
    ms = _dbl(0.0)
    _check(lib.helm_time_solve(plan, int(reps), ctypes.byref(ms)), "helm_time_solve", plan)
    return float(ms.value)


def helm_set_stream(plan, stream):
    _check(lib.helm_set_stream(plan, _vp(int(stream) if stream is not None else 0)), "helm_set_stream", plan)


def helm_set_auxiliary(plan, rho, phase_quarters):
    _check(lib.helm_set_auxiliary(plan, float(rho), int(phase_quarters)), "helm_set_auxiliary", plan)


def helm_set_refinement(plan, tol, max_iter):
    _check(lib.helm_set_refinement(plan, float(tol), int(max_iter)), "helm_set_refinement", plan)


def helm_set_residual(plan, kind):
    _check(lib.helm_set_residual(plan, int(kind)), "helm_set_residual", plan)


def helm_set_graphs(plan, enable):
    _check(lib.helm_set_graphs(plan, int(bool(enable))), "helm_set_graphs", plan)


def helm_solve(plan, f, u):
    _check(lib.helm_solve(plan, _ptr(f), _ptr(u)), "helm_solve", plan)


def helm_solve_many(plan, nrhs, f, u):
    _check(lib.helm_solve_many(plan, int(nrhs), _ptr(f), _ptr(u)), "helm_solve_many", plan)


def helm_set_rhs_concurrency(plan, k):
    _check(lib.helm_set_rhs_concurrency(plan, int(k)), "helm_set_rhs_concurrency", plan)


def helm_solve_host(plan, f, u):
    """f, u: host buffers (numpy arrays or pinned torch CPU tensors)."""
    fp = f.ctypes.data if hasattr(f, "ctypes") else _ptr(f)
    up = u.ctypes.data if hasattr(u, "ctypes") else _ptr(u)
    _check(lib.helm_solve_host(plan, fp, up), "helm_solve_host", plan)


def helm_solve_debug(plan, f, u, fhat=None, v_b=None, w_b=None):
    _check(lib.helm_solve_debug(plan, _ptr(f), _ptr(u), _ptr(fhat), _ptr(v_b), _ptr(w_b)), "helm_solve_debug", plan)


def helm_get_info(plan):
    info = helm_info()
    st = lib.helm_get_info(plan, ctypes.byref(info))
    if st not in (HELM_OK, HELM_ENOTCONV):
        _check(st, "helm_get_info", plan)
    return info, st


def helm_set_profiling(plan, enable):
    _check(lib.helm_set_profiling(plan, int(bool(enable))), "helm_set_profiling", plan)


def helm_get_profile(plan):
    """{kernel name: (launches, total device ms)} since the last call."""
    buf = (helm_profile_entry * 64)()
    k = lib.helm_get_profile(plan, buf, 64)
    if k < 0:
        _check(k, "helm_get_profile", plan)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(k)}


def helm_solve_2d_static(nx, ny, hx, hy, omega, f, u, stream=None):
    """Allocation-free complex128 2D solve (no plan): f, u device buffers."""
    st = lib.helm_solve_2d_static(int(nx), int(ny), float(hx), float(hy), float(omega), _ptr(f), _ptr(u),
                                  _vp(int(stream) if stream is not None else 0))
    _check(st, "helm_solve_2d_static")


def helm_destroy(plan):
    _check(lib.helm_destroy(plan), "helm_destroy")


def helm_abc_eigen(n, h, omega):
    """Host-side eigen-data of the absorbing 1D pencil: (lam, sigma, parity) numpy arrays."""
    import numpy as np
    lam = np.zeros(2 * n)
    sig = np.zeros(2 * n)
    par = np.zeros(n, dtype=np.int8)
    _check(lib.helm_abc_eigen(int(n), float(h), float(omega), lam.ctypes.data, sig.ctypes.data, par.ctypes.data),
           "helm_abc_eigen")
    return lam[0::2] + 1j * lam[1::2], sig[0::2] + 1j * sig[1::2], par.astype(np.int64)


def helm_dft_factor(n):
    import numpy as np
    r = np.zeros(32, dtype=np.int32)
    ns = lib.helm_dft_factor(int(n), r.ctypes.data, 32)
    return [int(x) for x in r[:ns]]


# ---- convenience wrapper ----------------------------------------------------

class Plan:
    """Owns one helm plan; solve(f, u) on torch CUDA tensors, current stream."""

    def __init__(self, shape, h, omega, dtype=HELM_C128, bc=None, element=HELM_ELEMENT_Q1):
        """bc: None (absorbing faces everywhere) or one HELM_BC_* (or "abc" /
        "neumann") per axis; element: HELM_ELEMENT_Q1 (or "q1") or
        HELM_ELEMENT_Q1_MODIFIED (or "q1mod")."""
        shape = tuple(int(n) for n in shape)
        self.shape = shape
        self.dtype = dtype
        if bc is not None:
            bc = [HELM_BC_NEUMANN if b in ("neumann", HELM_BC_NEUMANN) else HELM_BC_ABC for b in bc]
        element = {"q1": HELM_ELEMENT_Q1, "q1mod": HELM_ELEMENT_Q1_MODIFIED}.get(element, element)
        if len(shape) not in (2, 3):
            raise ValueError("shape must be 2D or 3D")
        if element != HELM_ELEMENT_Q1:
            opts = plan_opts(bc, element)
            self.handle = (helm_plan_2d_ex(shape[0], shape[1], h[0], h[1], omega, dtype, opts) if len(shape) == 2
                           else helm_plan_3d_ex(shape[0], shape[1], shape[2], h[0], h[1], h[2], omega, dtype, opts))
        elif len(shape) == 2:
            self.handle = (helm_plan_2d(shape[0], shape[1], h[0], h[1], omega, dtype) if bc is None else
                           helm_plan_2d_bc(shape[0], shape[1], h[0], h[1], omega, dtype, bc))
        elif len(shape) == 3:
            self.handle = (helm_plan_3d(shape[0], shape[1], shape[2], h[0], h[1], h[2], omega, dtype) if bc is None
                           else helm_plan_3d_bc(shape[0], shape[1], shape[2], h[0], h[1], h[2], omega, dtype, bc))
        else:
            raise ValueError("shape must be 2D or 3D")

    @property
    def tensor_dtype(self):
        import torch
        return torch.complex64 if self.dtype == HELM_C64_RAW else torch.complex128

    def _check_tensor(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.tensor_dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.tensor_dtype} tensor of shape {self.shape}")

    def solve(self, f, u=None, stream=None):
        import torch
        self._check_tensor(f, "f")
        if u is None:
            u = torch.empty_like(f)
        self._check_tensor(u, "u")
        s = torch.cuda.current_stream(f.device) if stream is None else stream
        helm_set_stream(self.handle, s.cuda_stream)
        helm_solve(self.handle, f, u)
        return u

    def info(self):
        return helm_get_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            helm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Plans solved together as one CUDA graph launch (helm_batch_*).

    solve(fs, us) takes lists of CUDA tensors, one pair per plan, laid out as
    for Plan.solve; the current torch stream is used."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (_vp * len(self.plans))(*[p.handle for p in self.plans])
        h = _vp()
        st = lib.helm_batch_create(ctypes.byref(h), len(self.plans), arr)
        if st != HELM_OK:
            raise HelmError(st, "helm_batch_create")
        self.handle = h

    def solve(self, fs, us, stream=None):
        import torch
        if len(fs) != len(self.plans) or len(us) != len(self.plans):
            raise ValueError("one f and one u per plan")
        for p, f, u in zip(self.plans, fs, us):
            p._check_tensor(f, "f")
            p._check_tensor(u, "u")
        s = torch.cuda.current_stream(fs[0].device) if stream is None else stream
        lib.helm_batch_set_stream(self.handle, _vp(s.cuda_stream))
        fa = (_vp * len(fs))(*[f.data_ptr() for f in fs])
        ua = (_vp * len(us))(*[u.data_ptr() for u in us])
        st = lib.helm_batch_solve(self.handle, fa, ua)
        if st != HELM_OK:
            raise HelmError(st, "helm_batch_solve", lib.helm_batch_last_error(self.handle).decode())
        return us

    def close(self):
        if getattr(self, "handle", None):
            lib.helm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A request server (helm_server_*): plan cache under a device-memory
    budget, `nslots` CUDA streams, a scheduler thread and a plan-builder
    thread.

    submit() takes CUDA tensors f and u holding nrhs right-hand sides one
    after another (shape (nrhs, *shape) or the plan layout when nrhs = 1);
    they must stay alive until wait() reports the request done."""

    def __init__(self, nslots=4, device_budget_bytes=64 << 30):
        h = _vp()
        st = lib.helm_server_create(ctypes.byref(h), int(nslots), int(device_budget_bytes))
        if st != HELM_OK:
            raise HelmError(st, "helm_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, shape, h, omega, f, u, dtype=HELM_C64_REFINED, residual=HELM_RESID_FF, tol=1e-12,
               max_iter=10, nrhs=1):
        r = helm_request()
        r.dim = len(shape)
        for k, n in enumerate(shape):
            r.n[k] = int(n)
            r.h[k] = float(h[k])
        r.omega = float(omega)
        r.dtype, r.residual, r.tol, r.max_iter, r.nrhs = int(dtype), int(residual), float(tol), int(max_iter), int(nrhs)
        r.f, r.u = _ptr(f), _ptr(u)
        t = _i64()
        st = lib.helm_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        if st != HELM_OK:
            raise HelmError(st, "helm_server_submit")
        self._keep[t.value] = (f, u)
        return t.value

    def wait(self, ticket, timeout_s=-1.0):
        res = helm_request_result()
        st = lib.helm_server_wait(self.handle, int(ticket), float(timeout_s), ctypes.byref(res))
        if st not in (HELM_OK, HELM_ETIMEOUT):
            raise HelmError(st, "helm_server_wait")
        if res.done:
            self._keep.pop(int(ticket), None)
        return res

    def error(self, ticket):
        """What failed for a request that did not complete ("" otherwise)."""
        return lib.helm_server_error(self.handle, int(ticket)).decode()

    def drain(self, timeout_s=-1.0):
        st = lib.helm_server_drain(self.handle, float(timeout_s))
        if st != HELM_OK:
            raise HelmError(st, "helm_server_drain")

    def stats(self):
        st = helm_server_stats()
        _check(lib.helm_server_get_stats(self.handle, ctypes.byref(st)), "helm_server_get_stats")
        return st

    def close(self):
        if getattr(self, "handle", None):
            lib.helm_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
