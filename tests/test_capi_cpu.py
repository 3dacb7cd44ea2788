"""C-ABI library checks that need no GPU: it loads, exports every symbol the
header declares, validates arguments, and its host-side plan logic (the
absorbing-pencil eigen-data of eqs. EVP1a / EVPcondA, the DFT factorisation)
agrees with the oracle."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def helm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1809_03808_gb300 as h

    return h


def test_every_header_symbol_is_exported(helm):
    hdr = open(os.path.join(ROOT, "include", "helm.h")).read()
    names = set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(helm_\w+)\s*\(", hdr, flags=re.M))
    assert len(names) >= 12
    for n in names:
        assert hasattr(helm.lib, n), n
    assert names == set(helm.EXPORTED)


def test_status_strings(helm):
    for s in range(-7, 1):
        assert helm.lib.helm_status_string(s).decode().startswith("HELM_")


@pytest.mark.parametrize("args", [(2, 5, 0.1, 0.1, 1.0, 0), (5, 5, 0.0, 0.1, 1.0, 0), (5, 5, 0.1, 0.1, -1.0, 0),
                                  (5, 5, 0.1, float("nan"), 1.0, 0), (5, 5, 0.1, 0.1, 1.0, 7)])
def test_plan_rejects_bad_arguments_before_touching_the_device(helm, args):
    import ctypes

    h = ctypes.c_void_p(1234)
    st = helm.lib.helm_plan_2d(ctypes.byref(h), *args)
    assert st == helm.HELM_EINVAL
    assert h.value is None


def test_null_plan_and_destroy_null(helm):
    assert helm.lib.helm_destroy(None) == helm.HELM_OK
    assert helm.lib.helm_solve(None, None, None) == helm.HELM_EINVAL
    assert helm.lib.helm_set_refinement(None, 1e-12, 3) == helm.HELM_EINVAL
    assert helm.lib.helm_set_residual(None, helm.HELM_RESID_FF) == helm.HELM_EINVAL


@pytest.mark.parametrize("n", [4, 9, 64, 129, 512, 1000, 1021, 4096, 8192, 6 * 49])
def test_dft_factorisation(helm, n):
    r = helm.helm_dft_factor(n)
    assert int(np.prod(r)) == n
    assert all(x >= 2 for x in r)


@pytest.mark.parametrize("n,h,ppw", [(17, 1 / 16, 6), (129, 1 / 128, 16), (257, 1 / 256, 10), (300, 0.003, 8)])
def test_abc_eigen_matches_dense_oracle(helm, n, h, ppw):
    from oracle import solvers

    omega = 2 * np.pi / (ppw * h)
    lam, sig, par = helm.helm_abc_eigen(n, h, omega)
    lo, V = solvers.abc_pencil_eig(n, h, omega)
    scale = np.abs(lo).max()
    # same spectrum (as a set)
    for i, l in enumerate(lam):
        j = int(np.argmin(np.abs(lo - l)))
        assert abs(lo[j] - l) <= 1e-9 * scale
        # sigma = V[1,l]^2 and parity = V[n,l]/V[1,l] for the matching eigenvector
        assert abs(V[0, j] ** 2 - sig[i]) <= 1e-7 * abs(sig[i])
        assert abs(V[-1, j] - par[i] * V[0, j]) <= 1e-6 * abs(V[0, j])
    assert len(np.unique(np.round(lam, 6))) == n


def test_abc_eigen_rejects_bad_input(helm):
    with pytest.raises(helm.HelmError):
        helm.helm_abc_eigen(1, 0.1, 1.0)
    with pytest.raises(helm.HelmError):
        helm.helm_abc_eigen(10, 0.1, -1.0)
    with pytest.raises(helm.HelmError):
        helm.helm_abc_eigen(10, 0.0, 1.0)


@pytest.mark.parametrize("n,h", [(9, 0.125), (64, 1 / 63), (301, 0.002)])
def test_neumann_eigen_matches_dense_oracle(helm, n, h):
    """w = 0: the Neumann pencil of a Gamma_N axis (corner 1 of eq. matrixK),
    against the oracle's dense generalized eigen-decomposition."""
    from oracle import solvers

    lam, sig, par = helm.helm_abc_eigen(n, h, 0.0)
    lo, V = solvers.abc_pencil_eig(n, h, 5.0, "neumann")
    scale = np.abs(lo).max()
    assert np.abs(lam.imag).max() == 0 and np.abs(sig.imag).max() == 0
    for i, l in enumerate(lam):
        j = int(np.argmin(np.abs(lo - l)))
        assert abs(lo[j] - l) <= 1e-9 * scale
        assert abs(V[0, j] ** 2 - sig[i]) <= 1e-9 * abs(sig[i])
        assert abs(V[-1, j] - par[i] * V[0, j]) <= 1e-7 * abs(V[0, j])


def test_server_rejects_bad_arguments_before_touching_the_device(helm):
    """helm_server_*: argument checks that precede any CUDA call."""
    import ctypes

    h = ctypes.c_void_p(1)
    assert helm.lib.helm_server_create(None, 2, 1 << 30) == helm.HELM_EINVAL
    for nslots, budget in [(0, 1 << 30), (17, 1 << 30), (2, 0)]:
        assert helm.lib.helm_server_create(ctypes.byref(h), nslots, budget) == helm.HELM_EINVAL
        assert h.value is None
    t = ctypes.c_int64(5)
    req = helm.helm_request()
    assert helm.lib.helm_server_submit(None, ctypes.byref(req), ctypes.byref(t)) == helm.HELM_EINVAL
    assert helm.lib.helm_server_wait(None, 1, 0.0, None) == helm.HELM_EINVAL
    assert helm.lib.helm_server_drain(None, 0.0) == helm.HELM_EINVAL
    assert helm.lib.helm_server_error(None, 1) == b""
    st = helm.helm_server_stats()
    assert helm.lib.helm_server_get_stats(None, ctypes.byref(st)) == helm.HELM_EINVAL
    assert helm.lib.helm_server_destroy(None) == helm.HELM_OK
