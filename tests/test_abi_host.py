"""The C-ABI library loads, exports every symbol include/rkl.h declares, and
its host-only logic (stage count, Appendix A coefficients, argument checks)
agrees with the oracle.  No GPU: nothing here launches a kernel."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1702_05487_gb300 import _lib
    return _lib


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(rkl_[A-Za-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lib):
    so = lib.load()
    declared = _declared_symbols()
    assert "rkl_super_step" in declared and "rkl_stage" in declared
    for name in sorted(declared):
        assert hasattr(so, name), f"{name} declared in include/ but not exported"
    # the binding covers the same set
    assert declared == set(lib.SIGNATURES), declared ^ set(lib.SIGNATURES)


def test_status_strings(lib):
    assert lib.status_name(0) == "RKL_OK"
    assert lib.status_name(lib.RKL_ERR_NONFINITE) == "RKL_ERR_NONFINITE"


@pytest.mark.parametrize("ratio", [0.01, 1.0, 2.5, 7.0, 20, 50, 100, 200, 400, 1234.5])
def test_num_stages_matches_oracle(lib, orc, ratio):
    assert lib.rkl_num_stages(ratio) == orc.num_stages(ratio)


@pytest.mark.parametrize("s", [2, 3, 9, 20, 40, 400])
def test_coeffs_match_oracle(lib, orc, s):
    got = lib.rkl_coeffs(s)
    want = orc.coeffs(s)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("ratio", [0.3, 1.0, 2.9, 20, 50, 100, 400, 1234.5])
def test_first_order_stage_counts_match_oracle(lib, orc, ratio):
    assert lib.rkl_num_stages_method(lib.RKL_METHOD_RKL2, ratio) == orc.num_stages(ratio)
    assert lib.rkl_num_stages_method(lib.RKL_METHOD_RKL1, ratio) == orc.num_stages_rkl1(ratio)
    for nu in (1e-3, 1e-2, 0.2):
        assert lib.rkl_num_stages_method(lib.RKL_METHOD_STS, ratio, nu) == orc.num_stages_sts(ratio, nu)


@pytest.mark.parametrize("s", [1, 2, 5, 14, 40])
def test_first_order_coefficients(lib, orc, s):
    """RKL1: the Legendre recursion (mu_j = (2j-1)/j, nu_j = -(j-1)/j,
    mut_j = mu_j w1, mut_1 = w1, gt = 0); AAG-STS: mu = 1, nu = 0, gt = 0 and
    mut_j = the oracle's sub-steps of a unit super-step."""
    mu, nu, mut, gt = lib.rkl_coeffs_method(lib.RKL_METHOD_RKL1, s)
    w1 = 2.0 / (s * s + s)
    j = np.arange(2, s + 1)
    assert abs(mut[1] - w1) < 1e-16
    assert np.allclose(mu[2:], (2 * j - 1) / j, rtol=1e-15, atol=0)
    assert np.allclose(nu[2:], -(j - 1) / j, rtol=1e-15, atol=0)
    assert np.allclose(mut[2:], (2 * j - 1) / j * w1, rtol=1e-15, atol=0)
    assert not np.any(gt)
    for nuv in (1e-3, 0.05):
        mu, nu, mut, gt = lib.rkl_coeffs_method(lib.RKL_METHOD_STS, s, nuv)
        assert np.all(mu[2:] == 1.0) and not np.any(nu) and not np.any(gt)
        assert np.allclose(mut[1:], orc.sts_substeps(s, nuv, 1.0), rtol=1e-13, atol=0)
    if s >= 2:
        assert all(np.array_equal(a, b) for a, b in zip(lib.rkl_coeffs_method(lib.RKL_METHOD_RKL2, s),
                                                         orc.coeffs(s)))


def test_method_argument_checks(lib):
    so = lib.load()
    s = ctypes.c_int(0)
    assert so.rkl_num_stages_method(7, 10.0, 1e-3, ctypes.byref(s)) == lib.RKL_ERR_INVALID_ARG
    for nu in (0.0, 1.0, -0.1, float("nan")):
        assert so.rkl_num_stages_method(lib.RKL_METHOD_STS, 10.0, nu, ctypes.byref(s)) == lib.RKL_ERR_INVALID_ARG
    assert so.rkl_num_stages_method(lib.RKL_METHOD_STS, 1e12, 1e-3, ctypes.byref(s)) == lib.RKL_ERR_INVALID_ARG
    arr = np.zeros(5)
    p = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert so.rkl_coeffs_method(lib.RKL_METHOD_RKL2, 1, 1e-3, p, p, p, p) == lib.RKL_ERR_INVALID_ARG
    assert so.rkl_coeffs_method(lib.RKL_METHOD_RKL1, 0, 1e-3, p, p, p, p) == lib.RKL_ERR_INVALID_ARG


def test_host_argument_checks(lib):
    so = lib.load()
    s = ctypes.c_int(0)
    for bad in (0.0, -1.0, float("nan"), float("inf"), 1e9):
        assert so.rkl_num_stages(bad, ctypes.byref(s)) == lib.RKL_ERR_INVALID_ARG
    arr = np.zeros(5)
    p = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert so.rkl_coeffs(1, p, p, p, p) == lib.RKL_ERR_INVALID_ARG
    assert so.rkl_coeffs(4097, p, p, p, p) == lib.RKL_ERR_INVALID_ARG
    assert so.rkl_coeffs(3, None, p, p, p) == lib.RKL_ERR_INVALID_ARG


def test_plan_create_rejects_bad_arguments_before_any_cuda_call(lib):
    from paper_1702_05487_gb300 import make_grid, make_phys
    good_g, good_p = make_grid((4, 4, 4)), make_phys()
    cases = []
    g = make_grid((4, 4, 4)); g.ndim = 4; cases.append((g, good_p))
    g = make_grid((4, 4)); g.n[2] = 3; cases.append((g, good_p))
    g = make_grid((4, 4, 4)); g.dx[1] = -1.0; cases.append((g, good_p))
    g = make_grid((4, 4, 4)); g.bc = 7; cases.append((g, good_p))
    g = make_grid((4, 4, 4)); g.dtype = 5; cases.append((g, good_p))
    p = make_phys(); p.kappa_par0 = 0.0; cases.append((good_g, p))
    p = make_phys(); p.cp = 0.7; cases.append((good_g, p))
    p = make_phys(saturate=True, phi=0.0); cases.append((good_g, p))
    for g, p in cases:
        with pytest.raises(lib.RklError) as ei:
            lib.rkl_plan_create(g, p)
        assert ei.value.status == lib.RKL_ERR_INVALID_ARG
