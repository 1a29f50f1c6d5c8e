"""The first-order super-time-steppers of Section 3.3 (RKL1, AAG-STS) on the
GPU, through the same stage kernels as RKL2, against the oracle's own
RKL1 and AAG-STS super-steps, element by element.  Includes the single-stage
case (s = 1, a forward-Euler step that lands in the caller's array) and the
stage-by-stage entry point with the plan's method."""
import numpy as np
import pytest

from gpu_util import F32_STATE_MAX, F32_STATE_REL_L2, F64_TOL, host, norm_max, rel_l2, rounded, torch_dev
from oracle import Problem
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


SPITZ = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
CASES = [
    ("3d_f32_x2", (24, 20, 64), SPITZ, "f32"),
    ("3d_f32_ragged", (13, 22, 30), SPITZ, "f32"),
    ("3d_f64", (11, 12, 13), SPITZ, "f64"),
    ("2d_f64_dirichlet", (33, 27), dict(kappa_par0=0.05, bc="dirichlet", bc_value=1.0), "f64"),
]


def _fields(shape, seed=23):
    if len(shape) == 3:
        nz, ny, nx = shape
        return workloads.tangled_box(nx, ny, nz, seed)
    ny, nx = shape
    T, b = workloads.tangled_box(nx, ny, 4, seed)
    b = b[:2, 0]
    return T[0], b / np.sqrt((b ** 2).sum(0))


def _oracle_step(orc, method, P, T, b, dt, nu):
    if method == "rkl1":
        return orc.rkl1_super_step(P, T, b, dt)
    return orc.sts_super_step(P, T, b, dt, nu)


@pytest.mark.parametrize("method,nu", [("rkl1", 0.0), ("sts", 1e-3), ("sts", 0.05)])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_first_order_super_steps(rk, orc, case, method, nu):
    name, shape, params, dtype = case
    T, b = _fields(shape)
    T, b = rounded(T, dtype), rounded(b, dtype)
    P = Problem(shape, **params)
    plan = rk.Plan(shape, dtype, params=params)
    plan.set_method(method, nu if nu > 0 else 1e-3)
    Td, bd = torch_dev(T, dtype), torch_dev(b, dtype)
    dt = 30.0 * orc.dt_expl(P, T)
    Tref = T.copy()
    periodic = params.get("bc", "periodic") == "periodic"
    for _ in range(2):
        s, eb, ea = plan.super_step(dt, Td, bd, energies=True)
        Tref, sref = _oracle_step(orc, method, P, Tref, b, dt, nu)
        assert s == sref
        if periodic:
            assert abs(ea - eb) <= (1e-12 if dtype == "f64" else 1e-6) * abs(eb)
    Tg = host(Td)
    if dtype == "f64":
        assert norm_max(Tg, Tref) < F64_TOL
    else:
        assert rel_l2(Tg, Tref) < F32_STATE_REL_L2
        assert norm_max(Tg, Tref) < F32_STATE_MAX
    assert plan.check() == 0


@pytest.mark.parametrize("method", ["rkl1", "sts"])
def test_single_stage_lands_in_caller_array(rk, orc, method):
    """dt below the explicit limit gives s = 1: one Euler step into T."""
    shape, dtype = (16, 16, 32), "f32"
    T, b = _fields(shape)
    T, b = rounded(T, dtype), rounded(b, dtype)
    P = Problem(shape, **SPITZ)
    plan = rk.Plan(shape, dtype, params=SPITZ)
    plan.set_method(method)
    Td, bd = torch_dev(T, dtype), torch_dev(b, dtype)
    dt = 0.4 * orc.dt_expl(P, T)
    s = plan.super_step(dt, Td, bd)
    Tref, sref = _oracle_step(orc, method, P, T, b, dt, 1e-3)
    assert s == sref == 1
    assert rel_l2(host(Td), Tref) < F32_STATE_REL_L2


def test_stage_entry_uses_plan_method(rk, orc):
    """rkl_stage with RKL1 coefficients, stage by stage, equals the oracle's
    RKL1 super-step (FP64, so to rounding)."""
    import torch
    shape, dtype = (10, 12, 14), "f64"
    T, b = _fields(shape)
    P = Problem(shape, **SPITZ)
    plan = rk.Plan(shape, dtype, params=SPITZ)
    plan.set_method("rkl1")
    dt = 12.0 * orc.dt_expl(P, T)
    s = orc.num_stages_rkl1(12.0)
    Td, bd = torch_dev(T, dtype), torch_dev(b, dtype)
    Y = [Td, torch.empty_like(Td), torch.empty_like(Td), torch.empty_like(Td)]
    MY0 = torch.empty_like(Td)
    plan.stage(1, s, dt, bd, Td, MY0, None, None, Y[1])
    jm2, jm1 = 0, 1
    for j in range(2, s + 1):
        out = next(k for k in (1, 2, 3) if k not in (jm1, jm2))
        plan.stage(j, s, dt, bd, Td, MY0, Y[jm1], Y[jm2], Y[out])
        jm2, jm1 = jm1, out
    Tref, _ = orc.rkl1_super_step(P, T, b, dt, s)
    assert norm_max(host(Y[jm1]), Tref) < F64_TOL
