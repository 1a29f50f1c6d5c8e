"""Operator splitting on the GPU (Section 3): donor-cell advection, Eq. dt_h
and the split driver's three conduction strategies against the FP64 oracle,
element by element."""
import math

import numpy as np
import pytest

import workloads
from gpu_util import F32_STATE_MAX, F32_STATE_REL_L2, F64_TOL, host, norm_max, rel_l2, rounded, torch_dev
from oracle import Problem

pytestmark = pytest.mark.gpu

SPITZ = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


def _abc(shape, scale):
    nz, ny, nx = shape
    cx = 2 * math.pi * (np.arange(nx) + 0.5) / nx
    cy = 2 * math.pi * (np.arange(ny) + 0.5) / ny
    cz = 2 * math.pi * (np.arange(nz) + 0.5) / nz
    z, y, x = np.meshgrid(cz, cy, cx, indexing="ij")
    return scale * np.stack([np.sin(z) + np.cos(y), np.sin(x) + np.cos(z), np.sin(y) + np.cos(x)])


def _fields(shape, seed=31):
    nz, ny, nx = shape
    return workloads.tangled_box(nx, ny, nz, seed)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_advect_and_dt_hyp(rk, orc, dtype):
    import torch
    shape = (20, 24, 36)
    T, _ = _fields(shape)
    u = _abc(shape, 0.7)
    T, u = rounded(T, dtype), rounded(u, dtype)
    P = Problem(shape, **SPITZ)
    plan = rk.Plan(shape, dtype, params=SPITZ)
    Td, ud = torch_dev(T, dtype), torch_dev(u, dtype)
    dt = plan.dt_hyperbolic(ud, 0.8)
    want = orc.dt_hyp(P, u, 0.8)
    assert dt == pytest.approx(want, rel=1e-6 if dtype == "f32" else 1e-14)
    out = torch.empty_like(Td)
    plan.advect(want, ud, Td, out)
    ref = orc.advect(P, T, u, want)
    tol = 2e-6 if dtype == "f32" else 1e-14
    assert norm_max(host(out), ref) < tol


def test_advect_dirichlet_2d_fp64(rk, orc):
    import torch
    W = workloads.ring(40)
    n = 40
    c = -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    y, x = np.meshgrid(c, c, indexing="ij")
    u = np.stack([-y, x])                      # solid rotation, ghosts copy the edge
    P = Problem(W.T.shape, **W.params)
    plan = rk.Plan(W.T.shape, "f64", params=W.params)
    Td, ud = torch_dev(W.T, "f64"), torch_dev(u, "f64")
    dt = orc.dt_hyp(P, u, 0.9)
    out = torch.empty_like(Td)
    plan.advect(dt, ud, Td, out)
    assert norm_max(host(out), orc.advect(P, W.T, u, dt)) < 1e-14


@pytest.mark.parametrize("strategy", ["rkl2", "subcycle", "explicit"])
def test_split_driver_strategies(rk, orc, strategy):
    import torch
    from paper_1702_05487_gb300.split import SplitDriver
    shape = (24, 20, 32)
    T, b = _fields(shape)
    u = _abc(shape, 0.05)
    T, b, u = rounded(T), rounded(b), rounded(u)
    P = Problem(shape, **SPITZ)
    drv = SplitDriver(shape, "f32", params=SPITZ, ch=0.8, strategy=strategy)
    Ta, bd, ud = torch_dev(T), torch_dev(b), torch_dev(u)
    Tb = torch.empty_like(Ta)
    e0 = orc.energy(P, T)
    ref = T.copy()
    cur, oth = Ta, Tb
    for _ in range(2):
        dth = orc.dt_hyp(P, u, 0.8)
        if strategy == "rkl2":
            new, dt, s = drv.step(cur, oth, bd, ud, dth)
            ref, dref, sref = orc.split_step(P, ref, b, u, 0.8)
            assert s == sref
        elif strategy == "subcycle":
            new, dt, n = drv.step(cur, oth, bd, ud, dth)
            ref, dref, nref = orc.split_step(P, ref, b, u, 0.8, conduction="subcycle", sub=n)
        else:
            n = 6
            new, dt, _ = drv.step(cur, oth, bd, ud, dth, n)
            for _ in range(n):
                ref = orc.euler_step(P, orc.advect(P, ref, u, dth / n), b, dth / n)
        oth = cur if new is not cur else oth
        cur = new
    got = host(cur)
    assert rel_l2(got, ref) < F32_STATE_REL_L2
    assert norm_max(got, ref) < F32_STATE_MAX
    assert abs(orc.energy(P, got) - e0) < 1e-6 * abs(e0)
    drv.close()
