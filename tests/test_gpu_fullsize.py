"""The three single-problem workloads at their full sizes, in the launch
configuration the benchmark times (rkl_super_step with cached graphs).

* 2D ring, FP64, 100x100, 400 super-steps: the whole run against the oracle.
* 3D tangled field, FP32, 256^3: the first super-step checked cell by cell
  on sampled cells, each recomputed by the oracle on a periodic window of
  side 2(s + 2) around it (the stencil reaches one cell per stage, so the
  window's own wrap cannot reach the centre); then all 10 super-steps with
  FP64 energy conservation.
* 3D saturated blob, FP32, 512^3: the same sampled check of the first
  super-step, then all 20 super-steps with FP64 energy conservation.
* The 256^3 tangled field with MC-limited transverse gradients at every
  face (the paired-cell kernel's limited build): the same checks."""
import numpy as np
import pytest

import workloads
from gpu_util import F32_LIMITER_MAX, F32_STATE_MAX, host, rounded, torch_dev, window
from oracle import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


def test_ring_fp64_full_run(rk, orc):
    W = workloads.ring(100)
    P = Problem(W.T.shape, **W.params)
    plan = rk.Plan(W.T.shape, "f64", params=W.params)
    Td, bd = torch_dev(W.T, "f64"), torch_dev(W.b, "f64")
    dt = W.ratio * orc.dt_expl(P, W.T)
    Tref = W.T.copy()
    for _ in range(W.n_super):
        s = plan.super_step(dt, Td, bd)
        Tref, sref = orc.super_step(P, Tref, W.b, dt)
        assert s == sref == 14
    Tg = host(Td)
    assert np.max(np.abs(Tg - Tref)) < 1e-11 * np.max(np.abs(Tref))
    assert Tg.min() < 10.0          # the undershoot of arithmetic-mean transverse gradients
    assert plan.check() == 0


def _sampled_first_step(rk, orc, W, dtype, cells, variant=0, tol=F32_STATE_MAX):
    import torch
    P = Problem(W.T.shape, **W.params)
    T = rounded(W.T, dtype)
    b = rounded(W.b, dtype)
    plan = rk.Plan(W.T.shape, dtype, params=W.params)
    plan.set_variant(variant)
    Td, bd = torch_dev(T, dtype), torch_dev(b, dtype)
    e0 = orc.energy(P, T)
    dt = W.ratio * orc.dt_expl(P, T)
    s = plan.super_step(dt, Td, bd)
    assert s == orc.num_stages(W.ratio)
    torch.cuda.synchronize()
    T1 = host(Td)
    half = s + 2
    errs = []
    for c in cells:
        Tw = window(T, c, half)
        bw = window(b, c, half, axes_first=1)
        Pw = Problem(Tw.shape, **W.params)
        Tw1, _ = orc.super_step(Pw, Tw, bw, dt, s)
        ref = Tw1[half, half, half]
        errs.append(abs(T1[tuple(c)] - ref) / np.max(np.abs(T)))
    assert max(errs) < tol, errs
    return plan, Td, bd, dt, e0, P


@pytest.mark.parametrize("variant", [0, 5, 6, 7, 8, 9, 10, 11])
def test_tangled_256_sampled_and_conservation(rk, orc, variant):
    """The benchmark's 256^3 workload with the default single-stage kernel,
    the two-stage kernel (tile edges at multiples of 60 and 7) and the
    single-stage kernel with bulk copies."""
    W = workloads.tangled(256, seed=2)
    rng = np.random.default_rng(0)
    cells = [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(5)] + [(0, 0, 0), (255, 128, 7)]
    cells += [(31, 7, 60), (32, 13, 59), (255, 255, 240)]
    plan, Td, bd, dt, e0, P = _sampled_first_step(rk, orc, W, "f32", cells, variant)
    for _ in range(W.n_super - 1):
        s, eb, ea = plan.super_step(dt, Td, bd, energies=True)
        assert abs(ea - eb) <= 1e-6 * abs(eb)
    assert abs(plan.energy(Td) - e0) <= 1e-5 * abs(e0)
    assert plan.check() == 0


@pytest.mark.parametrize("variant", [0, 3, 10])
def test_blob_512_saturated_sampled_and_conservation(rk, orc, variant):
    W = workloads.blob(512, seed=2)
    rng = np.random.default_rng(1)
    cells = [(256, 256, 256), (256, 270, 240), (230, 256, 290)] + \
            [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(2)]
    plan, Td, bd, dt, e0, P = _sampled_first_step(rk, orc, W, "f32", cells, variant)
    for _ in range(W.n_super - 1):
        s, eb, ea = plan.super_step(dt, Td, bd, energies=True)
        assert abs(ea - eb) <= 1e-6 * abs(eb)
    assert abs(plan.energy(Td) - e0) <= 1e-5 * abs(e0)
    assert plan.check() == 0


def test_tangled_256_limiter_sampled_and_conservation(rk, orc):
    """The 256^3 workload of the limiter benchmark (floor +inf): sampled
    cells of the first super-step against the oracle on windows, then the
    remaining super-steps with FP64 energy conservation."""
    import dataclasses
    W = workloads.tangled(256, seed=2)
    W = dataclasses.replace(W, params=dict(W.params, limiter="mc"))
    rng = np.random.default_rng(3)
    cells = [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(3)] + [(0, 0, 0), (32, 3, 63)]
    plan, Td, bd, dt, e0, P = _sampled_first_step(rk, orc, W, "f32", cells, 0, F32_LIMITER_MAX)
    for _ in range(3):
        s, eb, ea = plan.super_step(dt, Td, bd, energies=True)
        assert abs(ea - eb) <= 1e-6 * abs(eb)
    assert plan.check() == 0
