"""Every cell of the configured workloads against the FP64 oracle run on the
whole grid, in the launch configuration the benchmark times (rkl_super_step
with cached graphs, default kernel choice).

* 3D tangled field, FP32, 256^3, Spitzer: all 10 super-steps at
  dt = 100 dt_expl(T at t = 0).
* 3D saturated blob, FP32, 512^3: the first 2 super-steps at
  dt = 200 dt_expl.
* The batched ensemble (64 uneven problems, autotuned schedule): one
  super-step of every problem.
* The 2D ring, FP64, 100^2: the whole run (400 super-steps).

After every super-step the GPU state is compared with the oracle's, which
advances from the same FP32-rounded inputs in FP64 on its own (Eq.
rkl2scheme, s from Eq. RKL-s of its own state).  Asserted: the relative L2
error of T below 1e-5 (the method's FP32 target), and the relative L2 error
of the change T - T0 below the a priori rounding model of gpu_util
(C_STAGE roundings per stage, amplified through the stages by at most the
undamped-mode factor A_k(s)).  The errors are printed (PARITY lines) and,
when RKL_PARITY_LOG names a file, appended to it as JSON lines."""
import json
import os

import numpy as np
import pytest

import workloads
from gpu_util import change_errors, f32_state_model, host, rounded, torch_dev
from oracle import Problem

pytestmark = pytest.mark.gpu

F32_TARGET = 1e-5


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


def _report(name, step, s, errs, bound_dT):
    rec = dict(config=name, super_steps=step, s=s, bound_rel_l2_dT=bound_dT, **errs)
    print("PARITY " + json.dumps(rec))
    path = os.environ.get("RKL_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


def _run_single(rk, orc, W, n_super, name):
    import torch
    P = Problem(W.T.shape, **W.params)
    T0 = rounded(W.T)
    b = rounded(W.b)
    plan = rk.Plan(W.T.shape, "f32", params=W.params)
    Td, bd = torch_dev(T0), torch_dev(b)
    dt = W.ratio * orc.dt_expl(P, T0)
    Tref = T0
    stages = []
    worst = {}
    for k in range(1, n_super + 1):
        s = plan.super_step(dt, Td, bd)
        Tref, sref = orc.super_step(P, Tref, b, dt)
        assert s == sref, (k, s, sref)
        stages.append(s)
        torch.cuda.synchronize()
        Tg = host(Td)
        errs = change_errors(Tg, Tref, T0)
        bound_dT = f32_state_model(orc, stages) / errs["change_over_state"]
        _report(name, k, s, errs, bound_dT)
        assert errs["rel_l2_T"] < F32_TARGET, (k, errs)
        assert errs["rel_l2_dT"] < bound_dT, (k, errs, bound_dT)
        worst = errs
    assert plan.check() == 0
    plan.close()
    return worst


def test_tangled256_every_cell_ten_super_steps(rk, orc):
    W = workloads.tangled(256, seed=2)
    _run_single(rk, orc, W, W.n_super, "tangled256")


def test_blob512_every_cell_two_super_steps(rk, orc):
    W = workloads.blob(512, seed=2)
    _run_single(rk, orc, W, 2, "blob512")


def test_ensemble64_every_cell_one_super_step(rk, orc):
    """All 64 problems of the batched workload after one super-step in the
    autotuned schedule, each against its own oracle run."""
    import torch
    specs = []
    for sp in workloads.ensemble_specs(64, seed=4):
        shape = (sp["nz"], sp["ny"], sp["nx"])
        prm = dict(dx=(sp["h"],) * 3, kappa_model="spitzer", kappa_par0=sp["kappa_par0"], kappa_perp_ratio=1e-4)
        specs.append(dict(shape=shape, params=prm, seed=sp["seed"], ratio=sp["ratio"]))
    ens = rk.Ensemble([(sp["shape"], sp["params"]) for sp in specs])
    off = ens.offsets
    T_all = torch.empty(off[-1], device="cuda", dtype=torch.float32)
    b_all = torch.empty(3 * off[-1], device="cuda", dtype=torch.float32)
    views = ens.views(T_all, b_all)
    host_in, dts = [], []
    for sp, (Tv, bv) in zip(specs, views):
        nz, ny, nx = sp["shape"]
        T, b = workloads.tangled_box(nx, ny, nz, sp["seed"])
        T, b = rounded(T), rounded(b)
        Tv.copy_(torch.from_numpy(T.astype(np.float32)))
        bv.copy_(torch.from_numpy(b.astype(np.float32)))
        P = Problem(sp["shape"], **sp["params"])
        dts.append(sp["ratio"] * orc.dt_expl(P, T))
        host_in.append((P, T, b))
    ens.autotune(dts, T_all, b_all)
    s = ens.super_step(dts, T_all, b_all)
    torch.cuda.synchronize()
    assert ens.check() == 0
    num = den_T = den_dT = 0.0
    linf = 0.0
    for p, (P, T, b) in enumerate(host_in):
        ref, sref = orc.super_step(P, T, b, dts[p])
        assert s[p] == sref, p
        got = views[p][0].double().cpu().numpy()
        errs = change_errors(got, ref, T)
        bound_dT = f32_state_model(orc, [s[p]]) / errs["change_over_state"]
        assert errs["rel_l2_T"] < F32_TARGET, (p, errs)
        assert errs["rel_l2_dT"] < bound_dT, (p, errs, bound_dT)
        num += float(((got - ref) ** 2).sum())
        den_T += float((ref ** 2).sum())
        den_dT += float(((ref - T) ** 2).sum())
        linf = max(linf, float(np.max(np.abs(got - ref))))
    whole = dict(rel_l2_T=(num / den_T) ** 0.5, rel_l2_dT=(num / den_dT) ** 0.5, linf_abs=linf,
                 problems=len(specs), cells=int(off[-1]), s_min=min(s), s_max=max(s))
    print("PARITY " + json.dumps(dict(config="ensemble64", super_steps=1, **whole)))
    path = os.environ.get("RKL_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(config="ensemble64", super_steps=1, **whole)) + "\n")


def test_ring100_fp64_whole_run_errors(rk, orc):
    """FP64 GPU path: the whole 400-super-step run; rounding order only."""
    W = workloads.ring(100)
    P = Problem(W.T.shape, **W.params)
    plan = rk.Plan(W.T.shape, "f64", params=W.params)
    Td, bd = torch_dev(W.T, "f64"), torch_dev(W.b, "f64")
    dt = W.ratio * orc.dt_expl(P, W.T)
    Tref = W.T.copy()
    for _ in range(W.n_super):
        plan.super_step(dt, Td, bd)
        Tref, _ = orc.super_step(P, Tref, W.b, dt)
    errs = change_errors(host(Td), Tref, W.T)
    _report("ring100", W.n_super, 14, errs, None)
    assert errs["rel_l2_T"] < 1e-13 and errs["rel_l2_dT"] < 1e-11
