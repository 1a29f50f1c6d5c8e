"""Ensembles of uneven problems advanced together (persistent launch and
per-launch schedules) against the FP64 oracle, problem by problem.

* A small ensemble (8 problems, uneven sizes, conductivities, super-steps
  and stage counts, one Dirichlet problem): every cell of every problem
  after two super-steps, both schedules.
* A periodic one: the four schedules (per-launch or persistent, paired-cell
  or row-pair tiles) give the same bits, and match the oracle.
* The full batched workload (64 problems with per-axis sizes drawn from
  {32, 48, 64, 96, 128, 192}, kappa_par0 in [1e-3, 1e-1], dt/dt_expl in
  [20, 400]) in the autotuned schedule: sampled cells of a few problems
  after the first super-step, each recomputed by the oracle on a periodic
  window of side 2(s + 2); FP64 energy of every problem conserved.
* The bounded wait of the persistent kernel gives up with a timeout status
  on a dependency that can never be met, and the ensemble keeps working."""
import numpy as np
import pytest

import workloads
from gpu_util import F32_STATE_MAX, F32_STATE_REL_L2, rel_l2, rounded, window
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


def _build(rk, specs):
    """specs: list of dict(shape, params, seed, ratio).  Returns the ensemble,
    device arrays, FP64 copies of the inputs and the per-problem dt."""
    import torch
    import oracle
    ens = rk.Ensemble([(s["shape"], s["params"]) for s in specs])
    off = ens.offsets
    T_all = torch.empty(off[-1], device="cuda", dtype=torch.float32)
    b_all = torch.empty(3 * off[-1], device="cuda", dtype=torch.float32)
    views = ens.views(T_all, b_all)
    host, dts = [], []
    for s, (Tv, bv) in zip(specs, views):
        nz, ny, nx = s["shape"]
        T, b = workloads.tangled_box(nx, ny, nz, s["seed"])
        T, b = rounded(T), rounded(b)
        Tv.copy_(torch.from_numpy(T.astype(np.float32)))
        bv.copy_(torch.from_numpy(b.astype(np.float32)))
        P = Problem(s["shape"], **s["params"])
        dts.append(s["ratio"] * oracle.dt_expl(P, T))
        host.append((P, T, b))
    return ens, T_all, b_all, views, host, dts


def _small_specs():
    shapes = [(8, 12, 16), (20, 8, 12), (12, 16, 8), (6, 10, 20), (16, 16, 16), (10, 9, 24), (7, 5, 4),
              (14, 11, 36)]
    rng = np.random.default_rng(7)
    out = []
    for p, sh in enumerate(shapes):
        prm = dict(dx=(1.0 / sh[2], 1.0 / sh[1], 1.0 / sh[0]), kappa_model="spitzer",
                   kappa_par0=float(rng.uniform(1e-3, 1e-1)), kappa_perp_ratio=1e-4)
        if p == 5:
            prm.update(bc="dirichlet", bc_value=1.05)
        out.append(dict(shape=sh, params=prm, seed=500 + p, ratio=float(rng.uniform(10, 80))))
    return out


@pytest.mark.parametrize("persistent,nzchunk", [(1, 32), (1, 3), (0, 32), (0, 5)])
def test_small_ensemble_every_cell(rk, orc, persistent, nzchunk):
    import torch
    specs = _small_specs()
    ens, T_all, b_all, views, host, dts = _build(rk, specs)
    ens.set_schedule(persistent, nzchunk)
    refs = [T for (_, T, _) in host]
    for _ in range(2):
        s = ens.super_step(dts, T_all, b_all)
        for p, (P, _, b) in enumerate(host):
            refs[p], sref = orc.super_step(P, refs[p], b, dts[p])
            assert s[p] == sref
    torch.cuda.synchronize()
    assert ens.check() == 0
    for p, (Tv, _) in enumerate(views):
        got = Tv.double().cpu().numpy()
        assert rel_l2(got, refs[p]) < F32_STATE_REL_L2, p
        assert np.max(np.abs(got - refs[p])) < F32_STATE_MAX * np.max(np.abs(refs[p])), p


def _periodic_specs():
    """Eight periodic problems whose widths take both tile widths (32-column
    tiles for 32 and 96, 64-column ones for the rest) and whose heights and
    depths leave ragged last tiles."""
    shapes = [(8, 12, 32), (20, 8, 96), (12, 24, 64), (6, 10, 20), (16, 40, 128), (10, 9, 24), (7, 5, 4),
              (14, 17, 36)]
    rng = np.random.default_rng(11)
    out = []
    for p, sh in enumerate(shapes):
        prm = dict(dx=(1.0 / sh[2], 1.0 / sh[1], 1.0 / sh[0]), kappa_model="spitzer",
                   kappa_par0=float(rng.uniform(1e-3, 1e-1)), kappa_perp_ratio=1e-4)
        out.append(dict(shape=sh, params=prm, seed=700 + p, ratio=float(rng.uniform(10, 80))))
    return out


def test_ensemble_schedules_same_bits(rk, orc):
    """Every schedule (per-launch or persistent, paired-cell or row-pair
    tiles, several z-chunks) advances a periodic ensemble to the same bits,
    and every cell matches the oracle after two super-steps."""
    import torch
    specs = _periodic_specs()
    res = {}
    for sched, nz in [(0, 32), (1, 32), (1, 5), (2, 32), (2, 7), (3, 32), (3, 3), (3, 16)]:
        ens, T_all, b_all, views, host, dts = _build(rk, specs)
        ens.set_schedule(sched, nz)
        s_steps = [ens.super_step(dts, T_all, b_all) for _ in range(2)]
        torch.cuda.synchronize()
        assert ens.check() == 0
        res[(sched, nz)] = T_all.clone()
    for k, v in res.items():
        assert torch.equal(v, res[(0, 32)]), k
    refs = [T for (_, T, _) in host]
    for k in range(2):
        for p, (P, _, b) in enumerate(host):
            refs[p], sref = orc.super_step(P, refs[p], b, dts[p])
            assert s_steps[k][p] == sref
    for p, (Tv, _) in enumerate(views):
        got = Tv.double().cpu().numpy()
        assert rel_l2(got, refs[p]) < F32_STATE_REL_L2, p


def test_row_pair_schedule_needs_periodic_problems(rk):
    """The row-pair tile body wraps its halo periodically: an ensemble with
    a Dirichlet problem refuses schedules 2 and 3 (and the autotuner does not
    try them), rather than running them wrongly."""
    specs = _small_specs()                         # problem 5 is Dirichlet
    ens, T_all, b_all, views, host, dts = _build(rk, specs)
    for sched in (2, 3):
        with pytest.raises(Exception):
            ens.set_schedule(sched, 32)
    with pytest.raises(Exception):
        ens.set_schedule(4, 32)
    ens.set_schedule(1, 32)
    pers, nz, ms = ens.autotune(dts, T_all, b_all)
    assert pers in (0, 1)


def test_full_batched_workload_sampled(rk, orc):
    import torch
    specs = []
    for sp in workloads.ensemble_specs(64, seed=4):
        shape = (sp["nz"], sp["ny"], sp["nx"])
        prm = dict(dx=(sp["h"],) * 3, kappa_model="spitzer",
                   kappa_par0=sp["kappa_par0"], kappa_perp_ratio=1e-4)
        specs.append(dict(shape=shape, params=prm, seed=sp["seed"], ratio=sp["ratio"]))
    ens, T_all, b_all, views, host, dts = _build(rk, specs)
    T_before = T_all.clone()
    pers, nz, ms = ens.autotune(dts, T_all, b_all)
    assert torch.equal(T_all, T_before)            # the autotuner works on a scratch copy
    assert pers in (0, 1, 2, 3) and nz in (8, 16, 32, 48, 64) and ms > 0
    e0 = [float(Tv.double().sum()) for Tv, _ in views]
    s = ens.super_step(dts, T_all, b_all)
    torch.cuda.synchronize()
    assert ens.check() == 0
    # sampled cells: the problem with the largest s, the smallest grid, and two others
    order = sorted(range(len(specs)), key=lambda p: -s[p])
    smallest = min(range(len(specs)), key=lambda p: np.prod(specs[p]["shape"]))
    picks = [order[0], smallest, order[len(order) // 2], 17]
    rng = np.random.default_rng(3)
    for p in picks:
        P, T, b = host[p]
        got = views[p][0].double().cpu().numpy()
        half = s[p] + 2
        for _ in range(2):
            c = tuple(int(rng.integers(0, n)) for n in specs[p]["shape"])
            Tw = window(T, c, half)
            bw = window(b, c, half, axes_first=1)
            Tw1, sw = orc.super_step(Problem(Tw.shape, **specs[p]["params"]), Tw, bw, dts[p], s[p])
            ref = Tw1[half, half, half]
            assert abs(got[c] - ref) < F32_STATE_MAX * np.max(np.abs(T)), (p, c)
    # energy of every (periodic) problem is conserved
    for p, (Tv, _) in enumerate(views):
        assert abs(float(Tv.double().sum()) - e0[p]) <= 1e-6 * abs(e0[p]), p


def test_full_batched_workload_ten_steps_bounded(rk):
    """Ten super-steps of all 64 problems: every cell stays finite and inside
    the initial range (up to the small undershoot of the non-monotone
    transverse-gradient scheme), energy is conserved per problem."""
    import torch
    specs = []
    for sp in workloads.ensemble_specs(64, seed=4):
        shape = (sp["nz"], sp["ny"], sp["nx"])
        prm = dict(dx=(sp["h"],) * 3, kappa_model="spitzer", kappa_par0=sp["kappa_par0"], kappa_perp_ratio=1e-4)
        specs.append(dict(shape=shape, params=prm, seed=sp["seed"], ratio=sp["ratio"]))
    ens, T_all, b_all, views, host, dts = _build(rk, specs)
    e0 = [float(Tv.double().sum()) for Tv, _ in views]
    lo, hi = float(T_all.min()), float(T_all.max())
    for _ in range(10):
        ens.super_step(dts, T_all, b_all)
    torch.cuda.synchronize()
    assert ens.check() == 0
    assert bool(torch.isfinite(T_all).all())
    assert float(T_all.min()) > lo - 0.1 * (hi - lo) and float(T_all.max()) < hi + 0.1 * (hi - lo)
    for p, (Tv, _) in enumerate(views):
        assert abs(float(Tv.double().sum()) - e0[p]) <= 1e-5 * abs(e0[p]), p


def test_persistent_wait_times_out_and_recovers(rk, orc):
    import torch
    specs = _small_specs()[:3]
    ens, T_all, b_all, views, host, dts = _build(rk, specs)
    assert ens.selftest_timeout() == rk._lib.RKL_ERR_TIMEOUT
    assert ens.check() == 0                        # the self-test cleared its status
    s = ens.super_step(dts, T_all, b_all)          # and the context is still usable
    torch.cuda.synchronize()
    P, T, b = host[0]
    ref, _ = orc.super_step(P, T, b, dts[0])
    assert rel_l2(views[0][0].double().cpu().numpy(), ref) < F32_STATE_REL_L2
