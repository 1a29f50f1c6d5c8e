"""rkl_dt_expl_energy_noalloc: the entry point for callers that cannot
allocate device memory (it takes no plan and keeps its scratch in a fixed
array inside the library).  Its results must equal what the plan-based
rkl_dt_expl and rkl_energy return on the same arrays, call after call.

This file is collected last on purpose: the entry point shares one scratch
array per device across calls, so it is also exercised after everything
else has run in the same process."""
import numpy as np
import pytest

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


def _case(dtype, shape, seed):
    nz, ny, nx = shape
    T, _ = workloads.tangled_box(nx, ny, nz, seed)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    return T, params


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_plan_entry_points_twice(rk, dtype):
    import torch
    from paper_1702_05487_gb300 import _lib, make_grid, make_phys
    stream = torch.cuda.current_stream()
    # two different arrays, two calls in a row: the second call must not see
    # anything the first one left in the shared scratch
    for k, shape in enumerate([(40, 36, 44), (17, 65, 30)]):
        T, params = _case(dtype, shape, seed=100 + k)
        Td = torch.from_numpy(T.astype(np.float32 if dtype == "f32" else np.float64)).cuda()
        plan = rk.Plan(shape, dtype, params=params)
        want_dt = plan.dt_expl(Td)
        want_e = plan.energy(Td)
        plan.close()
        dt, e = _lib.rkl_dt_expl_energy_noalloc(make_grid(shape, dtype=dtype), make_phys(**params), Td,
                                                stream.cuda_stream)
        assert dt == pytest.approx(want_dt, rel=1e-14)     # the max is order independent
        assert e == pytest.approx(want_e, rel=1e-12)       # FP64 sums in another order


def test_noalloc_rejects_grids_beyond_its_scratch(rk):
    import torch
    from paper_1702_05487_gb300 import _lib, make_grid, make_phys
    T = torch.ones(8, device="cuda")
    # 2^27 + 2^18 cells: over the limit; rejected before anything touches T
    g = make_grid((513, 512, 512))
    with pytest.raises(rk.RklError) as ei:
        _lib.rkl_dt_expl_energy_noalloc(g, make_phys(), T)
    assert ei.value.status == _lib.RKL_ERR_INVALID_ARG
    assert "134217728" in str(ei.value)
    # exactly at the limit is accepted by the size check (bad physics then rejects it first)
    g = make_grid((512, 512, 512))
    p = make_phys()
    p.cp = 0.9
    with pytest.raises(rk.RklError) as ei:
        _lib.rkl_dt_expl_energy_noalloc(g, p, T)
    assert "cp" in str(ei.value)
    # a 2D grid whose unused third axis claims more than one cell would make
    # the reduction read past the end of T: rejected like rkl_plan_create does
    g = make_grid((2, 4))
    g.n[2] = 3
    with pytest.raises(rk.RklError) as ei:
        _lib.rkl_dt_expl_energy_noalloc(g, make_phys(), T)
    assert ei.value.status == _lib.RKL_ERR_INVALID_ARG
    assert "inactive axis" in str(ei.value)


def test_noalloc_reports_nonfinite_under_any_kappa(rk):
    """Unlike rkl_dt_expl under constant kappa (which never reads T), this
    entry point reads every cell and reports NaN / Inf as an error."""
    import torch
    from paper_1702_05487_gb300 import _lib, make_grid, make_phys
    T = torch.ones((6, 5, 7), device="cuda")
    T[3, 2, 6] = float("nan")
    for kappa in ("const", "spitzer"):
        with pytest.raises(rk.RklError) as ei:
            _lib.rkl_dt_expl_energy_noalloc(make_grid((6, 5, 7)), make_phys(kappa_model=kappa), T)
        assert ei.value.status == _lib.RKL_ERR_NONFINITE
    T[3, 2, 6] = 1.0
    dt, e = _lib.rkl_dt_expl_energy_noalloc(make_grid((6, 5, 7)), make_phys(), T)
    assert e == pytest.approx(1.0)          # 210 cells of T = 1, each of volume 1/210


def test_noalloc_at_its_largest_grid_against_the_oracle(rk, orc):
    """A 512^3 FP32 grid, 2^27 cells, fills every partial slot of the
    scratch.  The hottest and the coldest cell sit in the last block, so
    dt_expl depends on the top slot; the result must match the FP64 oracle's
    Eq. dt_exp and energy, and a small grid reduced right after must not see
    the large one's partials."""
    import torch
    from oracle import Problem
    from paper_1702_05487_gb300 import _lib, make_grid, make_phys
    n = 512
    rng = np.random.default_rng(27)
    T = (0.8 + 0.4 * rng.random(n ** 3, dtype=np.float32)).reshape(n, n, n)
    T[-1, -1, -1] = np.float32(1.75)
    T[-1, -1, -3] = np.float32(0.5)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    P = Problem(T.shape, dx=(1.0 / n,) * 3, **params)
    T64 = T.astype(np.float64)
    want_dt, want_e = orc.dt_expl(P, T64), orc.energy(P, T64)
    del T64
    Td = torch.from_numpy(T).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    dt, e = _lib.rkl_dt_expl_energy_noalloc(make_grid(T.shape), make_phys(**params), Td, stream)
    assert dt == pytest.approx(want_dt, rel=1e-14)
    assert e == pytest.approx(want_e, rel=1e-12)
    del Td
    Ts = torch.full((3, 4, 5), 2.0, device="cuda")
    dt2, e2 = _lib.rkl_dt_expl_energy_noalloc(make_grid((3, 4, 5)), make_phys(**params), Ts, stream)
    Ps = Problem((3, 4, 5), dx=(1 / 5, 1 / 4, 1 / 3), **params)
    assert dt2 == pytest.approx(orc.dt_expl(Ps, np.full((3, 4, 5), 2.0)), rel=1e-14)
    assert e2 == pytest.approx(orc.energy(Ps, np.full((3, 4, 5), 2.0)), rel=1e-14)
