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
