"""GPU path against the FP64 oracle, element by element, through the C ABI.

Sizes span several tiles of the tiled kernel with ragged tails; the FP32
tolerances are derived in gpu_util.  Inputs are the seeded workload fields,
rounded to the kernel dtype and handed to both sides."""
import math

import numpy as np
import pytest

import workloads
from gpu_util import (F32_FLUX_TOL, F32_LIMITER_MAX, F32_STATE_MAX, F32_STATE_REL_L2, F64_TOL, change_errors,
                      f32_state_model, host, norm_max, rel_l2, rounded, torch_dev)
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


def _cases():
    # (name, shape, params, dtype)
    spitz = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    return [
        ("3d_spitzer_perp", (35, 37, 40), spitz, "f32"),
        ("3d_const_aniso", (17, 70, 33), dict(kappa_par0=0.02), "f32"),
        ("3d_saturated", (24, 33, 66), dict(kappa_model="spitzer", kappa_par0=0.01, saturate=True,
                                            phi=0.3), "f32"),
        ("3d_saturated_upwind", (20, 18, 35), dict(kappa_model="spitzer", kappa_par0=0.01,
                                                   saturate=True, phi=0.05, sat_upwind=True), "f32"),
        # constant kappa with saturation (the paired-cell kernel: nx % 4 == 0)
        ("3d_saturated_const", (16, 20, 48), dict(kappa_par0=0.02, kappa_perp_ratio=0.1, saturate=True,
                                                  phi=0.003), "f32"),
        ("3d_dirichlet", (19, 21, 34), dict(spitz, bc="dirichlet", bc_value=0.9), "f32"),
        ("3d_f64", (13, 15, 17), spitz, "f64"),
        ("2d_f64_dirichlet", (41, 29), dict(kappa_par0=0.05, bc="dirichlet", bc_value=1.0), "f64"),
        ("2d_f32", (45, 67), spitz, "f32"),
        ("1d_f32", (300,), dict(kappa_par0=0.3, kappa_perp_ratio=1.0), "f32"),
        # MC-limited transverse gradients (Appendix C; generic and tiled kernels)
        ("3d_limiter_mc", (20, 22, 24), dict(spitz, limiter="mc"), "f32"),
        ("3d_limiter_sat", (12, 16, 20), dict(kappa_model="spitzer", kappa_par0=0.01, saturate=True, phi=0.3,
                                               limiter="mc"), "f32"),
        ("2d_f64_limiter_floor", (30, 26), dict(kappa_par0=0.05, bc="dirichlet", bc_value=1.0, limiter="mc",
                                                limiter_floor=1.02), "f64"),
    ]


def _fields(shape, seed=11):
    """Tangled-field T and b on any grid shape (2D/1D take slices)."""
    nd = len(shape)
    full = tuple(shape) + (1,) * (3 - nd) if nd < 3 else shape
    if nd == 3:
        nz, ny, nx = shape
        T, b = workloads.tangled_box(nx, ny, nz, seed)
    elif nd == 2:
        ny, nx = shape
        T, b = workloads.tangled_box(nx, ny, 4, seed)
        T, b = T[0], b[:2, 0]
        b = b / np.sqrt((b ** 2).sum(0))
    else:
        T, b = workloads.tangled_box(shape[0], 4, 4, seed)
        T, b = T[0, 0], np.ones((1, shape[0]))
    return T, b


def _setup(rk, name, shape, params, dtype, variant=0):
    T, b = _fields(shape)
    P = Problem(shape, **params)
    plan = rk.Plan(shape, dtype, params=params)
    plan.set_variant(variant)
    Td, bd = torch_dev(T, dtype), torch_dev(b, dtype)
    return P, plan, rounded(T, dtype), rounded(b, dtype), Td, bd


@pytest.mark.parametrize("case", _cases(), ids=[c[0] for c in _cases()])
def test_flux_and_M(rk, orc, case):
    import torch
    name, shape, params, dtype = case
    P, plan, T, b, Td, bd = _setup(rk, *case)
    nd = len(shape)
    F = [torch.empty_like(Td) for _ in range(nd)]
    plan.flux(Td, bd, *F)
    M = torch.empty_like(Td)
    plan.apply_M(Td, bd, M)
    torch.cuda.synchronize()
    Fref = orc.flux(P, T, b)
    Mref = orc.apply_M(P, T, b)
    tol = F64_TOL if dtype == "f64" else F32_FLUX_TOL
    for d in range(nd):
        assert norm_max(host(F[d]), Fref[d]) < tol, (name, d)
    assert norm_max(host(M), Mref) < tol, name
    if params.get("bc", "periodic") == "periodic":
        # one flux per face: M sums to zero up to rounding
        assert abs(float(host(M).sum())) <= 1e-5 * float(np.abs(host(M)).sum())


@pytest.mark.parametrize("case", _cases(), ids=[c[0] for c in _cases()])
def test_stages_one_by_one(rk, orc, case):
    """rkl_stage for j = 1, 2, 3 against the oracle's stages from the same inputs."""
    import torch
    name, shape, params, dtype = case
    P, plan, T, b, Td, bd = _setup(rk, *case)
    s = 7
    dt = 10 * orc.dt_expl(P, T)
    MY0 = torch.empty_like(Td)
    Y1 = torch.empty_like(Td)
    plan.stage(1, s, dt, bd, Td, MY0, None, None, Y1)
    Y1r, MY0r = orc.stage(P, 1, s, dt, b, T, None, None, None)
    torch.cuda.synchronize()
    tol = F64_TOL if dtype == "f64" else F32_FLUX_TOL
    assert norm_max(host(MY0), MY0r) < tol
    assert norm_max(host(Y1), Y1r) < (F64_TOL if dtype == "f64" else F32_STATE_MAX)
    # stage 2 and 3 from oracle-side inputs rounded to the kernel dtype
    Y1in = rounded(Y1r, dtype)
    MY0in = rounded(MY0r, dtype)
    Y2 = torch.empty_like(Td)
    plan.stage(2, s, dt, bd, Td, torch_dev(MY0in, dtype), torch_dev(Y1in, dtype), Td, Y2)
    Y2r, _ = orc.stage(P, 2, s, dt, b, T, MY0in, Y1in, T)
    Y3 = torch.empty_like(Td)
    Y2in = rounded(Y2r, dtype)
    plan.stage(3, s, dt, bd, Td, torch_dev(MY0in, dtype), torch_dev(Y2in, dtype), torch_dev(Y1in, dtype), Y3)
    Y3r, _ = orc.stage(P, 3, s, dt, b, T, MY0in, Y2in, Y1in)
    torch.cuda.synchronize()
    stol = F64_TOL if dtype == "f64" else F32_STATE_MAX
    assert norm_max(host(Y2), Y2r) < stol
    assert norm_max(host(Y3), Y3r) < stol


def _variant_cases():
    out = []
    for c in _cases():
        out.append(c + (0,))
        if c[3] == "f32" and len(c[1]) == 3:
            out.append(c + (1,))        # the generic kernel on the same 3D FP32 case
            out.append(c + (2,))        # the tiled one-cell-per-thread kernel
    # grids with nx % 4 == 0 (the paired-cell kernel) and Dirichlet partial tiles
    spitz = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    sat = dict(kappa_model="spitzer", kappa_par0=0.01, saturate=True, phi=0.3)
    for v in (2, 3, 4, 5, 6, 7, 8, 9, 10):
        if v not in (5, 6, 8, 10):  # two-stage, bulk, tensor-map and row-pair kernels are periodic only
            out.append(("3d_x4_dirichlet", (21, 19, 36), dict(spitz, bc="dirichlet", bc_value=0.9), "f32", v))
        out.append(("3d_x4_sat", (18, 26, 68), sat, "f32", v))
        out.append(("3d_x4_sat_upwind", (10, 9, 132), dict(sat, phi=0.05, sat_upwind=True), "f32", v))
        out.append(("3d_x4_const", (33, 17, 44), dict(kappa_par0=0.02, kappa_perp_ratio=0.1), "f32", v))
    # MC limiter on the tiled kernel: Dirichlet ghosts, a floor inside the
    # temperature range (both branches per face), several 32 x 8 tiles
    lim = dict(spitz, bc="dirichlet", bc_value=0.95, limiter="mc", limiter_floor=1.0)
    for v in (0, 1, 2):
        out.append(("3d_limiter_floor_dirichlet", (14, 18, 70), lim, "f32", v))
    # MC limiter at every face on the paired-cell kernel (variant 0 and the
    # paired-cell variants all launch its limited build): Dirichlet ghosts,
    # two tile columns with a ragged one, several 64 x 4 tiles, saturation
    lim_all = dict(spitz, bc="dirichlet", bc_value=0.95, limiter="mc")
    for v in (0, 3, 7):
        out.append(("3d_limiter_all_dirichlet", (14, 18, 68), lim_all, "f32", v))
    out.append(("3d_limiter_all_periodic", (21, 13, 132), dict(spitz, limiter="mc"), "f32", 4))
    out.append(("3d_limiter_all_sat_const", (9, 10, 40), dict(kappa_par0=0.02, kappa_perp_ratio=0.1, saturate=True,
                                                             phi=0.003, limiter="mc"), "f32", 0))
    # two-stage kernel: several 60 x 7 tiles with ragged edges in x, y and z
    out.append(("3d_pair_spitzer", (45, 30, 128), spitz, "f32", 5))
    out.append(("3d_pair_small", (5, 4, 8), spitz, "f32", 5))
    # bulk (TMA-engine) copies: x-halo rows split at the periodic edge, ragged y
    out.append(("3d_bulk_spitzer", (37, 21, 200), spitz, "f32", 6))
    out.append(("3d_bulk_x72", (9, 16, 72), spitz, "f32", 6))
    # tensor-map bundles: zero-filled boxes at every edge patched with the
    # periodic images (ragged x and y tiles; the smallest grid they take,
    # 72 x 6, with a second tile column of 8 and a tile row of 2)
    out.append(("3d_tmaps_ragged", (37, 21, 200), spitz, "f32", 8))
    out.append(("3d_tmaps_thin", (11, 6, 72), spitz, "f32", 8))
    out.append(("3d_tmaps_sat", (13, 12, 132), sat, "f32", 8))
    # 32-column tiles (two rows of 16 lanes per warp, eight rows per tile):
    # widths of one, two and a ragged three tiles, ragged rows, Dirichlet
    out.append(("3d_cols32_ragged", (9, 21, 68), spitz, "f32", 9))
    out.append(("3d_cols32_narrow", (12, 10, 32), spitz, "f32", 9))
    out.append(("3d_cols32_dirichlet", (7, 13, 96), dict(spitz, bc="dirichlet", bc_value=0.9), "f32", 9))
    # row-pair kernel (two rows per warp, 64 x 8 tiles): ragged tile rows and
    # columns, a grid lower than one tile, one narrower than one tile
    out.append(("3d_rowpair_ragged", (37, 21, 200), spitz, "f32", 10))
    out.append(("3d_rowpair_low", (11, 5, 136), spitz, "f32", 10))
    out.append(("3d_rowpair_narrow", (19, 17, 36), sat, "f32", 10))
    return out


@pytest.mark.parametrize("case", _variant_cases(), ids=[f"{c[0]}-v{c[4]}" for c in _variant_cases()])
def test_super_steps(rk, orc, case):
    """Three super-steps with s chosen from dt / dt_expl; FP64 energies."""
    name, shape, params, dtype, variant = case
    P, plan, T, b, Td, bd = _setup(rk, name, shape, params, dtype, variant)
    ratio = 100.0 if len(shape) == 3 else 50.0
    dt = ratio * orc.dt_expl(P, T)
    Tref = T.copy()
    periodic = params.get("bc", "periodic") == "periodic"
    stages = []
    for k in range(3):
        s, eb, ea = plan.super_step(dt, Td, bd, energies=True)
        Tref, sref = orc.super_step(P, Tref, b, dt)
        assert s == sref
        stages.append(s)
        if periodic:
            assert abs(ea - eb) <= (1e-12 if dtype == "f64" else 1e-6) * abs(eb)
    Tg = host(Td)
    if dtype == "f64":
        assert norm_max(Tg, Tref) < F64_TOL
    else:
        assert rel_l2(Tg, Tref) < F32_STATE_REL_L2
        assert norm_max(Tg, Tref) < (F32_LIMITER_MAX if params.get("limiter") == "mc" else F32_STATE_MAX)
        if params.get("limiter") != "mc":
            # the change T - T0 against the a priori rounding model (the MC
            # limiter's kinks are outside the model: a rounding that crosses
            # one changes a slope by up to a factor 2)
            errs = change_errors(Tg, Tref, T)
            assert errs["rel_l2_dT"] < f32_state_model(orc, stages) / errs["change_over_state"], errs
    assert plan.check() == 0


@pytest.mark.parametrize("shape,nzchunk", [((32, 32, 32), 0), ((7, 9, 5), 0), ((40, 3, 70), 0),
                                           ((1, 33, 64), 0), ((65, 8, 36), 0), ((37, 24, 128), 5),
                                           ((64, 16, 64), 64), ((9, 40, 4), 2), ((3, 8, 200), 1),
                                           ((37, 24, 128), -1), ((100, 16, 68), -1)])
def test_tiled_kernels_match_generic(rk, orc, shape, nzchunk):
    """The tiled kernels (variants 2 and 3, the latter when nx % 4 == 0,
    with several z-chunk lengths, and nzchunk -1 = the balanced schedule
    whose runs cross tile columns) and the generic kernel (variant 1) on
    tile-aligned, ragged and degenerate shapes; all against the oracle."""
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    variants = (1, 2, 3, 4, 5, 6, 8, 9, 10, 11) if shape[2] % 4 == 0 else (1, 2)
    res = {}
    for v in variants:
        P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32", v)
        if v >= 3:
            plan.set_variant(v, nzchunk if v != 5 else max(nzchunk, 0))
        dt = 40 * orc.dt_expl(P, T)
        for _ in range(2):
            plan.super_step(dt, Td, bd)
        res[v] = host(Td)
    Tref = T
    for _ in range(2):
        Tref, _ = orc.super_step(P, Tref, b, dt)
    for v in variants:
        assert rel_l2(res[v], Tref) < F32_STATE_REL_L2, v
        assert norm_max(res[v], res[1]) < F32_STATE_MAX, v


@pytest.mark.parametrize("params", [
    dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4),
    dict(kappa_model="spitzer", kappa_par0=0.01, saturate=True, phi=0.3),
    dict(kappa_par0=0.02, kappa_perp_ratio=0.1, saturate=True, phi=0.003),
    dict(kappa_model="spitzer", kappa_par0=0.01, saturate=True, phi=0.05, sat_upwind=True),
    dict(kappa_par0=0.02, kappa_perp_ratio=0.1),
    dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4, limiter="mc"),
    dict(kappa_model="spitzer", kappa_par0=0.01, saturate=True, phi=0.3, limiter="mc"),
], ids=["spitzer", "sat", "sat_const", "sat_upwind", "const", "mc", "mc_sat"])
@pytest.mark.parametrize("shape,nzchunk", [((37, 21, 200), 0), ((16, 16, 128), 0), ((40, 9, 68), 7),
                                           ((3, 8, 64), 1), ((24, 40, 4), 0)])
def test_row_pair_kernel_same_bits_as_paired_cell(rk, orc, params, shape, nzchunk):
    """The row-pair kernel (variant 10: 64 x 8 tiles; variant 11: 32 x 16
    tiles, two row pairs per warp) evaluates every face, slope, divergence
    term and update as the paired-cell kernel of the same tile width
    (variant 3: 64 x 4; variant 9: 32 x 8) does, with tile boundaries at
    other rows and other z-chunks: after two super-steps (every stage, the
    first one included) each pair of states agrees bit for bit, and both
    with the oracle.  (Across tile widths the bits differ: a cell on a
    tile's left edge adds its left x-face to the divergence after the rest,
    so columns at multiples of 32 but not 64 round differently.)"""
    import torch
    res = {}
    for v in (3, 9, 10, 11):
        P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32", v)
        plan.set_variant(v, nzchunk)
        dt = 60 * orc.dt_expl(P, T)
        for _ in range(2):
            plan.super_step(dt, Td, bd)
        assert plan.check() == 0
        res[v] = Td.clone()
    assert torch.equal(res[3], res[10])
    assert torch.equal(res[9], res[11])
    Tref = T
    for _ in range(2):
        Tref, _ = orc.super_step(P, Tref, b, dt)
    assert rel_l2(host(res[10]), Tref) < F32_STATE_REL_L2
    assert rel_l2(host(res[11]), Tref) < F32_STATE_REL_L2


def test_row_pair_kernel_unsupported_plans(rk):
    """Variants 10 and 11 take periodic FP32 3D grids with nx % 4 == 0,
    without a limiter or with it at every face; any other plan is refused,
    not silently routed elsewhere."""
    spitz = dict(kappa_model="spitzer", kappa_par0=0.01)
    for shape, params, dtype in [((8, 8, 30), spitz, "f32"),
                                 ((8, 8, 32), dict(spitz, bc="dirichlet", bc_value=1.0), "f32"),
                                 ((8, 8, 32), dict(spitz, limiter="mc", limiter_floor=1.0), "f32"),
                                 ((8, 8, 32), spitz, "f64"),
                                 ((16, 32), spitz, "f32")]:
        plan = rk.Plan(shape, dtype, params=params)
        for v in (10, 11):
            with pytest.raises(Exception):
                plan.set_variant(v)


@pytest.mark.parametrize("shape,nzchunk", [((7, 9, 4), 0), ((40, 3, 68), 0), ((1, 33, 64), 0), ((37, 24, 128), 5),
                                           ((9, 40, 8), 2), ((3, 8, 200), 1), ((37, 24, 128), -1),
                                           ((21, 16, 68), -1)])
def test_limited_paired_cell_shapes_and_schedules(rk, orc, shape, nzchunk):
    """The paired-cell kernel's MC-limited build on tile-aligned, ragged and
    degenerate shapes, with several z-chunk lengths and the balanced
    schedule (nzchunk -1), against the oracle and the generic kernel."""
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4, limiter="mc")
    res = {}
    for v in (1, 3):
        P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32", v)
        if v == 3:
            plan.set_variant(v, nzchunk)
        dt = 40 * orc.dt_expl(P, T)
        for _ in range(2):
            plan.super_step(dt, Td, bd)
        assert plan.check() == 0
        res[v] = host(Td)
    Tref = T
    for _ in range(2):
        Tref, _ = orc.super_step(P, Tref, b, dt)
    for v in (1, 3):
        assert rel_l2(res[v], Tref) < F32_STATE_REL_L2, v
        assert norm_max(res[v], Tref) < F32_LIMITER_MAX, v


def test_autotune_keeps_input_and_parity(rk, orc):
    """The autotuner times every kernel on a scratch copy, leaves T alone,
    and the kernel it picks still matches the oracle."""
    import torch
    shape = (40, 24, 64)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32")
    dt = 50 * orc.dt_expl(P, T)
    T_before = Td.clone()
    v, nz, ms = plan.autotune(dt, Td, bd)
    assert torch.equal(Td, T_before)
    assert 1 <= v <= 10 and ms > 0           # any kernel that applies to the grid
    plan.super_step(dt, Td, bd)
    Tref, _ = orc.super_step(P, T, b, dt)
    assert rel_l2(host(Td), Tref) < F32_STATE_REL_L2


def test_autotune_limiter_plan(rk, orc):
    """A limiter plan (floor +inf) autotunes over the generic, tiled and
    limited paired-cell kernels only, and the pick matches the oracle."""
    import torch
    shape = (20, 16, 64)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4, limiter="mc")
    P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32")
    dt = 50 * orc.dt_expl(P, T)
    T_before = Td.clone()
    v, nz, ms = plan.autotune(dt, Td, bd)
    assert torch.equal(Td, T_before)
    assert v in (1, 2, 3) and ms > 0
    plan.super_step(dt, Td, bd)
    Tref, _ = orc.super_step(P, T, b, dt)
    assert rel_l2(host(Td), Tref) < F32_STATE_REL_L2
    assert norm_max(host(Td), Tref) < F32_LIMITER_MAX


def test_dt_expl_and_energy(rk, orc):
    shape = (24, 20, 36)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32")
    assert plan.dt_expl(Td) == pytest.approx(orc.dt_expl(P, T), rel=1e-14)
    assert plan.energy(Td) == pytest.approx(orc.energy(P, T), rel=1e-12)


def test_super_step_s_and_timing(rk, orc):
    import torch
    shape = (32, 32, 32)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32")
    dt = 30 * orc.dt_expl(P, T)
    s = orc.num_stages(30)
    plan.set_timing(True)
    for _ in range(4):
        plan.super_step_s(dt, s, Td, bd)
    ms, n = plan.timing()
    assert n == 4 * (s - 1) and ms > 0
    plan.set_timing(False)
    Tref = T
    for _ in range(4):
        Tref, _ = orc.super_step(P, Tref, b, dt, s)
    assert rel_l2(host(Td), Tref) < F32_STATE_REL_L2


def test_run_host_matches_device_path(rk, orc):
    import torch
    shape = (20, 24, 28)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    P, plan, T, b, Td, bd = _setup(rk, "x", shape, params, "f32")
    dt = 50 * orc.dt_expl(P, T)
    Th = np.ascontiguousarray(T, dtype=np.float32)
    bh = np.ascontiguousarray(b, dtype=np.float32)
    s = plan.run_host(dt, 2, Th, bh)
    for _ in range(2):
        s_dev = plan.super_step(dt, Td, bd)
    torch.cuda.synchronize()
    assert s == s_dev
    assert np.array_equal(Th, host(Td).astype(np.float32))


def test_run_host_batch_edge_cases(rk):
    """No jobs is a no-op; a null host buffer is an argument error raised
    before any copy."""
    import ctypes
    shape = (8, 8, 16)
    params = dict(kappa_model="spitzer", kappa_par0=0.01)
    plan = rk.Plan(shape, "f32", params=params)
    assert plan.run_host_batch(1e-3, 1, [], []) == []
    T = np.ones(shape, dtype=np.float32)
    b = np.zeros((3,) + shape, dtype=np.float32)
    b[0] = 1.0
    lib = rk._lib.load()
    Tp = (ctypes.c_void_p * 2)(T.ctypes.data, None)
    bp = (ctypes.c_void_p * 2)(b.ctypes.data, b.ctypes.data)
    st = lib.rkl_run_host_batch(plan.handle, 1e-3, 1, 2, Tp, bp, None)
    assert st == rk._lib.RKL_ERR_INVALID_ARG
    assert np.all(T == 1.0)
    assert plan.check() == 0


@pytest.mark.parametrize("n_jobs", [1, 2, 5])
def test_run_host_batch_matches_serial_and_oracle(rk, orc, n_jobs):
    """Jobs streamed with overlapping copies give, bit for bit, what one
    rkl_run_host call per job gives (page-locked and pageable buffers), and
    job 0 matches the oracle."""
    import torch
    shape = (20, 24, 32)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    P = Problem(shape, **params)
    plan = rk.Plan(shape, "f32", params=params)
    jobs = []
    for i in range(n_jobs):
        T, b = _fields(shape, seed=40 + i)
        jobs.append((rounded(T, "f32"), rounded(b, "f32")))
    dt = 30 * orc.dt_expl(P, jobs[0][0])
    pinned = n_jobs != 2
    mk = (lambda a: torch.from_numpy(a.astype(np.float32)).pin_memory()) if pinned else \
        (lambda a: np.ascontiguousarray(a, dtype=np.float32))
    Ts = [mk(T) for T, _ in jobs]
    bs = [mk(b) for _, b in jobs]
    s_batch = plan.run_host_batch(dt, 2, Ts, bs)
    for i, (T, b) in enumerate(jobs):
        Th = np.ascontiguousarray(T, dtype=np.float32)
        bh = np.ascontiguousarray(b, dtype=np.float32)
        s = plan.run_host(dt, 2, Th, bh)
        got = Ts[i].numpy() if pinned else Ts[i]
        assert s == s_batch[i]
        assert np.array_equal(got, Th), i
    ref = jobs[0][0]
    for _ in range(2):
        ref, _ = orc.super_step(P, ref, jobs[0][1], dt)
    got0 = (Ts[0].numpy() if pinned else Ts[0]).astype(np.float64)
    assert rel_l2(got0, ref) < F32_STATE_REL_L2
    assert plan.check() == 0


@pytest.mark.parametrize("nbuf", [2, 3])
def test_run_host_batch_rotating_host_buffers(rk, nbuf):
    """Seven jobs over nbuf page-locked host buffers used in rotation (job
    i + nbuf starts from job i's result, the way bench.py streams its
    steps): with two buffers the copy-in of job i must wait for job i - 2's
    copy-out into the same buffer; with three, copies of neighbouring jobs
    run side by side.  Both give, bit for bit, the same sequence run one
    rkl_run_host call at a time."""
    import torch
    shape = (12, 16, 64)
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    plan = rk.Plan(shape, "f32", params=params)
    fields = [_fields(shape, seed=60 + k) for k in range(nbuf)]
    dt = 3e-5
    Th = [torch.from_numpy(T.astype(np.float32)).pin_memory() for T, _ in fields]
    bh = [torch.from_numpy(b.astype(np.float32)).pin_memory() for _, b in fields]
    n_jobs = 7
    s_batch = plan.run_host_batch(dt, 1, [Th[i % nbuf] for i in range(n_jobs)], [bh[i % nbuf] for i in range(n_jobs)])
    Tr = [np.ascontiguousarray(T, dtype=np.float32) for T, _ in fields]
    br = [np.ascontiguousarray(b, dtype=np.float32) for _, b in fields]
    for i in range(n_jobs):
        s = plan.run_host(dt, 1, Tr[i % nbuf], br[i % nbuf])
        assert s == s_batch[i], i
    for k in range(nbuf):
        assert np.array_equal(Th[k].numpy(), Tr[k]), k
    assert plan.check() == 0


def test_invalid_arguments_and_device_status(rk):
    import torch
    shape = (16, 16, 16)
    params = dict(kappa_model="spitzer", kappa_par0=0.01)
    plan = rk.Plan(shape, "f32", params=params)
    T = torch.ones(shape, device="cuda")
    b = torch.zeros((3,) + shape, device="cuda")
    b[0] = 1
    with pytest.raises(rk.RklError) as ei:
        plan.super_step(-1.0, T, b)
    assert ei.value.status == 1
    with pytest.raises(rk.RklError):
        plan.stage(3, 2, 1e-3, b, T, T, T, T, T)
    # a non-positive temperature under Spitzer kappa is reported, not hidden
    T2 = T.clone()
    T2[3, 4, 5] = -1.0
    with pytest.raises(rk.RklError) as ei:
        plan.super_step(1e-3, T2, b)
    assert ei.value.status == rk._lib.RKL_ERR_NONPOSITIVE_T
    T3 = T.clone()
    T3[1, 2, 3] = float("nan")
    with pytest.raises(rk.RklError) as ei:
        plan.super_step(1e-3, T3, b)
    assert ei.value.status == rk._lib.RKL_ERR_NONFINITE
    # a stage that produces a bad value raises the device status word
    Y = torch.empty_like(T)
    M0 = torch.empty_like(T)
    plan.stage(1, 2, 1e-3, b, T3, M0, None, None, Y)
    assert plan.check() == rk._lib.RKL_ERR_NONFINITE
    assert plan.check() == 0


def test_limiter_plan_kernel_routing(rk, orc):
    """A limiter plan with the floor at +inf runs the row-pair kernel's
    limited build under variant 0 and 10, the paired-cell kernel's under
    every paired-cell variant (the two write the same bits), the tiled
    kernel under variant 2; with a finite floor neither the paired-cell nor
    the row-pair variants apply."""
    params = dict(kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4, limiter="mc")
    shape = (12, 9, 72)
    outs = {}
    for v in (0, 3, 4, 6, 7, 10, 2):
        P, plan, T, b, Td, bd = _setup(rk, "routing", shape, params, "f32", v)
        dt = 100.0 * orc.dt_expl(P, T)
        plan.super_step(dt, Td, bd)
        assert plan.check() == 0
        outs[v] = host(Td)
    for v in (3, 4, 6, 7, 10):
        assert np.array_equal(outs[v], outs[0]), v
    # the tiled kernel's rounding differs, its result agrees within FP32
    assert rel_l2(outs[2], outs[0]) < 1e-6
    P, plan, T, b, Td, bd = _setup(rk, "routing", shape, dict(params, limiter_floor=1.0), "f32", 0)
    for v in (3, 4, 6, 7, 10, 11):
        with pytest.raises(rk.RklError):
            plan.set_variant(v)
