"""Pins for the oracle's limited transverse gradients (Appendix C, the
monotonised-central limiter of Sharma & Hammett 2007).  No GPU.

* A linear temperature (all one-sided differences equal) and a smooth field
  (neighbouring differences within a factor of three) give exactly the
  arithmetic-mean gradient of Eq. qT: MC(a, b) = (a + b)/2 there.
* A hand-made stencil fixes the order of the limiting: the two one-sided
  differences of each cell first, then across the two cells (the other
  pairing gives a different number on the same stencil).
* At a transverse extremum the limited gradient vanishes.
* The explicit scheme with the limiter keeps the ring test's minimum at its
  initial value while the unlimited scheme undershoots (Section 4.1.3,
  Appendix C).
* The floor switch: a floor below every temperature is the unlimited
  scheme, an infinite floor limits every face."""
import math

import numpy as np
import pytest

import workloads
from oracle import Problem


def _mc(a, b):
    if a * b <= 0:
        return 0.0
    m = min(abs(a + b) / 2, 2 * abs(a), 2 * abs(b))
    return math.copysign(m, a)


def test_linear_temperature_gives_the_mean_gradient(orc):
    n = 8
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    T = 1.0 + 0.03 * x + 0.02 * y - 0.01 * z
    rng = np.random.default_rng(2)
    b = rng.normal(size=(3, n, n, n))
    b /= np.sqrt((b ** 2).sum(0))
    kw = dict(bc="dirichlet", bc_value=1.0, kappa_model="spitzer", kappa_par0=0.1, kappa_perp_ratio=0.01)
    P0, P1 = Problem((n, n, n), **kw), Problem((n, n, n), limiter="mc", **kw)
    for d in range(3):
        for (i, j, k) in [(3, 3, 3), (2, 4, 5), (4, 2, 3)]:
            a = orc.face_flux(P0, T, b, d, (i, j, k))
            c = orc.face_flux(P1, T, b, d, (i, j, k))
            assert abs(a - c) <= 1e-14 * abs(a)


def test_smooth_field_gives_the_mean_gradient(orc):
    n = 32
    y, x = np.meshgrid(np.arange(n) / n, np.arange(n) / n, indexing="ij")
    T = 1.0 + 0.5 * np.exp(0.3 * x + 0.2 * y)          # monotone, slopes vary slowly
    b = np.stack([np.full((n, n), 0.6), np.full((n, n), 0.8)])
    kw = dict(bc="dirichlet", bc_value=1.0, kappa_par0=0.1)
    P0, P1 = Problem((n, n), **kw), Problem((n, n), limiter="mc", **kw)
    M0, M1 = orc.apply_M(P0, T, b), orc.apply_M(P1, T, b)
    inner = (slice(2, -2), slice(2, -2))
    assert np.max(np.abs(M0[inner] - M1[inner])) <= 1e-11 * np.max(np.abs(M0[inner]))


def test_limiting_order_on_a_hand_made_stencil(orc):
    """x-face between cells L = (1, 2) and R = (2, 2) of a 2D grid; one-sided
    y-differences up_L = 1.0, down_L = 0.2, up_R = down_R = 0.5.  Cell-first
    limiting: MC(MC(1, .2), MC(.5, .5)) = MC(.4, .5) = .45; pairing across
    the cells first would give MC(MC(1, .5), MC(.2, .5)) = .55."""
    ny, nx = 5, 4
    T = np.full((ny, nx), 2.0)
    T[1, 1], T[2, 1], T[3, 1] = 1.8, 2.0, 3.0
    T[1, 2], T[2, 2], T[3, 2] = 2.0, 2.5, 3.0
    b = np.stack([np.full((ny, nx), 1 / math.sqrt(2)), np.full((ny, nx), 1 / math.sqrt(2))])
    kappa, dx, dy = 0.7, 0.25, 0.2
    P = Problem((ny, nx), dx=(dx, dy), kappa_par0=kappa, limiter="mc")
    Fx = orc.face_flux(P, T, b, 0, (1, 2))
    gx = (T[2, 2] - T[2, 1]) / dx
    gy = -2.0 * Fx / kappa - gx            # F_x = -kappa/2 (g_x + g_y) for b at 45 degrees
    want = _mc(_mc(1.0, 0.2), _mc(0.5, 0.5)) / dy
    assert abs(want - 0.45 / dy) < 1e-15
    assert abs(gy - want) < 1e-12 * abs(want)
    other = _mc(_mc(1.0, 0.5), _mc(0.2, 0.5)) / dy
    assert abs(gy - other) > 0.05 / dy


def test_transverse_extremum_has_zero_limited_gradient(orc):
    ny, nx = 6, 4
    yy = np.arange(ny)[:, None] * np.ones((1, nx))
    T = 1.0 + 0.1 * (yy - 2.0) ** 2 + 0.05 * np.arange(nx)[None, :]     # minimum in y at row 2
    b = np.stack([np.full((ny, nx), 0.6), np.full((ny, nx), 0.8)])
    kappa, dx = 0.5, 0.1
    P = Problem((ny, nx), dx=(dx, dx), kappa_par0=kappa, limiter="mc", bc="dirichlet", bc_value=1.0)
    Fx = orc.face_flux(P, T, b, 0, (1, 2))
    gx = (T[2, 2] - T[2, 1]) / dx
    assert abs(Fx - (-kappa * 0.6 * 0.6 * gx)) < 1e-14


def test_limiter_keeps_the_ring_minimum(orc):
    """40 x 40 ring, 400 forward-Euler steps at C_p = 1/4: the unlimited
    scheme undershoots the initial minimum T = 10, the limited one does not."""
    W = workloads.ring(40)
    mins = {}
    for lim in ("none", "mc"):
        P = Problem(W.T.shape, limiter=lim, **W.params)
        T = W.T.copy()
        dt = 0.5 * orc.dt_expl(P, T)
        for _ in range(400):
            T = orc.euler_step(P, T, W.b, dt)
        mins[lim] = T.min()
        assert T.max() <= 12.0
    assert mins["none"] < 10.0 - 1e-3
    assert mins["mc"] >= 10.0 - 1e-12


def test_floor_switch(orc):
    rng = np.random.default_rng(9)
    shape = (10, 12, 8)
    T = 10.0 + 2.0 * rng.random(shape)
    b = rng.normal(size=(3,) + shape)
    b /= np.sqrt((b ** 2).sum(0))
    kw = dict(kappa_par0=0.05)
    M_none = orc.apply_M(Problem(shape, **kw), T, b)
    M_low = orc.apply_M(Problem(shape, limiter="mc", limiter_floor=5.0, **kw), T, b)
    M_all = orc.apply_M(Problem(shape, limiter="mc", **kw), T, b)
    M_mid = orc.apply_M(Problem(shape, limiter="mc", limiter_floor=11.0, **kw), T, b)
    assert np.array_equal(M_low, M_none)
    assert not np.allclose(M_all, M_none)
    assert not np.allclose(M_mid, M_none) and not np.allclose(M_mid, M_all)
