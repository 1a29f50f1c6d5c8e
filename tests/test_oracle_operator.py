"""Pins for the oracle's conduction operator M(T) = -div F (Section 3; Eqs.
Fclass, Fclass_HD, Fc, Fsat; Appendix B Eqs. qN, qT).  No GPU.

Each test fixes the operator against something other than itself: textbook
finite-difference Laplacians (isotropic and field-aligned special cases),
second-order convergence to the exact divergence of a manufactured smooth
solution (derived symbolically), exact conservation, and the saturation
limits of Eq. Fc."""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import Problem


def _lap_periodic(T, dx):
    """Textbook second-order Laplacian on a periodic grid ([z][y][x] axes)."""
    out = np.zeros_like(T)
    nd = T.ndim
    for ax in range(nd):
        h = dx[nd - 1 - ax]
        out += (np.roll(T, -1, ax) - 2 * T + np.roll(T, 1, ax)) / (h * h)
    return out


@pytest.mark.parametrize("shape", [(17,), (9, 12), (6, 7, 8)])
def test_isotropic_operator_is_textbook_laplacian(orc, shape):
    """b = 0 and kappa_perp = kappa: F = -kappa grad T (Eq. Fclass_HD), so M
    is kappa times the standard 2*ndim+1 point Laplacian."""
    rng = np.random.default_rng(1)
    T = rng.uniform(0.5, 1.5, shape)
    b = np.zeros((3,) + shape)
    dx = tuple(0.1 * (d + 1) for d in range(len(shape)))
    P = Problem(shape, dx=dx, kappa_par0=0.7, kappa_perp_ratio=1.0)
    got = orc.apply_M(P, T, b)
    want = 0.7 * _lap_periodic(T, dx)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_dirichlet_1d_isotropic_uses_ghost_value(orc):
    """1D with Dirichlet ghosts T = bc_value at both ends: M is the second
    difference with the ghost values substituted."""
    rng = np.random.default_rng(2)
    T = rng.uniform(0.0, 1.0, 13)
    dx = 0.05
    P = Problem((13,), dx=(dx,), bc="dirichlet", bc_value=0.25, kappa_par0=2.0,
                kappa_perp_ratio=1.0)
    got = orc.apply_M(P, T, np.zeros((3, 13)))
    Tg = np.concatenate([[0.25], T, [0.25]])
    want = 2.0 * (Tg[2:] - 2 * Tg[1:-1] + Tg[:-2]) / dx ** 2
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    # a uniform T equal to the ghost value is a steady state
    assert np.max(np.abs(orc.apply_M(P, np.full(13, 0.25), np.zeros((3, 13))))) == 0.0


def test_field_along_x_gives_1d_diffusion(orc):
    """b = x-hat, kappa_perp = 0: F_x = -kappa b_x^2 dT/dx, the transverse
    terms vanish (Eqs. qN, qT), so M is the x second difference only."""
    rng = np.random.default_rng(3)
    shape = (5, 6, 7)
    T = rng.uniform(0.5, 1.5, shape)
    b = np.zeros((3,) + shape)
    b[0] = 1.0
    dx = (0.1, 0.2, 0.3)
    P = Problem(shape, dx=dx, kappa_par0=1.3)
    got = orc.apply_M(P, T, b)
    want = 1.3 * (np.roll(T, -1, 2) - 2 * T + np.roll(T, 1, 2)) / 0.01
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_transverse_gradient_stencil_on_linear_field(orc):
    """For T linear in y and uniform b at 45 degrees in xy, the x-face flux is
    -kappa b_x (b_x dT/dx + b_y dT/dy) with the transverse gradient exact,
    away from the periodic seam (Eq. qT averaged to the face)."""
    ny, nx = 12, 10
    dx, dy = 0.1, 0.2
    y = (np.arange(ny) + 0.5) * dy
    x = (np.arange(nx) + 0.5) * dx
    T = 3.0 * y[:, None] + 0.5 * x[None, :]
    b = np.zeros((3, ny, nx))
    b[0] = b[1] = 1 / math.sqrt(2)
    P = Problem((ny, nx), dx=(dx, dy), kappa_par0=0.9)
    Fx, Fy = orc.flux(P, T, b)
    want_x = -0.9 * 0.5 * (0.5 + 3.0)
    want_y = -0.9 * 0.5 * (0.5 + 3.0)
    inner = (slice(2, ny - 2), slice(2, nx - 2))
    assert np.allclose(Fx[inner], want_x, rtol=1e-13)
    assert np.allclose(Fy[inner], want_y, rtol=1e-13)


def _manufactured(ndim, saturate, spitzer, kperp):
    xs = sp.symbols("x y z")[:ndim]
    two_pi = 2 * sp.pi
    if ndim == 2:
        x, y = xs
        T = 1 + sp.Rational(1, 5) * sp.sin(two_pi * x) * sp.cos(two_pi * y) + sp.Rational(1, 10) * sp.sin(two_pi * y + 1)
        B = [sp.Rational(6, 5) + sp.sin(two_pi * y), sp.Rational(4, 5) + sp.cos(two_pi * x) / 2, 0]
    else:
        x, y, z = xs
        T = (1 + sp.Rational(1, 5) * sp.sin(two_pi * x) * sp.cos(two_pi * y)
             + sp.Rational(1, 10) * sp.sin(two_pi * z + 1) + sp.Rational(1, 20) * sp.cos(two_pi * (x - z)))
        B = [sp.Rational(6, 5) + sp.sin(two_pi * y), sp.Rational(4, 5) + sp.cos(two_pi * z) / 2,
             sp.Rational(3, 5) + sp.sin(two_pi * x) * sp.Rational(2, 5)]
    Bm = sp.sqrt(sum(c * c for c in B))
    b = [c / Bm for c in B]
    k0 = sp.Rational(3, 10)
    kpar = k0 * T ** sp.Rational(5, 2) if spitzer else k0
    kperp_ = kperp * kpar
    grad = [sp.diff(T, v) for v in xs] + [0] * (3 - ndim)
    bdg = sum(b[e] * grad[e] for e in range(3))
    F = [-kpar * b[e] * bdg - kperp_ * grad[e] for e in range(3)]
    if saturate:
        phi = sp.Rational(1, 50)
        q = 5 * phi * T ** sp.Rational(3, 2)
        Fm = sp.sqrt(sum(f * f for f in F))
        F = [q / (q + Fm) * f for f in F]
    M = -sum(sp.diff(F[e], xs[e]) for e in range(ndim))
    fT = sp.lambdify(xs, T, "numpy")
    fb = [sp.lambdify(xs, c, "numpy") for c in b]
    fM = sp.lambdify(xs, M, "numpy")
    return fT, fb, fM


@pytest.mark.parametrize("ndim,saturate,spitzer,kperp", [
    (2, False, False, 0.0),
    (2, False, True, 0.01),
    (2, True, True, 0.0),
    (3, False, True, 1e-2),
    (3, True, True, 0.0),
])
def test_manufactured_solution_second_order(orc, ndim, saturate, spitzer, kperp):
    """M_h(T) converges to the exact -div F of a smooth periodic T and b at
    second order (central differences, Section 3): a wrong sign, index,
    factor or missing term leaves an O(1) error instead.  With saturation
    the blend q F/(q + |F|) has a kink in its second derivative wherever F
    changes sign, so there only the L2 error is required to converge (at
    better than first order)."""
    fT, fb, fM = _manufactured(ndim, saturate, spitzer, kperp)
    errs = []
    sizes = (16, 32, 64) if ndim == 2 else (12, 24, 48)
    for n in sizes:
        c = (np.arange(n) + 0.5) / n
        grids = np.meshgrid(*([c] * ndim), indexing="ij")     # [z][y][x] order
        xyz = list(reversed(grids))                           # x, y, (z)
        T = np.broadcast_to(fT(*xyz), (n,) * ndim).astype(np.float64)
        b = np.stack([np.broadcast_to(f(*xyz), (n,) * ndim) for f in fb])
        want = np.broadcast_to(fM(*xyz), (n,) * ndim)
        P = Problem((n,) * ndim, kappa_model="spitzer" if spitzer else "const",
                    kappa_par0=0.3, kappa_perp_ratio=kperp, saturate=saturate, phi=0.02)
        got = orc.apply_M(P, T, b)
        if saturate:
            errs.append(np.sqrt(np.mean((got - want) ** 2) / np.mean(want ** 2)))
        else:
            errs.append(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    if saturate:
        assert errs[-1] < 0.07
        assert all(r > 1.0 for r in rates), (errs, rates)
    else:
        assert errs[-1] < 0.05
        assert 1.7 < rates[-1] < 2.4, (errs, rates)


@pytest.mark.parametrize("saturate,upwind", [(False, False), (True, False), (True, True)])
def test_periodic_conservation(orc, saturate, upwind):
    """One flux per face (Section 3): sum_c M(T)_c dV = 0 on a periodic grid."""
    rng = np.random.default_rng(4)
    shape = (7, 9, 11)
    T = rng.uniform(0.5, 2.0, shape)
    b = rng.normal(size=(3,) + shape)
    b /= np.sqrt((b ** 2).sum(0))
    P = Problem(shape, kappa_model="spitzer", kappa_par0=0.05, kappa_perp_ratio=1e-3,
                saturate=saturate, phi=0.05, sat_upwind=upwind)
    M = orc.apply_M(P, T, b)
    assert abs(M.sum()) <= 1e-13 * np.abs(M).sum()


def test_saturation_limits(orc):
    """Eq. Fc: kappa -> infinity gives |F| -> q = 5 phi rho c_iso^3 down the
    gradient; q -> infinity (phi large) gives back the classical flux."""
    n = 16
    T = 1.0 + 0.5 * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n)
    b = np.zeros((3, n))
    b[0] = 1.0
    Pc = Problem((n,), kappa_par0=0.2)
    Fc = orc.flux(Pc, T, b)[0]
    Pq = Problem((n,), kappa_par0=0.2, saturate=True, phi=1e12)
    assert np.allclose(orc.flux(Pq, T, b)[0], Fc, rtol=1e-10, atol=0)
    Pk = Problem((n,), kappa_par0=1e12, saturate=True, phi=0.3, rho=1.7)
    Fk = orc.flux(Pk, T, b)[0]
    Tf = 0.5 * (T + np.roll(T, -1))
    q = 5 * 0.3 * 1.7 * Tf ** 1.5
    sgn = -np.sign(np.roll(T, -1) - T)
    assert np.allclose(Fk, q * sgn, rtol=1e-9)
    # upwind variant: q from the cell the heat leaves
    Pu = Problem((n,), kappa_par0=1e12, saturate=True, phi=0.3, rho=1.7, sat_upwind=True)
    Fu = orc.flux(Pu, T, b)[0]
    Tup = np.where(sgn > 0, T, np.roll(T, -1))
    assert np.allclose(Fu, 5 * 0.3 * 1.7 * Tup ** 1.5 * sgn, rtol=1e-9)


def test_dt_expl_closed_form(orc):
    """Eq. dt_exp with chi_d = kappa_par + kappa_perp, gamma = 2, rho = 1."""
    rng = np.random.default_rng(5)
    shape = (4, 5, 6)
    T = rng.uniform(0.8, 1.2, shape)
    dx = (0.1, 0.2, 0.4)
    inv = sum(1 / h ** 2 for h in dx)
    P = Problem(shape, dx=dx, kappa_par0=0.3, kappa_perp_ratio=0.1)
    assert orc.dt_expl(P, T) == pytest.approx(0.5 / (0.3 * 1.1 * inv), rel=1e-14)
    Ps = Problem(shape, dx=dx, kappa_model="spitzer", kappa_par0=0.3, kappa_perp_ratio=0.1, cp=0.4)
    assert orc.dt_expl(Ps, T) == pytest.approx(0.4 / (0.3 * T.max() ** 2.5 * 1.1 * inv), rel=1e-13)
