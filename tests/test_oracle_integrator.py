"""Pins for the oracle's RKL2 super-step (Eq. rkl2scheme) and explicit
steps.  No GPU.

The super-step is fixed against: the closed-form Gaussian (Eq.
gaussian_exact) in 1D, along a grid diagonal and in 3D; the matrix
exponential of the linear semi-discrete operator (Eq. ODE) with a measured
second-order temporal rate; the Legendre form of the stability polynomial
applied to that matrix (Eqs. stabpara, recLegP); brute-force forward Euler
on the nonlinear (Spitzer) problem; exact conservation; positivity of every
stage; and the ring test's undershoot without limiters (Section 4.1.3)."""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads
from oracle import Problem


def _gauss_exact(x2, t, sigma, kappa, ndim):
    g = 1 + 2 * kappa * t / sigma ** 2
    return g ** (-ndim / 2) * np.exp(-x2 / (2 * sigma ** 2 * g))


def _run(orc, P, T, b, dt, nsteps, s=0):
    for _ in range(nsteps):
        T, _s = orc.super_step(P, T, b, dt, s)
    return T


def test_gaussian_1d_second_order(orc):
    """Section 4.1.1: kappa = 1, sigma = 0.1 on [-2, 2] (periodic; the tails
    stay below 1e-9 at the boundary up to t_end), super-step tied to the mesh
    as dt/dx = C_p0/(N_0 kappa) with N_0 = 64, C_p0 = 0.45 (Eq.
    gauss_constraint), b along x.  The L1 error of Eq. gauss_emax converges at
    second order."""
    sigma, kappa, t_end = 0.1, 1.0, 0.04
    errs = []
    for n in (128, 256, 512):
        T0, dx, x = workloads.gaussian(n, 1, sigma)
        b = np.zeros((3, n))
        b[0] = 1.0
        P = Problem((n,), dx=(dx,), kappa_par0=kappa)
        dt_target = 0.45 * 4.0 * dx / (64 * kappa)     # dt/dx = C_p0 L/(N_0 kappa), L = 4
        m = max(1, round(t_end / dt_target))
        T = _run(orc, P, T0, b, t_end / m, m)
        errs.append(np.mean(np.abs(T - _gauss_exact(x * x, t_end, sigma, kappa, 1))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 2e-5
    assert 1.8 < rates[-1] < 2.3, (errs, rates)


def test_gaussian_3d_isotropic_product_form(orc):
    """3D isotropic (b = 0, kappa_perp = kappa): the product-form closed
    solution with amplitude (1 + 2 kappa t / sigma^2)^(-3/2), at second order."""
    sigma, kappa, t_end = 0.15, 1.0, 0.01
    errs = []
    for n in (20, 40):
        T0, dx, c = workloads.gaussian(n, 3, sigma, L=2.0)
        b = np.zeros((3,) + T0.shape)
        P = Problem(T0.shape, dx=(dx,) * 3, kappa_par0=kappa, kappa_perp_ratio=1.0)
        ratio = 30.0
        dt = ratio * orc.dt_expl(P, T0)
        m = max(1, math.ceil(t_end / dt))
        T = _run(orc, P, T0, b, t_end / m, m)
        zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
        ex = _gauss_exact(xx ** 2 + yy ** 2 + zz ** 2, t_end, sigma, kappa, 3)
        errs.append(np.max(np.abs(T - ex)))
    assert errs[-1] < 0.06 * _gauss_exact(0.0, t_end, sigma, kappa, 3)
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_gaussian_ridge_along_diagonal(orc):
    """b at 45 degrees to the grid and T a Gaussian ridge in xi = (x+y)/sqrt 2
    (periodised): anisotropic conduction reduces to the 1D law along xi with
    kappa_par, reached at second order through the averaged transverse
    gradients of Eq. qT."""
    sigma, kappa, t_end, L = 0.12, 1.0, 0.006, 2.0
    errs = []
    for n in (32, 64):
        dx = L / n
        c = -L / 2 + (np.arange(n) + 0.5) * dx
        yy, xx = np.meshgrid(c, c, indexing="ij")

        def ridge(t):
            out = np.zeros_like(xx)
            for m in range(-3, 4):
                xi = (xx + yy - m * L) / math.sqrt(2)
                out += _gauss_exact(xi * xi, t, sigma, kappa, 1)
            return out
        T0 = ridge(0.0)
        b = np.zeros((3, n, n))
        b[0] = b[1] = 1 / math.sqrt(2)
        P = Problem((n, n), dx=(dx, dx), kappa_par0=kappa)
        dt = 20.0 * orc.dt_expl(P, T0)
        m = max(1, math.ceil(t_end / dt))
        T = _run(orc, P, T0, b, t_end / m, m)
        errs.append(np.max(np.abs(T - ridge(t_end))))
    assert errs[-1] < 0.01
    assert 1.6 < math.log2(errs[0] / errs[1]) < 2.6, errs


def _linear_problem(n=6, seed=7):
    rng = np.random.default_rng(seed)
    shape = (n, n)
    b = rng.normal(size=(3,) + shape)
    b[2] = 0
    b /= np.sqrt((b ** 2).sum(0))
    P = Problem(shape, kappa_par0=0.8, kappa_perp_ratio=0.05)
    return P, b, rng


def _matrix(orc, P, b):
    N = P.ncell
    A = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        A[:, c] = orc.apply_M(P, e.reshape(P.shape), b).ravel()
    return A


def test_super_step_is_legendre_polynomial_of_operator(orc):
    """For constant kappa M is linear, and Y_s = a_s u + b_s P_s(I + w_1 tau M) u
    (Eq. stabpara) with P_s built by the three-term recursion (Eq. recLegP)."""
    P, b, rng = _linear_problem()
    A = _matrix(orc, P, b)
    u0 = rng.uniform(0.5, 1.5, P.shape)
    lam = np.max(np.abs(np.linalg.eigvals(A)))
    for s in (2, 3, 6, 11):
        w1 = 4.0 / (s * s + s - 2)
        tau = 0.95 * 2.0 / (w1 * lam)
        X = np.eye(A.shape[0]) + w1 * tau * A
        Pm2, Pm1 = np.eye(A.shape[0]), X.copy()
        for j in range(2, s + 1):
            Pm2, Pm1 = Pm1, ((2 * j - 1) / j) * X @ Pm1 - ((j - 1) / j) * Pm2
        bs = (s * s + s - 2) / (2.0 * s * (s + 1))
        want = (1 - bs) * u0.ravel() + bs * (Pm1 @ u0.ravel())
        got, _ = orc.super_step(P, u0, b, tau, s)
        assert np.max(np.abs(got.ravel() - want)) < 1e-12 * np.max(np.abs(want))


def test_temporal_order_against_matrix_exponential(orc):
    """Global error against expm(t M) u0 falls as tau^2 (RKL2 is second order,
    Section 4.1.1)."""
    P, b, rng = _linear_problem()
    A = _matrix(orc, P, b)
    u0 = rng.uniform(0.5, 1.5, P.shape)
    t_end = 0.02
    exact = (scipy.linalg.expm(t_end * A) @ u0.ravel()).reshape(P.shape)
    errs = []
    for m in (2, 4, 8, 16):
        T = _run(orc, P, u0, b, t_end / m, m, s=4)
        errs.append(np.max(np.abs(T - exact)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert 1.85 < rates[-1] < 2.2, (errs, rates)


def test_nonlinear_against_brute_force_euler(orc):
    """Spitzer kappa(T) re-evaluated at every stage: the RKL2 super-step
    approaches many tiny forward-Euler steps (s = 1, Section 3.3) at second
    order in tau."""
    n = 8
    rng = np.random.default_rng(9)
    c = (np.arange(n) + 0.5) / n
    yy, xx = np.meshgrid(c, c, indexing="ij")
    T0 = 1.0 + 0.3 * np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * yy)
    b = rng.normal(size=(3, n, n))
    b[2] = 0
    b /= np.sqrt((b ** 2).sum(0))
    P = Problem((n, n), kappa_model="spitzer", kappa_par0=0.02, kappa_perp_ratio=0.01)
    t_end = 20 * orc.dt_expl(P, T0)
    ref = T0.copy()
    ne = 16000
    for _ in range(ne):
        ref = orc.euler_step(P, ref, b, t_end / ne)
    errs = []
    for m in (4, 8, 16):                  # s = 5 is stable up to dt = 7 dt_expl
        T = _run(orc, P, T0, b, t_end / m, m, s=5)
        errs.append(np.max(np.abs(T - ref)))
    assert errs[-1] < 1e-3 * np.max(np.abs(ref - T0))
    assert math.log2(errs[1] / errs[2]) > 1.7, errs


def test_euler_step_definition(orc):
    P, b, rng = _linear_problem()
    T = rng.uniform(0.5, 1.5, P.shape)
    got = orc.euler_step(P, T, b, 1e-3)
    assert np.allclose(got, T + 1e-3 * orc.apply_M(P, T, b), rtol=0, atol=1e-15)


def test_super_step_conserves_energy_periodic(orc):
    W = workloads.tangled(16, seed=3)
    P = Problem(W.T.shape, **W.params)
    dt = 100 * orc.dt_expl(P, W.T)
    T, s = orc.super_step(P, W.T, W.b, dt)
    assert s == 20
    e0, e1 = orc.energy(P, W.T), orc.energy(P, T)
    assert abs(e1 - e0) <= 1e-13 * abs(e0)
    assert np.max(np.abs(T - W.T)) > 1e-4          # something happened


def test_saturated_super_step_conserves_energy(orc):
    W = workloads.blob(16, seed=3)
    P = Problem(W.T.shape, **W.params)
    dt = 200 * orc.dt_expl(P, W.T)
    T, s = orc.super_step(P, W.T, W.b, dt)
    assert s == 28
    assert abs(orc.energy(P, T) - orc.energy(P, W.T)) <= 1e-13 * orc.energy(P, W.T)


def test_every_stage_stays_positive(orc):
    """RKL stages keep T >= 0 for the Gaussian even at large C_p (Section
    4.1.1), where T falls to ~0 far from the peak."""
    n = 256
    T0, dx, _ = workloads.gaussian(n, 1, 0.05)
    b = np.zeros((3, n))
    b[0] = 1.0
    P = Problem((n,), dx=(dx,), kappa_par0=1.0)
    T = T0
    for ratio in (50, 400, 2000):
        T, s, mn = orc.super_step(P, T, b, ratio * orc.dt_expl(P, T), return_stage_min=True)
        assert mn >= 0.0, (ratio, s, mn)


def test_ring_undershoots_without_limiters(orc):
    """Section 4.1.3: with arithmetic-mean transverse gradients the minimum
    temperature falls below the initial minimum of 10; the hot sector cools
    and heat spreads along the ring (values stay within a bounded band)."""
    W = workloads.ring(100)
    P = Problem(W.T.shape, **W.params)
    dt = W.ratio * orc.dt_expl(P, W.T)
    T = W.T
    for _ in range(10):
        T, s = orc.super_step(P, T, W.b, dt)
    assert s == 14
    assert T.min() < 10.0
    assert T.min() > 9.5
    assert T.max() < 12.0


def test_anisotropic_cells_leave_the_stability_interval(orc):
    """Eq. dt_exp bounds the spectrum by chi sum_d 1/dx_d^2, and RKL2 is
    stable for eigenvalues on [-2/w_1, 0].  With arithmetic-mean transverse
    gradients and a varying field the discrete operator is not symmetric;
    on cubic cells its spectrum stays inside the RKL2 stability region at
    dt = 320 dt_expl (s = 36), but on cells of aspect ratio 6 it does not
    (max |R_s(tau lambda)| > 1): the batched workload therefore uses cubic
    cells (its boxes are bricks of equal cells)."""
    from numpy.polynomial import legendre as npleg
    nx, ny, nz = 36, 6, 12
    T, b = workloads.tangled_box(nx, ny, nz, 7)
    out = {}
    for cubic in (False, True):
        dx = (1.0 / max(nx, ny, nz),) * 3 if cubic else (1.0 / nx, 1.0 / ny, 1.0 / nz)
        P = Problem((nz, ny, nx), dx=dx, kappa_par0=1.0, kappa_perp_ratio=1e-4)
        lam = np.linalg.eigvals(_matrix(orc, P, b))
        ratio = 320.0
        s = orc.num_stages(ratio)
        tau = ratio * orc.dt_expl(P, np.ones(P.shape))
        w1 = 4.0 / (s * s + s - 2)
        bs = (s * s + s - 2) / (2.0 * s * (s + 1))
        R = (1 - bs) + bs * npleg.legval(1 + w1 * tau * lam, [0] * s + [1])
        out[cubic] = float(np.abs(R).max())
    assert out[True] <= 1 + 1e-9
    assert out[False] > 1.2
