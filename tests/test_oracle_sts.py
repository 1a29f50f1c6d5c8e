"""Pins for the oracle's first-order super-time-steppers of Section 3.3:
RKL1 and AAG-STS.  No GPU.

* RKL1: the scalar amplification factor equals the Legendre polynomial
  P_s(1 + w1 z) with w1 = 2/(s^2 + s) (Eq. stabpara with a_s = 0, b_s = 1)
  evaluated by numpy's Legendre series, is bounded by 1 on the stability
  interval, and matches the Taylor series to first order only; on the linear
  semi-discrete operator the super-step equals that polynomial of the matrix,
  evaluated through its eigen-decomposition; the stage count inverts Eq.
  RKL-s.
* AAG-STS: the sub-steps sum to the super-step of Eq. AAG-STS, their
  reciprocals follow the cosine law, the gain has the two limits of Eq.
  STS-limit, and the amplification factor stays within 1 on the explicit
  stability interval.
* Both converge at first order in time against the matrix exponential
  (Section 4.1.1) and conserve energy with periodic boundaries."""
import math

import numpy as np
import pytest
import scipy.linalg
from numpy.polynomial import legendre

from oracle import Problem


def _legendre_P(s, x):
    return legendre.legval(x, [0.0] * s + [1.0])


@pytest.mark.parametrize("s", [2, 3, 5, 10, 17, 40])
def test_rkl1_scalar_is_shifted_legendre(orc, s):
    w1 = 2.0 / (s * s + s)
    zs = np.linspace(-2.0 / w1, 0.0, 301)
    got = np.array([orc.rkl1_scalar(s, z) for z in zs])
    want = _legendre_P(s, 1.0 + w1 * zs)
    assert np.max(np.abs(got - want)) < 1e-12
    assert np.max(np.abs(got)) <= 1.0 + 1e-12
    # Taylor terms: R(0) = 1, R'(0) = 1, R''(0) = 2 * (s-1)(s+2) / (4 s (s+1)) != 1
    h = 1e-4
    d1 = (orc.rkl1_scalar(s, h) - orc.rkl1_scalar(s, -h)) / (2 * h)
    d2 = (orc.rkl1_scalar(s, h) - 2 * orc.rkl1_scalar(s, 0.0) + orc.rkl1_scalar(s, -h)) / h ** 2
    assert abs(orc.rkl1_scalar(s, 0.0) - 1.0) < 1e-14
    assert abs(d1 - 1.0) < 1e-7
    assert abs(d2 - (s - 1) * (s + 2) / (2.0 * s * (s + 1))) < 1e-5


@pytest.mark.parametrize("ratio", [0.3, 1.0, 2.9, 3.0, 10.0, 50.0, 100.0, 1234.5])
def test_rkl1_stage_count_inverts_eq_rkl_s(orc, ratio):
    s = orc.num_stages_rkl1(ratio)
    # 1 + floor(x) with (x^2 + x)/2 = ratio: the previous count falls short
    assert (s - 1) * s / 2.0 <= ratio < (s * s + s) / 2.0


def _linear_problem(n=6, seed=11):
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


def test_rkl1_super_step_is_legendre_polynomial_of_operator(orc):
    """Y_s = P_s(I + w1 tau M) u0, evaluated on the eigen-decomposition of M
    with numpy's Legendre series (complex eigenvalues included)."""
    P, b, rng = _linear_problem()
    A = _matrix(orc, P, b)
    u0 = rng.uniform(0.5, 1.5, P.shape)
    lam, V = np.linalg.eig(A)
    Vinv = np.linalg.inv(V)
    for s in (2, 4, 9):
        w1 = 2.0 / (s * s + s)
        tau = 0.9 * 2.0 / (w1 * np.max(np.abs(lam)))
        want = (V @ (legendre.legval(1.0 + w1 * tau * lam, [0.0] * s + [1.0]) * (Vinv @ u0.ravel()))).real
        got, _ = orc.rkl1_super_step(P, u0, b, tau, s)
        assert np.max(np.abs(got.ravel() - want)) < 1e-10 * np.max(np.abs(want)), s


@pytest.mark.parametrize("N,nu", [(1, 1e-3), (2, 0.05), (5, 1e-3), (10, 1e-3), (33, 1e-2), (64, 1e-4)])
def test_sts_substeps_sum_to_eq_aag_sts(orc, N, nu):
    """The sub-steps of a super-step dt sum to dt, and dt / dt_p is the
    closed form of Eq. AAG-STS: the reciprocal sub-steps follow
    dt_p / tau_j = (nu - 1) cos((2j - 1) pi / 2N) + 1 + nu with a single dt_p."""
    dt = 0.37
    tau = orc.sts_substeps(N, nu, dt)
    assert abs(tau.sum() - dt) < 1e-12 * dt
    assert np.all(tau > 0)
    j = np.arange(1, N + 1)
    dtp = tau * ((nu - 1.0) * np.cos((2 * j - 1) * np.pi / (2 * N)) + 1.0 + nu)
    assert np.max(np.abs(dtp - dtp[0])) < 1e-12 * dtp[0]
    r = math.sqrt(nu)
    gain = N / (2 * r) * ((1 + r) ** (2 * N) - (1 - r) ** (2 * N)) / ((1 + r) ** (2 * N) + (1 - r) ** (2 * N))
    assert abs(dt / dtp[0] - gain) < 1e-11 * gain
    assert abs(orc.sts_gain(N, nu) - gain) < 1e-12 * gain


def test_sts_gain_limits_of_eq_sts_limit(orc):
    """Gain ~ N^2 (C_p ~ N^2/2) while N sqrt(nu) << 1, ~ N/(2 sqrt(nu)) beyond."""
    nu = 1e-6
    for N in (2, 5, 10):                          # N sqrt(nu) <= 0.01
        assert abs(orc.sts_gain(N, nu) / N ** 2 - 1) < 1e-3
    nu = 1e-2
    for N in (200, 500):                          # N sqrt(nu) >= 20
        assert abs(orc.sts_gain(N, nu) * 2 * math.sqrt(nu) / N - 1) < 1e-9


@pytest.mark.parametrize("ratio,nu", [(0.5, 1e-3), (1.0, 1e-3), (50.0, 1e-3), (400.0, 1e-2), (30.0, 0.1)])
def test_sts_stage_count_is_smallest(orc, ratio, nu):
    N = orc.num_stages_sts(ratio, nu)
    assert orc.sts_gain(N, nu) >= ratio
    assert N == 1 or orc.sts_gain(N - 1, nu) < ratio


@pytest.mark.parametrize("N,nu", [(4, 1e-3), (12, 1e-3), (30, 1e-2)])
def test_sts_amplification_bounded_on_explicit_interval(orc, N, nu):
    """prod_j (1 + tau_j lambda) stays within [-1, 1] for lambda dt_p in [-2, 0]."""
    g = orc.sts_gain(N, nu)
    tau = orc.sts_substeps(N, nu, g)               # dt_p = 1
    z = np.linspace(-2.0, 0.0, 20001)
    R = np.ones_like(z)
    for t in tau:
        R *= 1.0 + t * z
    assert np.max(np.abs(R)) <= 1.0 + 1e-12


def test_first_order_in_time_against_matrix_exponential(orc):
    """Section 4.1.1: RKL1 and AAG-STS are first order (global error halves
    with the super-step)."""
    P, b, rng = _linear_problem()
    A = _matrix(orc, P, b)
    u0 = rng.uniform(0.5, 1.5, P.shape)
    t_end = 0.05
    exact = (scipy.linalg.expm(t_end * A) @ u0.ravel()).reshape(P.shape)
    for step in ("rkl1", "sts"):
        errs = []
        for m in (4, 8, 16, 32):
            T = u0.copy()
            for _ in range(m):
                if step == "rkl1":
                    T, _ = orc.rkl1_super_step(P, T, b, t_end / m, 4)
                else:
                    T, _ = orc.sts_super_step(P, T, b, t_end / m, 1e-3, 4)
            errs.append(np.max(np.abs(T - exact)))
        rate = math.log2(errs[-2] / errs[-1])
        assert 0.9 < rate < 1.15, (step, errs)


def test_first_order_steppers_conserve_energy(orc):
    n = 12
    rng = np.random.default_rng(5)
    b = rng.normal(size=(3, n, n, n))
    b /= np.sqrt((b ** 2).sum(0))
    T0 = 1.0 + 0.3 * rng.random((n, n, n))
    P = Problem((n, n, n), kappa_model="spitzer", kappa_par0=0.05, kappa_perp_ratio=1e-3)
    dt = 20 * orc.dt_expl(P, T0)
    e0 = orc.energy(P, T0)
    T1, s = orc.rkl1_super_step(P, T0, b, dt)
    assert s == orc.num_stages_rkl1(20.0)
    assert abs(orc.energy(P, T1) - e0) < 1e-13 * abs(e0)
    T2, N = orc.sts_super_step(P, T0, b, dt, 1e-3)
    assert N == orc.num_stages_sts(20.0, 1e-3)
    assert abs(orc.energy(P, T2) - e0) < 1e-13 * abs(e0)
    assert np.all(np.isfinite(T1)) and np.all(np.isfinite(T2))
