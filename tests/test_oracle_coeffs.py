"""Pins for the oracle's stage count and RKL2 coefficients (Appendix A,
Eq. RKL-s, Eq. stabpara, Eq. recLegP).  No GPU."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rkl2_s3_appendixA.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = Fraction(v)
    return out


def test_s3_coefficients_match_appendix_a(orc):
    g = _golden()
    mu, nu, mut, gt = orc.coeffs(3)
    for j in (2, 3):
        assert mu[j] == pytest.approx(float(g[f"mu_{j}"]), rel=1e-15, abs=1e-15)
        assert nu[j] == pytest.approx(float(g[f"nu_{j}"]), rel=1e-15, abs=1e-15)
        assert mut[j] == pytest.approx(float(g[f"mut_{j}"]), rel=1e-15, abs=1e-15)
        assert gt[j] == pytest.approx(float(g[f"gt_{j}"]), rel=1e-15, abs=1e-15)
    assert mut[1] == pytest.approx(float(g["mut_1"]), rel=1e-15)
    assert 1 - mu[3] - nu[3] == pytest.approx(float(g["c0_3"]), rel=1e-14)


def test_s3_stability_polynomial_is_printed_cubic(orc):
    g = _golden()
    for z in np.linspace(-5.0, 0.5, 23):
        want = sum(float(g[f"R3_{p}"]) * z ** p for p in range(4))
        assert orc.rkl2_scalar(3, z) == pytest.approx(want, rel=1e-14, abs=1e-14)
    # the printed Legendre form 7/12 + 5/12 P_3(1 + 2/5 z)
    for z in np.linspace(-5.0, 0.0, 11):
        want = float(g["a_3"]) + float(g["b_3"]) * npleg.legval(1 + float(g["w1"]) * z, [0, 0, 0, 1])
        assert orc.rkl2_scalar(3, z) == pytest.approx(want, rel=1e-14, abs=1e-14)
    # the printed interval -5 <= tau*lambda <= 0 is where the Legendre
    # argument 1 + w_1 z stays in [-1, 1]; |R_3| <= 1 on all of it
    zmin = float(g["zmin_3"])
    assert 1 + float(g["w1"]) * zmin == pytest.approx(-1.0, abs=1e-15)
    for z in np.linspace(zmin, 0.0, 101):
        assert abs(orc.rkl2_scalar(3, z)) <= 1 + 1e-14


@pytest.mark.parametrize("s", [2, 3, 4, 5, 9, 14, 20, 28, 40, 64])
def test_recurrence_reproduces_legendre_stability_polynomial(orc, s):
    """Y_s of the scalar recurrence equals a_s + b_s P_s(1 + w_1 z) (Eq.
    stabpara) with P_s from numpy's Legendre series, on the whole stability
    interval, and |R_s| <= 1 there (tau |lambda| <= 2 / w_1)."""
    w1 = 4.0 / (s * s + s - 2)
    bs = (s * s + s - 2) / (2.0 * s * (s + 1))
    cs = [0] * s + [1]
    zs = np.linspace(-2.0 / w1, 0.0, 257)
    got = np.array([orc.rkl2_scalar(s, z) for z in zs])
    want = (1 - bs) + bs * npleg.legval(1 + w1 * zs, cs)
    assert np.max(np.abs(got - want)) < 1e-12
    assert np.max(np.abs(got)) <= 1 + 1e-12


@pytest.mark.parametrize("s", [2, 3, 7, 16, 33])
def test_second_order_taylor_match(orc, s):
    """R_s(0) = 1, R_s'(0) = 1, R_s''(0) = 1 (Appendix A), from an exact
    polynomial interpolation of the recurrence at s + 1 small nodes."""
    h = 1e-2
    zs = h * np.cos(np.pi * (np.arange(s + 1) + 0.5) / (s + 1))
    vals = [orc.rkl2_scalar(s, z) for z in zs]
    p = np.polynomial.Polynomial.fit(zs, vals, s, domain=[-h, h], window=[-h, h])
    c = p.coef
    assert c[0] == pytest.approx(1.0, abs=1e-12)
    assert c[1] == pytest.approx(1.0, abs=1e-9)
    assert 2 * c[2] == pytest.approx(1.0, abs=1e-6)


def test_legendre_identities_used_by_appendix_a():
    """P_s(1) = 1, P_s'(1) = s(s+1)/2, P_s''(1) = ((s^2+s-2)/4) P_s'(1), so
    b_s = P''/P'^2 and w_1 = P'/P'' take the closed forms the oracle uses."""
    for s in range(2, 65):
        cs = [0] * s + [1]
        p1 = npleg.legval(1.0, cs)
        d1 = npleg.legval(1.0, npleg.legder(cs, 1))
        d2 = npleg.legval(1.0, npleg.legder(cs, 2))
        assert p1 == pytest.approx(1.0, rel=1e-12)
        assert d1 == pytest.approx(s * (s + 1) / 2, rel=1e-12)
        assert d2 == pytest.approx((s * s + s - 2) / 4 * d1, rel=1e-10)
        assert d2 / d1 ** 2 == pytest.approx((s * s + s - 2) / (2 * s * (s + 1)), rel=1e-10)
        assert d1 / d2 == pytest.approx(4.0 / (s * s + s - 2), rel=1e-10)


def test_coefficients_exact_rationals(orc):
    """All coefficients against exact rational arithmetic of the Appendix A
    formulas for s up to 40 (independent of the oracle's floating point)."""
    for s in (2, 3, 4, 9, 20, 40):
        w1 = Fraction(4, s * s + s - 2)
        b = [Fraction(1, 3)] * 3 + [Fraction(j * j + j - 2, 2 * j * (j + 1)) for j in range(3, s + 1)]
        mu, nu, mut, gt = orc.coeffs(s)
        assert mut[1] == pytest.approx(float(b[1] * w1), rel=1e-15)
        for j in range(2, s + 1):
            m = Fraction(2 * j - 1, j) * b[j] / b[j - 1]
            n = -Fraction(j - 1, j) * b[j] / b[j - 2]
            assert mu[j] == pytest.approx(float(m), rel=1e-15)
            assert nu[j] == pytest.approx(float(n), rel=1e-15)
            assert mut[j] == pytest.approx(float(m * w1), rel=1e-15)
            assert gt[j] == pytest.approx(float(-(1 - b[j - 1]) * m * w1), rel=1e-14)


@pytest.mark.parametrize("ratio,s", [(20, 9), (50, 14), (100, 20), (200, 28), (400, 40)])
def test_num_stages_known(orc, ratio, s):
    assert orc.num_stages(ratio) == s


def test_num_stages_brute_force(orc):
    """s is the integer after the real root of dt/dt_p = (s^2+s-2)/4 (Eq.
    RKL-s, rounded by s -> 1 + floor(s)): checked against a direct search
    for the largest integer s' with (s'^2+s'-2)/4 <= ratio."""
    rng = np.random.default_rng(0)
    for ratio in np.concatenate([rng.uniform(0.01, 2000, 400), [1.0, 2.5, 5.0, 7.0, 10.0]]):
        sp = 1
        while ((sp + 1) ** 2 + (sp + 1) - 2) / 4.0 <= ratio:
            sp += 1
        assert orc.num_stages(ratio) == sp + 1
        s = orc.num_stages(ratio)
        # the chosen s is stable for this super-step: (s^2+s-2)/4 > ratio
        assert (s * s + s - 2) / 4.0 > ratio


def test_effective_cfl_asymptote(orc):
    """C_p = dt/(2 dt_p) -> s^2/8 for large s (RKL-2 limit in Section 3.3)."""
    for s in (50, 100, 400):
        ratio = (s * s + s - 2) / 4.0
        assert ratio / 2 / (s * s / 8.0) == pytest.approx(1.0, rel=3.0 / s)


@pytest.mark.parametrize("s", [2, 9, 20, 28, 40])
def test_stage_perturbations_grow_most_on_undamped_modes(orc, s):
    """The FP32 error model of the GPU tests propagates a perturbation of
    stage k by the homogeneous recurrence of Eq. rkl2scheme at z = tau lambda
    = 0.  On an eigenmode with z in the real stability interval
    [-(s^2+s-2)/2, 0] the recurrence is e_j = (mu_j + mu~_j z) e_{j-1} +
    nu_j e_{j-2}: its reach |e_s| never exceeds the z = 0 value A_k(s)."""
    import numpy as np
    from gpu_util import stage_amplification
    mu, nu, mut, _ = orc.coeffs(s)
    A = stage_amplification(orc, s)
    zs = -np.linspace(0.0, (s * s + s - 2) / 2.0, 801)
    for k in range(1, s + 1):
        e = np.zeros((s + 1, zs.size))
        e[k] = 1.0
        for j in range(k + 1, s + 1):
            e[j] = (mu[j] + mut[j] * zs) * e[j - 1] + nu[j] * e[j - 2]
        assert np.max(np.abs(e[s])) <= A[k - 1] * (1 + 1e-12), k
    assert A[-1] == 1.0
