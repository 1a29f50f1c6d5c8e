"""Exactness of the algebraic rewrites the paired-cell stage kernel uses,
restated in numpy at the kernel's precision and checked against the
definitions they replace.  No GPU.

* MC limiter (Appendix C): the kernel carries half slopes, with
  MC(a, b) / 2 = sign(a) min(|a + b| / 4, |a|, |b|) for a b > 0 (else 0),
  and takes a face's limited gradient as 4 * half(sL / 2, sR / 2).  Both
  factors 2 are powers of two, so in FP32 the results must be bit-identical
  to MC(a, b) = sign(a) min(|a + b| / 2, 2|a|, 2|b|) and MC(sL, sR).
* Saturated flux (Eqs. Fc, Fsat), q at the face temperature: with
  Ts = T_L + T_R, F = nk Ts^2.5 V (Spitzer) and q = q0 (Ts / 2)^1.5, the
  blend F q / (q + |F|) equals nk Ts^2.5 X / (1 + s Ts |V|) with
  s = -nk / (q0 2^-1.5) (and Ts^1.5 X / (Ts^1.5 + s |V|) for a constant
  kappa); checked in FP64 to rounding."""
import numpy as np

f32 = np.float32


def _mc_direct(a, b):
    m = np.minimum(np.minimum(np.abs(f32(0.5) * (a + b)), f32(2) * np.abs(a)), f32(2) * np.abs(b))
    return np.where(a * b <= 0, f32(0), np.where(a > 0, m, -m)).astype(np.float32)


def _mc_half(a, b):
    m = np.minimum(f32(0.25) * np.abs(a + b), np.minimum(np.abs(a), np.abs(b)))
    return np.where(a * b > 0, np.copysign(m, a), f32(0)).astype(np.float32)


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-6, 3, size=n)
    a = (rng.normal(size=n) * mag).astype(np.float32)
    b = (rng.normal(size=n) * mag * 10.0 ** rng.uniform(-2, 2, size=n)).astype(np.float32)
    # equal, opposite, zero and one-sided pairs
    a[:8] = [1, 1, -1, 0, 2, -3, 1e-3, 5]
    b[:8] = [1, -1, -1, 1, 0, -3, 3e-3, 1e-2]
    return a, b


def test_half_limit_is_exactly_half_the_limit_in_fp32():
    a, b = _samples(400_000, 1)
    ref = _mc_direct(a, b)
    half = _mc_half(a, b)
    assert np.array_equal(f32(2) * half, ref)
    # a hand-checked value: MC(1, 3) = min(2, 2, 6) = 2
    assert _mc_direct(np.array([1], np.float32), np.array([3], np.float32))[0] == 2.0


def test_face_limit_of_half_slopes_matches_the_limit_of_slopes():
    # per-cell slopes as the kernel forms them from one-sided differences
    uL, dL = _samples(200_000, 2)
    uR, dR = _samples(200_000, 3)
    sL, sR = _mc_direct(uL, dL), _mc_direct(uR, dR)
    ref = _mc_direct(sL, sR)
    hL, hR = _mc_half(uL, dL), _mc_half(uR, dR)
    assert np.array_equal(hL, sL * f32(0.5)) and np.array_equal(hR, sR * f32(0.5))
    got = f32(4) * _mc_half(hL, hR)
    assert np.array_equal(got, ref)
    # times 1/dx: (4 m) / dx and m (4 / dx) round alike
    inv_dx = f32(1.0 / 3.0)
    assert np.array_equal(_mc_half(hL, hR) * (f32(4) * inv_dx), ref * inv_dx)


def _sat_direct(nk, q0, Ts, X, Y1, Y2, spitzer):
    k = nk * (Ts ** 2.5 if spitzer else 1.0)
    F = k * X
    Fmag = np.abs(k) * np.sqrt(X * X + Y1 * Y1 + Y2 * Y2)
    q = q0 * (Ts / 2.0) ** 1.5
    return F * q / (q + Fmag)


def _sat_cancelled(nk, q0, Ts, X, Y1, Y2, spitzer):
    s = -nk / (q0 * 2.0 ** -1.5)
    Vm = np.sqrt(X * X + Y1 * Y1 + Y2 * Y2)
    if spitzer:
        return nk * Ts * Ts * np.sqrt(Ts) * X / (1.0 + s * Ts * Vm)
    T15 = Ts * np.sqrt(Ts)
    return nk * T15 * X / (T15 + s * Vm)


def test_saturated_blend_with_the_face_temperature_cancelled():
    rng = np.random.default_rng(4)
    n = 100_000
    Ts = 10.0 ** rng.uniform(-2, 2, size=n)
    X, Y1, Y2 = (rng.normal(size=n) * 10.0 ** rng.uniform(-3, 3, size=n) for _ in range(3))
    for spitzer in (True, False):
        for nk, q0 in ((-0.25 * 0.01 * 2.0 ** -2.5, 1.5), (-0.25 * 0.02, 0.015), (-2.0, 3e-4)):
            d = _sat_direct(nk, q0, Ts, X, Y1, Y2, spitzer)
            c = _sat_cancelled(nk, q0, Ts, X, Y1, Y2, spitzer)
            assert np.allclose(c, d, rtol=1e-12, atol=0.0), (spitzer, nk, q0)
    # the two limits: q -> infinity leaves F, |F| >> q gives |F_sat| -> q
    for spitzer in (True, False):
        d = _sat_cancelled(-0.01, 1e30, Ts, X, Y1, Y2, spitzer)
        F = -0.01 * (Ts ** 2.5 if spitzer else 1.0) * X
        assert np.allclose(d, F, rtol=1e-12)
    Ts1 = np.array([2.0])
    big = np.array([1e12])
    sat = _sat_cancelled(-1.0, 0.7, Ts1, big, np.zeros(1), np.zeros(1), True)
    assert np.allclose(np.abs(sat), 0.7 * (Ts1 / 2.0) ** 1.5, rtol=1e-9)
