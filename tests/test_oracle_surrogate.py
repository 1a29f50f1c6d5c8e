"""Pins for the surrogate oracle (oracle/surrogate.py).  No GPU.

The periodic 3x3x3 convolution and its two adjoints are checked against
torch's conv3d with circular padding and its autograd (library special
cases, FP64 on CPU); the whole network's loss gradient against central
finite differences; the flux-form head against exact conservation and its
adjoint identity; Adam against its closed-form first step."""
import numpy as np
import pytest

from oracle import surrogate as S


def _torch():
    return pytest.importorskip("torch")


def _rand(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


def test_conv3d_matches_torch_circular():
    torch = _torch()
    F = torch.nn.functional
    x = _rand((5, 6, 7, 8), 1)
    w = _rand((4, 5, 3, 3, 3), 2)
    b = _rand((4,), 3)
    got = S.conv3d(x, w, b)
    xt = F.pad(torch.from_numpy(x)[None], (1, 1, 1, 1, 1, 1), mode="circular")
    want = F.conv3d(xt, torch.from_numpy(w), torch.from_numpy(b))[0].numpy()
    assert np.max(np.abs(got - want)) < 1e-12


def test_conv3d_adjoints_match_autograd():
    torch = _torch()
    F = torch.nn.functional
    x = _rand((3, 5, 6, 4), 4)
    w = _rand((6, 3, 3, 3, 3), 5)
    b = _rand((6,), 6)
    gy = _rand((6, 5, 6, 4), 7)
    xt = torch.tensor(x, requires_grad=True)
    wt = torch.tensor(w, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    y = F.conv3d(F.pad(xt[None], (1, 1, 1, 1, 1, 1), mode="circular"), wt, bt)[0]
    y.backward(torch.from_numpy(gy))
    assert np.max(np.abs(S.conv3d_grad_input(gy, w) - xt.grad.numpy())) < 1e-11
    gw, gb = S.conv3d_grad_weight(gy, x)
    assert np.max(np.abs(gw - wt.grad.numpy())) < 1e-10
    assert np.max(np.abs(gb - bt.grad.numpy())) < 1e-11


def test_flux_head_conserves_and_adjoint_identity():
    G = _rand((3, 5, 6, 7), 8)
    dx = (0.1, 0.2, 0.3)
    dT = S.flux_divergence(G, 0.7, dx)
    assert abs(dT.sum()) < 1e-12 * np.abs(dT).sum()
    y = _rand((5, 6, 7), 9)
    lhs = float(np.sum(dT * y))
    rhs = float(np.sum(G * S.flux_divergence_adjoint(y, 0.7, dx)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _tiny_net(seed=10, chans=(6, 4, 4, 3)):
    rng = np.random.default_rng(seed)
    return [(rng.normal(scale=0.3, size=(co, ci, 3, 3, 3)), rng.normal(scale=0.1, size=(co,)))
            for ci, co in zip(chans[:-1], chans[1:])]


def test_network_gradient_against_finite_differences():
    params = _tiny_net()
    x = _rand((6, 4, 5, 6), 11)
    target = _rand((4, 5, 6), 12) * 0.1
    tau, dx = 0.05, (0.25, 0.2, 1.0 / 6)
    loss, grads, _ = S.loss_and_grad(params, x, target, tau, dx)
    rng = np.random.default_rng(13)
    h = 1e-6
    for li in range(len(params)):
        w, b = params[li]
        for _ in range(4):
            idx = tuple(int(rng.integers(0, n)) for n in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = list(params); pp[li] = (wp, b)
            pm = list(params); pm[li] = (wm, b)
            fd = (S.loss_and_grad(pp, x, target, tau, dx)[0] - S.loss_and_grad(pm, x, target, tau, dx)[0]) / (2 * h)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        k = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        pp = list(params); pp[li] = (w, bp)
        pm = list(params); pm[li] = (w, bm)
        fd = (S.loss_and_grad(pp, x, target, tau, dx)[0] - S.loss_and_grad(pm, x, target, tau, dx)[0]) / (2 * h)
        assert grads[li][1][k] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_step_closed_form():
    p = _rand((7,), 14)
    g = _rand((7,), 15)
    p1, m, v = S.adam(p, g, np.zeros(7), np.zeros(7), 1, lr=0.01)
    # bias-corrected m/sqrt(v) = g/|g| on the first step
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_round_bf16_against_torch_and_ties():
    """round_bf16 against torch's FP32 -> BF16 conversion (round to nearest
    even) on FP32 values, where one rounding from FP64 and torch's agree,
    and on hand-made ties."""
    import torch
    from oracle.surrogate import round_bf16
    rng = np.random.default_rng(0)
    x32 = np.concatenate([rng.normal(size=20000), rng.normal(size=2000) * 1e-30, rng.normal(size=2000) * 1e30,
                          [0.0, -0.0, 1.0, -2.5]]).astype(np.float32)
    want = torch.from_numpy(x32).to(torch.bfloat16).float().numpy().astype(np.float64)
    assert np.array_equal(round_bf16(x32.astype(np.float64)), want)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (even: 1);
    # 1 + 3 2^-8 halfway between 1 + 2^-7 and 1 + 2^-6 (even: 1 + 2^-6)
    t = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 1 + 2.0 ** -8 + 2.0 ** -40])
    assert list(round_bf16(t)) == [1.0, 1 + 2.0 ** -6, -1.0, 1 + 2.0 ** -7]
    y = round_bf16(rng.normal(size=1000))
    assert np.array_equal(round_bf16(y), y)


def test_bf16_storage_emulation_reduces_to_rounded_operands():
    """One linear layer: storing in BF16 is the FP64 convolution of the
    rounded input and weights (the store points are exactly those)."""
    from oracle.surrogate import round_bf16
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 4, 4, 8))
    w = rng.normal(size=(3, 3, 3, 3, 3)) * 0.2
    b = rng.normal(size=3)
    got, _ = S.forward([(w, b)], x, 1.0, (1.0, 1.0, 1.0), store=round_bf16)
    want, _ = S.forward([(round_bf16(w), b)], round_bf16(x), 1.0, (1.0, 1.0, 1.0))
    assert np.array_equal(got, want)
    plain, _ = S.forward([(w, b)], x, 1.0, (1.0, 1.0, 1.0))
    assert 0 < np.abs(got - plain).max() < 1e-2 * np.abs(plain).max()
