"""The learned surrogate's kernels against the FP64 oracle (oracle/surrogate.py):
forward increments, loss, every layer's weight and bias gradients, one
Adam step; exact conservation of the flux-form head; the accept and
fallback branches of the surrogate super-step.

Tolerances.  The network keeps its inputs, weights, hidden activations
and back-propagated gradients in BF16 (8 significant bits).  What that
storage costs on a given input is a property of the arithmetic, not of the
kernels: the oracle measures it by running in FP64 with every stored value
rounded to BF16 (``store=round_bf16``) and comparing with its plain FP64
run; call that gap g.  The GPU rounds at the same points, so it differs
from the BF16-storage oracle only where its FP32 accumulation moves a value
across a BF16 rounding boundary.  Tensor cores add the products of each
K = 16 step with truncated alignment, so one step can lose up to 2^-23 of
the magnitudes it adds, with a bias that makes the losses add up: a dot
product of n steps is off by at most n 2^-23 sum|w x| = n 2^-23 c |z|,
c the conditioning sum|w x| / |sum w x| of that layer's dot products, which
the oracle computes on the same input.  A stored value therefore crosses a
rounding boundary with probability P = n c 2^-23 / 2^-8 (its position
inside a BF16 unit is uniform) and then moves by one unit, against the
uniformly distributed rounding error (rms one unit / sqrt(12)) behind g:
the GPU's distance to the BF16-storage oracle is about sqrt(12 P) g, its
distance to the FP64 oracle about g (1 + sqrt(12 P)).  The tests allow
LAMBDA = 2 times the flip term (P from the worst-conditioned layer).  The
kernels' indexing is checked separately with zero tolerance on exactly
representable operands (test_gpu_surrogate_exact.py)."""
import numpy as np
import pytest

import workloads
from gpu_util import host, torch_dev
from oracle import surrogate as S

pytestmark = pytest.mark.gpu

REAL_IN = 6      # used input channels of layer 0
REAL_OUT = 3     # used output channels of layer 5

LAMBDA = 2.0


def _cond(a_abs, a):
    return float(np.linalg.norm(a_abs.ravel()) / max(np.linalg.norm(a.ravel()), 1e-300))


def _flip(params, x, hs, dx, target=None):
    """sqrt(12 P) for the worst-conditioned stored dot product of the BF16
    network's forward (and, with a target, backward-data) convolutions on
    this input: P = n c 2^-15, n the K = 16 steps of a dot product."""
    st = S.round_bf16
    h = st(x)
    pre, conds = [], []
    for li, (w, b) in enumerate(params):
        ws = st(w)
        z = S.conv3d(h, ws, b)
        conds.append((27 * h.shape[0] / 16, _cond(S.conv3d(np.abs(h), np.abs(ws), np.abs(b)), z)))
        pre.append(z)
        h = st(np.maximum(z, 0.0)) if li < len(params) - 1 else z
    if target is not None:
        r = S.flux_divergence(h, hs, dx) - target
        g = st(S.flux_divergence_adjoint(r / r.size, hs, dx))
        for li in range(len(params) - 1, 0, -1):
            ws = st(params[li][0])
            m = pre[li - 1] > 0.0
            gi = S.conv3d_grad_input(g, ws) * m
            conds.append((27 * g.shape[0] / 16, _cond(S.conv3d_grad_input(np.abs(g), np.abs(ws)) * m, gi)))
            g = st(gi)
    P = min(1.0, max(n * c for n, c in conds) * 2.0 ** -15)
    return float(np.sqrt(12.0 * P))


def _bounds(gap, flip):
    """(allowed distance to the BF16-storage oracle, to the FP64 oracle)."""
    return LAMBDA * flip * gap, gap * (1 + LAMBDA * flip)


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


def _init_params(rk, seed=0, real_in=REAL_IN):
    rng = np.random.default_rng(seed)
    params = []
    for l in range(6):
        co, ci = rk._lib.rkl_sur_layer_shape(l)
        rci = real_in if l == 0 else ci
        rco = REAL_OUT if l == 5 else co
        w = np.zeros((27, co, ci), dtype=np.float32)
        w[:, :rco, :rci] = rng.normal(scale=np.sqrt(2.0 / (27 * rci)), size=(27, rco, rci))
        b = np.zeros(co, dtype=np.float32)
        b[:rco] = rng.normal(scale=0.05, size=rco)
        params.append((w, b))
    return params


def _oracle_params(params, real_in=REAL_IN):
    out = []
    for l, (w, b) in enumerate(params):
        co, ci = w.shape[1], w.shape[2]
        wo = w.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
        rci = real_in if l == 0 else ci
        rco = REAL_OUT if l == 5 else co
        out.append((wo[:rco, :rci], b.astype(np.float64)[:rco]))
    return out


def _stats(a, ref):
    a, ref = a.ravel().astype(np.float64), ref.ravel().astype(np.float64)
    rl2 = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    cos = float(a @ ref / (np.linalg.norm(a) * np.linalg.norm(ref)))
    return rl2, cos


def _setup(rk, shape=(8, 16, 32), seed=3):
    import torch
    nz, ny, nx = shape
    T, b = workloads.tangled_box(nx, ny, nz, seed)
    T = T.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    dx = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    sur = rk._lib.rkl_sur_create(nz, ny, nx, dx, torch.cuda.current_stream().cuda_stream)
    params = _init_params(rk)
    for l, (w, bb) in enumerate(params):
        rk._lib.rkl_sur_set_params(sur, l, w, bb)
    Td, bd = torch_dev(T), torch_dev(b)
    return sur, params, T, b, Td, bd, dx


def test_forward_matches_oracle_and_conserves(rk):
    import torch
    sur, params, T, b, Td, bd, dx = _setup(rk)
    kappa0, ratio, hs = 0.01, 100.0, 2e-3
    rk._lib.rkl_sur_features(sur, Td, bd, kappa0, True, ratio)
    dT = torch.empty_like(Td)
    rk._lib.rkl_sur_forward(sur, hs, dT)
    torch.cuda.synchronize()
    x = S.features(T, b, kappa0, True, ratio)
    ref, _ = S.forward(_oracle_params(params), x, hs, dx)
    ref16, _ = S.forward(_oracle_params(params), x, hs, dx, store=S.round_bf16)
    got = host(dT)
    gap = _stats(ref16, ref)[0]
    flip = _flip(_oracle_params(params), x, hs, dx)
    to16, to64 = _bounds(gap, flip)
    rl2_16, _ = _stats(got, ref16)
    rl2, cos = _stats(got, ref)
    print(f"surrogate forward: BF16 storage gap {gap:.3e}, flip factor {flip:.3f}; "
          f"GPU vs BF16-storage oracle {rl2_16:.3e} "
          f"(bound {to16:.3e}), vs FP64 oracle {rl2:.3e} (bound {to64:.3e}), cosine {cos:.6f}")
    assert rl2_16 < to16 and rl2 < to64
    # flux form: the increment sums to zero
    assert abs(got.sum()) <= 1e-5 * np.abs(got).sum()
    rk._lib.rkl_sur_destroy(sur)


def test_forward_with_flux_features_matches_oracle(rk, orc):
    """Channels 6-8 carry the scaled face fluxes of T as the plan evaluates
    them (Eqs. Fclass, qN, qT); the forward pass on these nine features
    against the oracle's forward on its own FP64 fluxes."""
    import torch
    from oracle import Problem
    sur, params, T, b, Td, bd, dx = _setup(rk)
    params = _init_params(rk, seed=4, real_in=9)
    for l, (w, bb) in enumerate(params):
        rk._lib.rkl_sur_set_params(sur, l, w, bb)
    shape = T.shape
    prm = dict(dx=dx, kappa_model="spitzer", kappa_par0=0.01, kappa_perp_ratio=1e-4)
    plan = rk.Plan(shape, "f32", params=prm)
    ratio, hs, fscale = 100.0, 2e-3, 300.0      # flux channels of rms about 1
    rk._lib.rkl_sur_features_flux(sur, plan.handle, Td, bd, ratio, fscale)
    dT = torch.empty_like(Td)
    rk._lib.rkl_sur_forward(sur, hs, dT)
    torch.cuda.synchronize()
    F = [fscale * f for f in orc.flux(Problem(shape, **prm), T, b)]
    x = S.features(T, b, 0.01, True, ratio, flux=F)
    op = _oracle_params(params, 9)
    ref, _ = S.forward(op, x, hs, dx)
    ref16, _ = S.forward(op, x, hs, dx, store=S.round_bf16)
    gap = _stats(ref16, ref)[0]
    to16, to64 = _bounds(gap, _flip(op, x, hs, dx))
    got = host(dT)
    rl2_16, rl2 = _stats(got, ref16)[0], _stats(got, ref)[0]
    print(f"flux features: BF16 gap {gap:.3e}; GPU vs BF16-storage oracle {rl2_16:.3e} (bound {to16:.3e}), "
          f"vs FP64 {rl2:.3e} (bound {to64:.3e})")
    assert rl2_16 < to16 and rl2 < to64
    # without the flux channels the same network sees zeros there: a different output
    rk._lib.rkl_sur_features(sur, Td, bd, 0.01, True, ratio)
    dT0 = torch.empty_like(Td)
    rk._lib.rkl_sur_forward(sur, hs, dT0)
    assert _stats(host(dT0), got)[0] > 10 * to16
    plan.close()
    rk._lib.rkl_sur_destroy(sur)


def test_gradients_match_oracle(rk):
    import torch
    sur, params, T, b, Td, bd, dx = _setup(rk)
    kappa0, ratio, hs = 0.02, 60.0, 2e-3
    rng = np.random.default_rng(5)
    target = rng.normal(scale=1e-3, size=T.shape)
    target -= target.mean()
    rk._lib.rkl_sur_features(sur, Td, bd, kappa0, True, ratio)
    rk._lib.rkl_sur_forward(sur, hs)
    loss = rk._lib.rkl_sur_backward(sur, torch_dev(target))
    x = S.features(T, b, kappa0, True, ratio)
    tgt = target.astype(np.float32).astype(np.float64)
    loss_ref, grads, _ = S.loss_and_grad(_oracle_params(params), x, tgt, hs, dx)
    loss16, grads16, _ = S.loss_and_grad(_oracle_params(params), x, tgt, hs, dx, store=S.round_bf16)
    flip = _flip(_oracle_params(params), x, hs, dx, tgt)
    # the loss 0.5 mean(r^2) moves by at most |r - r16| (|r| + |r16|) / (2 n)
    # when dT does, and dT's distance to the BF16-storage oracle is bounded
    # as in the forward test
    dT16, _ = S.forward(_oracle_params(params), x, hs, dx, store=S.round_bf16)
    dT64, _ = S.forward(_oracle_params(params), x, hs, dx)
    to16, _ = _bounds(_stats(dT16, dT64)[0], flip)
    r16 = dT16 - tgt
    dr = to16 * np.linalg.norm(dT16)
    lbound = dr * (2 * np.linalg.norm(r16) + dr) / (2 * r16.size)
    print(f"surrogate loss {loss:.6e} oracle {loss_ref:.6e} BF16-storage oracle {loss16:.6e} "
          f"(bound on the distance {lbound:.3e}); flip factor {flip:.3f}")
    assert abs(loss - loss16) <= lbound + 1e-7 * loss16
    for l in range(6):
        gw, gb = rk._lib.rkl_sur_get_grads(sur, l)
        co, ci = gw.shape[1], gw.shape[2]
        gw_or = gw.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
        rci = REAL_IN if l == 0 else ci
        rco = REAL_OUT if l == 5 else co
        gap = _stats(grads16[l][0], grads[l][0])[0]
        to16, to64 = _bounds(gap, flip)
        rl2_16 = _stats(gw_or[:rco, :rci], grads16[l][0])[0]
        rl2, cos = _stats(gw_or[:rco, :rci], grads[l][0])
        print(f"layer {l}: dW BF16 gap {gap:.3e}; GPU vs BF16-storage oracle {rl2_16:.3e} (bound {to16:.3e}), "
              f"vs FP64 {rl2:.3e} (bound {to64:.3e}) cos {cos:.6f}")
        assert rl2_16 < to16 and rl2 < to64, l
        if l < 5:
            gapb = _stats(grads16[l][1], grads[l][1])[0]
            b16, b64 = _bounds(gapb, flip)
            rlb16 = _stats(gb[:rco], grads16[l][1])[0]
            rlb = _stats(gb[:rco], grads[l][1])[0]
            print(f"layer {l}: db BF16 gap {gapb:.3e}; vs BF16-storage {rlb16:.3e}, vs FP64 {rlb:.3e}")
            assert rlb16 < b16 and rlb < b64, l
        else:
            # a constant face flux has no divergence: the head's bias gradient
            # is exactly zero (the adjoint telescopes); only rounding remains
            assert np.max(np.abs(grads[l][1])) <= 1e-9 * np.max(np.abs(grads[l][0]))
            assert np.max(np.abs(gb[:rco])) <= 1e-2 * np.max(np.abs(gw))
        # padded channels stay exactly zero
        assert np.all(gw[:, rco:, :] == 0) and np.all(gw[:, :, rci:] == 0)
    rk._lib.rkl_sur_destroy(sur)


def test_adam_first_step_and_training_reduces_loss(rk):
    import torch
    sur, params, T, b, Td, bd, dx = _setup(rk)
    kappa0, ratio, hs, lr = 0.01, 100.0, 2e-3, 1e-3
    rng = np.random.default_rng(6)
    target = rng.normal(scale=1e-3, size=T.shape)
    target -= target.mean()
    tgt = torch_dev(target)
    rk._lib.rkl_sur_features(sur, Td, bd, kappa0, True, ratio)
    rk._lib.rkl_sur_forward(sur, hs)
    rk._lib.rkl_sur_backward(sur, tgt)
    g = [rk._lib.rkl_sur_get_grads(sur, l) for l in range(6)]
    rk._lib.rkl_sur_adam(sur, lr)
    # first bias-corrected Adam step: p1 = p0 - lr g / (|g| + eps)
    for l in range(6):
        w1, b1 = rk._lib.rkl_sur_get_params(sur, l)
        want = params[l][0] - lr * g[l][0] / (np.abs(g[l][0]) + 1e-8)
        assert np.allclose(w1, want, rtol=0, atol=2e-6), l
    losses = []
    for _ in range(30):
        losses.append(rk._lib.rkl_sur_train_step(sur, hs, tgt, 3e-3))
    print("training losses:", losses[0], losses[-1])
    assert losses[-1] < 0.7 * losses[0]
    rk._lib.rkl_sur_destroy(sur)


def test_surrogate_super_step_accept_and_fallback(rk):
    import torch
    shape = (16, 16, 32)
    sur, params, T, b, Td, bd, dx = _setup(rk, shape=shape)
    prm = dict(dx=(1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0]), kappa_model="spitzer", kappa_par0=0.01,
               kappa_perp_ratio=1e-4)
    plan = rk.Plan(shape, "f32", params=prm)
    dt = 50 * plan.dt_expl(Td)
    hs = 2e-3
    # threshold 0: always the fallback, identical to the plain super-step
    T1 = Td.clone()
    acc, rho, s = rk._lib.rkl_sur_super_step(sur, plan.handle, dt, T1, bd, hs, 0.0)
    T2 = Td.clone()
    s2 = plan.super_step(dt, T2, bd)
    torch.cuda.synchronize()
    assert not acc and s == s2 and rho > 0
    assert torch.equal(T1, T2)
    # threshold infinity: accepted, T + predicted increment
    T3 = Td.clone()
    acc, rho, s = rk._lib.rkl_sur_super_step(sur, plan.handle, dt, T3, bd, hs, float("inf"))
    ratio = dt / plan.dt_expl(Td)
    rk._lib.rkl_sur_features(sur, Td, bd, 0.01, True, ratio)
    dT = torch.empty_like(Td)
    rk._lib.rkl_sur_forward(sur, hs, dT)
    torch.cuda.synchronize()
    assert acc and s == 0
    assert torch.allclose(T3, Td + dT, rtol=0, atol=1e-6)
    rk._lib.rkl_sur_destroy(sur)


def test_residual_check_with_flux_features_evaluates_m_once(rk):
    """With flux features the residual check takes M(Y0) as the divergence
    of the face fluxes the features already hold, and evaluates M only at
    Y0 + dT: the residual it reports equals the trapezoidal residual built
    from two full M evaluations (plan.apply_M) up to FP32 rounding."""
    import torch
    shape = (16, 16, 32)
    sur, params, T, b, Td, bd, dx = _setup(rk, shape=shape)
    prm = dict(dx=(1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0]), kappa_model="spitzer", kappa_par0=0.01,
               kappa_perp_ratio=1e-4)
    plan = rk.Plan(shape, "f32", params=prm)
    dt = 50 * plan.dt_expl(Td)
    hs, c = 2e-3, 1.0 / 16
    rk._lib.rkl_sur_set_flux_features(sur, c)
    T1 = Td.clone()
    acc, rho, _ = rk._lib.rkl_sur_super_step(sur, plan.handle, dt, T1, bd, hs, 0.0)
    assert not acc
    ratio = dt / plan.dt_expl(Td)
    rk._lib.rkl_sur_features_flux(sur, plan.handle, Td, bd, ratio, c * dt / hs)
    dT = torch.empty_like(Td)
    rk._lib.rkl_sur_forward(sur, hs, dT)
    M0, Mp = torch.empty_like(Td), torch.empty_like(Td)
    plan.apply_M(Td, bd, M0)
    plan.apply_M(Td + dT, bd, Mp)
    torch.cuda.synchronize()
    d = dT.double()
    r = d - 0.5 * dt * (M0.double() + Mp.double())
    ref = float(r.norm() / d.norm())
    assert abs(rho - ref) <= 1e-3 * ref, (rho, ref)
    rk._lib.rkl_sur_destroy(sur)


def test_tcgen05_backend_matches_warp_mma_and_oracle(rk):
    """The tcgen05 convolutions (TMEM accumulators) against the warp-level
    mma.sync ones on the same BF16 inputs -- they differ only in the order
    of the FP32 accumulation and in the BF16 rounding it can flip -- and
    against the FP64 oracle with the same bounds as the forward test;
    then the weight gradients of a backward pass whose backward-data
    convolutions run on tcgen05."""
    import torch
    sur, params, T, b, Td, bd, dx = _setup(rk, shape=(8, 32, 16))
    kappa0, ratio, hs = 0.01, 100.0, 2e-3
    rk._lib.rkl_sur_features(sur, Td, bd, kappa0, True, ratio)
    out = {}
    for backend in (0, 1):
        rk._lib.rkl_sur_set_backend(sur, backend)
        dT = torch.empty_like(Td)
        rk._lib.rkl_sur_forward(sur, hs, dT)
        rk._lib.rkl_sur_check(sur)
        out[backend] = host(dT)
    rl2, cos = _stats(out[1], out[0])
    print(f"tcgen05 vs mma.sync forward: rel-L2 {rl2:.3e}, cosine {cos:.6f}")
    assert rl2 < 1e-2 and cos > 0.9999
    x = S.features(T, b, kappa0, True, ratio)
    ref, _ = S.forward(_oracle_params(params), x, hs, dx)
    ref16, _ = S.forward(_oracle_params(params), x, hs, dx, store=S.round_bf16)
    to16, to64 = _bounds(_stats(ref16, ref)[0], _flip(_oracle_params(params), x, hs, dx))
    for backend in (0, 1):
        assert _stats(out[backend], ref16)[0] < to16 and _stats(out[backend], ref)[0] < to64, backend
    assert abs(out[1].sum()) <= 1e-5 * np.abs(out[1]).sum()
    # backward with tcgen05 backward-data against the oracle's gradients
    rng = np.random.default_rng(5)
    target = rng.normal(scale=1e-3, size=T.shape)
    target -= target.mean()
    rk._lib.rkl_sur_set_backend(sur, 1)
    rk._lib.rkl_sur_forward(sur, hs)
    rk._lib.rkl_sur_backward(sur, torch_dev(target))
    rk._lib.rkl_sur_check(sur)
    tgt = target.astype(np.float32).astype(np.float64)
    _, grads, _ = S.loss_and_grad(_oracle_params(params), x, tgt, hs, dx)
    _, grads16, _ = S.loss_and_grad(_oracle_params(params), x, tgt, hs, dx, store=S.round_bf16)
    flip = _flip(_oracle_params(params), x, hs, dx, tgt)
    for l in range(5):
        gw, gb = rk._lib.rkl_sur_get_grads(sur, l)
        co, ci = gw.shape[1], gw.shape[2]
        gw_or = gw.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
        rci = REAL_IN if l == 0 else ci
        to16, to64 = _bounds(_stats(grads16[l][0], grads[l][0])[0], flip)
        rl2_16 = _stats(gw_or[:, :rci], grads16[l][0])[0]
        rl2, cos = _stats(gw_or[:, :rci], grads[l][0])
        print(f"tcgen05 backward layer {l}: dW vs BF16-storage {rl2_16:.3e} (bound {to16:.3e}), "
              f"vs FP64 {rl2:.3e} (bound {to64:.3e}) cos {cos:.6f}")
        assert rl2_16 < to16 and rl2 < to64, l
    rk._lib.rkl_sur_destroy(sur)


def test_trained_surrogate_gains_over_no_network(rk):
    """What training buys, on held-out RKL2 pairs of 32^3 patches (tangled
    fields of seeds the training pool does not contain, dt / dt_expl in
    [50, 150]): the relative L2 error of the
    predicted end-of-super-step state against the plain RKL2 super-step,
    for the trained network, the same network before training, and no
    network at all (T unchanged).  Also times one forward pass against one
    RKL2 super-step on the same patch; the figures are printed."""
    import torch
    from paper_1702_05487_gb300.surrogate import Surrogate, SurrogateConfig
    sur = Surrogate(SurrogateConfig(n=32, pool=6, seed0=700))

    # held-out fields: seeds the training pool does not use
    test_pool = []
    for k in range(3):
        T, bb = workloads.tangled_box(32, 32, 32, 900 + k)
        test_pool.append((torch.from_numpy(T.astype(np.float32)).cuda(),
                          torch.from_numpy(bb.astype(np.float32)).cuda()))

    def heldout(n, seed):
        rng_state, pool = sur.rng, sur.pool
        sur.rng, sur.pool = np.random.default_rng(seed), test_pool
        rows = []
        for _ in range(n):
            T0, b, kappa0, ratio, dt, target = sur.draw()
            if sur.cfg.head_scale <= 0.0:
                sur.cfg.head_scale = float(target.double().pow(2).mean().sqrt()) * sur.dx[0]
            dT = sur.predict(T0, b, kappa0, ratio)
            Tt = (T0 + target).double()
            nrm = float(Tt.norm())
            rows.append((float((dT - target).double().norm()) / nrm, float(target.double().norm()) / nrm))
        sur.rng, sur.pool = rng_state, pool
        return np.array(rows)

    before = heldout(12, 99)
    sur.train(600)
    after = heldout(12, 99)
    e_net, e_none, e_untrained = np.median(after[:, 0]), np.median(after[:, 1]), np.median(before[:, 0])
    # time of one forward pass and one super-step at dt = 100 dt_expl
    T0, b = sur.pool[0]
    plan = sur.plan(0.01)
    dt = 100.0 * plan.dt_expl(T0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    T1 = T0.clone()
    plan.super_step(dt, T1, b)
    sur.predict(T0, b, 0.01, 100.0)
    torch.cuda.synchronize()
    ev[0].record(sur.stream)
    for _ in range(5):
        plan.super_step(dt, T1, b)
    ev[1].record(sur.stream)
    for _ in range(5):
        rk._lib.rkl_sur_forward(sur.handle, sur.cfg.head_scale)
    ev[2].record(sur.stream)
    torch.cuda.synchronize()
    print(f"held-out state error (median): trained {e_net:.2e}, untrained {e_untrained:.2e}, "
          f"no network {e_none:.2e}; 32^3 RKL2 super-step {ev[0].elapsed_time(ev[1]) / 5:.3f} ms, "
          f"forward {ev[1].elapsed_time(ev[2]) / 5:.3f} ms")
    assert e_net < 0.5 * e_none
    assert e_net < 0.5 * e_untrained
    sur.close()


@pytest.mark.parametrize("shape", [(64, 64, 64), (100, 64, 96)])
def test_tcgen05_persistent_ctas_with_several_items(rk, shape):
    """Grids with more work items (8 x 16 column blocks x 6-plane chunks)
    than resident CTAs, so that CTAs run several items in a row (ending with
    a short last chunk) and the pipeline's barriers go through many phases:
    the tcgen05 forward and backward-data passes against the warp-level
    mma.sync ones, layer by layer through the whole network, and the
    increment's exact conservation."""
    import torch
    sur, params, T, b, Td, bd, dx = _setup(rk, shape=shape)
    kappa0, ratio, hs = 0.01, 100.0, 2e-3
    rk._lib.rkl_sur_features(sur, Td, bd, kappa0, True, ratio)
    rng = np.random.default_rng(9)
    target = torch_dev(rng.normal(scale=1e-3, size=shape))
    out, grads = {}, {}
    for backend in (0, 1):
        rk._lib.rkl_sur_set_backend(sur, backend)
        dT = torch.empty_like(Td)
        rk._lib.rkl_sur_forward(sur, hs, dT)
        rk._lib.rkl_sur_backward(sur, target)
        rk._lib.rkl_sur_check(sur)
        out[backend] = host(dT)
        grads[backend] = [rk._lib.rkl_sur_get_grads(sur, l)[0] for l in range(6)]
    rl2, cos = _stats(out[1], out[0])
    print(f"{shape}: tcgen05 vs mma.sync forward rel-L2 {rl2:.3e}, cosine {cos:.6f}")
    assert rl2 < 1e-2 and cos > 0.9999
    assert abs(out[1].sum()) <= 1e-5 * np.abs(out[1]).sum()
    for l in range(6):
        rl2, cos = _stats(grads[1][l], grads[0][l])
        assert rl2 < 2e-2 and cos > 0.9998, (l, rl2, cos)
    rk._lib.rkl_sur_destroy(sur)
