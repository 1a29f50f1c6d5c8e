"""The learned surrogate's kernels against the FP64 oracle (oracle/surrogate.py):
forward increments, loss, every layer's weight and bias gradients, one
Adam step; exact conservation of the flux-form head; the accept and
fallback branches of the surrogate super-step.

BF16 weights and activations (8-bit mantissa, relative rounding 2^-9 per
stored value, accumulated over six layers forward and five BF16 gradient
layers backward, then differenced by the flux-form divergence) bound the
agreement with FP64: the increment within 5e-2 relative L2 and cosine
0.998 (measured 1.8e-2, 0.99985), weight and bias gradients within 1e-1
relative L2 and cosine 0.995 (measured 3e-2 to 6e-2, cosine >= 0.998 on
the deepest layer); the errors are printed."""
import numpy as np
import pytest

import workloads
from gpu_util import host, torch_dev
from oracle import surrogate as S

pytestmark = pytest.mark.gpu

REAL_IN = 6      # used input channels of layer 0
REAL_OUT = 3     # used output channels of layer 5


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


def _init_params(rk, seed=0):
    rng = np.random.default_rng(seed)
    params = []
    for l in range(6):
        co, ci = rk._lib.rkl_sur_layer_shape(l)
        rci = REAL_IN if l == 0 else ci
        rco = REAL_OUT if l == 5 else co
        w = np.zeros((27, co, ci), dtype=np.float32)
        w[:, :rco, :rci] = rng.normal(scale=np.sqrt(2.0 / (27 * rci)), size=(27, rco, rci))
        b = np.zeros(co, dtype=np.float32)
        b[:rco] = rng.normal(scale=0.05, size=rco)
        params.append((w, b))
    return params


def _oracle_params(params):
    out = []
    for l, (w, b) in enumerate(params):
        co, ci = w.shape[1], w.shape[2]
        wo = w.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
        rci = REAL_IN if l == 0 else ci
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
    got = host(dT)
    rl2, cos = _stats(got, ref)
    print(f"surrogate forward: rel-L2 {rl2:.3e}, cosine {cos:.6f}")
    assert rl2 < 5e-2 and cos > 0.998
    # flux form: the increment sums to zero
    assert abs(got.sum()) <= 1e-5 * np.abs(got).sum()
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
    loss_ref, grads, _ = S.loss_and_grad(_oracle_params(params), x, target.astype(np.float32).astype(np.float64),
                                         hs, dx)
    print(f"surrogate loss {loss:.6e} oracle {loss_ref:.6e}")
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    for l in range(6):
        gw, gb = rk._lib.rkl_sur_get_grads(sur, l)
        co, ci = gw.shape[1], gw.shape[2]
        gw_or = gw.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
        rci = REAL_IN if l == 0 else ci
        rco = REAL_OUT if l == 5 else co
        rl2, cos = _stats(gw_or[:rco, :rci], grads[l][0])
        rlb, cosb = _stats(gb[:rco], grads[l][1])
        print(f"layer {l}: dW rel-L2 {rl2:.3e} cos {cos:.6f}; db rel-L2 {rlb:.3e} cos {cosb:.6f}")
        assert rl2 < 1e-1 and cos > 0.995, l
        if l < 5:
            assert rlb < 1e-1 and cosb > 0.995, l
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
    rl2, cos = _stats(out[1], ref)
    assert rl2 < 5e-2 and cos > 0.998
    assert abs(out[1].sum()) <= 1e-5 * np.abs(out[1]).sum()
    # backward with tcgen05 backward-data against the oracle's gradients
    rng = np.random.default_rng(5)
    target = rng.normal(scale=1e-3, size=T.shape)
    target -= target.mean()
    rk._lib.rkl_sur_set_backend(sur, 1)
    rk._lib.rkl_sur_forward(sur, hs)
    rk._lib.rkl_sur_backward(sur, torch_dev(target))
    rk._lib.rkl_sur_check(sur)
    _, grads, _ = S.loss_and_grad(_oracle_params(params), x, target.astype(np.float32).astype(np.float64), hs, dx)
    for l in range(5):
        gw, gb = rk._lib.rkl_sur_get_grads(sur, l)
        co, ci = gw.shape[1], gw.shape[2]
        gw_or = gw.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
        rci = REAL_IN if l == 0 else ci
        rl2, cos = _stats(gw_or[:, :rci], grads[l][0])
        print(f"tcgen05 backward layer {l}: dW rel-L2 {rl2:.3e} cos {cos:.6f}")
        assert rl2 < 1e-1 and cos > 0.995, l
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
