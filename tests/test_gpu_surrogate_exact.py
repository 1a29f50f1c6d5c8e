"""The surrogate's convolution kernels, one layer at a time, against the FP64
oracle (oracle/surrogate.py) with zero tolerance.

Operands are small integers (activations and gradients in [-2, 2], weights
in {-1, 0, 1} with few nonzeros, biases in [-4, 4]): every one is exact in
BF16, every product and every partial sum is an integer far below 2^24, so
the FP32 accumulation of the tensor cores is exact in any order and every
stored BF16 result (|value| <= 256) is exact too.  The kernels' output must
then equal the oracle's element for element.  A wrong halo plane, a
misplaced edge voxel, a transposed weight block or a dropped channel
changes some integer and fails the comparison; no rounding can hide it.

Checked for both backends of the forward and backward-data convolutions
(tcgen05 with TMEM accumulators, and the warp-level mma.sync kernels) and
for the weight and bias gradients, on a small patch and on one whose
tcgen05 grid runs several work items per CTA with a short last chunk."""
import numpy as np
import pytest

from oracle import surrogate as S

pytestmark = pytest.mark.gpu

SHAPES = [(8, 16, 32), (36, 48, 48)]


@pytest.fixture(scope="module")
def rk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1702_05487_gb300 as rk
    rk.load()
    return rk


def _bf16(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    assert np.array_equal(t.float().numpy(), a), "operand not exact in BF16"
    return t.cuda()


def _ints(rng, shape, lo, hi):
    return rng.integers(lo, hi + 1, size=shape).astype(np.float32)


def _sparse_weights(rng, co, ci, nnz_per_row=12):
    """[27][co][ci] with about nnz_per_row nonzeros (+-1) per output channel."""
    w = np.zeros((27, co, ci), dtype=np.float32)
    for o in range(co):
        idx = rng.choice(27 * ci, size=nnz_per_row, replace=False)
        w.reshape(27, co, ci)[idx // ci, o, idx % ci] = rng.choice([-1.0, 1.0], size=nnz_per_row)
    return w


def _to_oracle_w(w):
    """[27][co][ci] -> [co][ci][3][3][3] indexed [dz+1][dy+1][dx+1]."""
    co, ci = w.shape[1], w.shape[2]
    return w.astype(np.float64).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)


def _chfirst(a, shape):
    """[V][C] channels last -> [C][D][H][W]."""
    return a.reshape(shape + (a.shape[-1],)).transpose(3, 0, 1, 2).astype(np.float64)


def _chlast(a):
    return a.transpose(1, 2, 3, 0).reshape(-1, a.shape[0])


def _make(rk, shape, backend, seed):
    import torch
    nz, ny, nx = shape
    sur = rk._lib.rkl_sur_create(nz, ny, nx, (1.0 / nx, 1.0 / ny, 1.0 / nz), torch.cuda.current_stream().cuda_stream)
    rk._lib.rkl_sur_set_backend(sur, backend)
    rng = np.random.default_rng(seed)
    params = []
    for l in range(6):
        co, ci = rk._lib.rkl_sur_layer_shape(l)
        w = _sparse_weights(rng, co, ci)
        b = _ints(rng, (co,), -4, 4)
        rk._lib.rkl_sur_set_params(sur, l, w, b)
        params.append((w, b))
    return sur, params, rng


@pytest.mark.parametrize("backend", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_layer_forward_exact(rk, shape, backend):
    import torch
    sur, params, rng = _make(rk, shape, backend, seed=11 + backend)
    V = int(np.prod(shape))
    for l in range(6):
        co, ci = rk._lib.rkl_sur_layer_shape(l)
        x = _ints(rng, (V, ci), -2, 2)
        w, b = params[l]
        last = l == 5
        out = torch.empty((V, co), device="cuda", dtype=torch.float32 if last else torch.bfloat16)
        rk._lib.rkl_sur_layer_forward(sur, l, _bf16(x), out)
        rk._lib.rkl_sur_check(sur)
        ref = S.conv3d(_chfirst(x, shape), _to_oracle_w(w), b.astype(np.float64))
        if not last:
            ref = np.maximum(ref, 0.0)
        assert np.abs(ref).max() <= 256                 # exact in BF16 as stored
        got = out.float().cpu().numpy().astype(np.float64)
        bad = np.argwhere(got != _chlast(ref))
        assert bad.size == 0, (l, bad[:5], got[tuple(bad[0])], _chlast(ref)[tuple(bad[0])])
    rk._lib.rkl_sur_destroy(sur)


@pytest.mark.parametrize("backend", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_layer_backward_data_exact(rk, shape, backend):
    import torch
    sur, params, rng = _make(rk, shape, backend, seed=21 + backend)
    V = int(np.prod(shape))
    for l in range(1, 6):
        co, ci = rk._lib.rkl_sur_layer_shape(l)
        dz = _ints(rng, (V, co), -2, 2)
        mask = _ints(rng, (V, ci), -1, 1)
        out = torch.empty((V, ci), device="cuda", dtype=torch.bfloat16)
        rk._lib.rkl_sur_layer_backward_data(sur, l, _bf16(dz), _bf16(mask), out)
        rk._lib.rkl_sur_check(sur)
        ref = S.conv3d_grad_input(_chfirst(dz, shape), _to_oracle_w(params[l][0]))
        ref = _chlast(ref) * (mask > 0)
        assert np.abs(ref).max() <= 256
        got = out.float().cpu().numpy().astype(np.float64)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, (l, bad[:5])
    rk._lib.rkl_sur_destroy(sur)


@pytest.mark.parametrize("shape", SHAPES)
def test_layer_weight_grad_exact_and_repeatable(rk, shape):
    sur, params, rng = _make(rk, shape, 0, seed=31)
    V = int(np.prod(shape))
    for l in range(6):
        co, ci = rk._lib.rkl_sur_layer_shape(l)
        dz = _ints(rng, (V, co), -2, 2)
        x = _ints(rng, (V, ci), -2, 2)
        dzd, xd = _bf16(dz), _bf16(x)
        rk._lib.rkl_sur_layer_weight_grad(sur, l, dzd, xd)
        gw, gb = rk._lib.rkl_sur_get_grads(sur, l)
        gw_ref, gb_ref = S.conv3d_grad_weight(_chfirst(dz, shape), _chfirst(x, shape))
        gw_ref = gw_ref.reshape(co, ci, 27).transpose(2, 0, 1)
        assert np.array_equal(gw.astype(np.float64), gw_ref), l
        assert np.array_equal(gb.astype(np.float64), gb_ref), l
        # a second call gives the same bits (fixed-order sums, no atomics)
        rk._lib.rkl_sur_layer_weight_grad(sur, l, dzd, xd)
        gw2, gb2 = rk._lib.rkl_sur_get_grads(sur, l)
        assert np.array_equal(gw, gw2) and np.array_equal(gb, gb2), l
    rk._lib.rkl_sur_destroy(sur)


def test_training_steps_repeat_bit_for_bit(rk):
    """Real-valued data: two surrogates with the same parameters and the same
    targets take three training steps each; every weight must agree bit for
    bit (no order-dependent reduction anywhere in forward, backward or
    Adam)."""
    import torch
    import workloads
    shape = (8, 32, 16)
    nz, ny, nx = shape
    T, b = workloads.tangled_box(nx, ny, nz, 3)
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    rng = np.random.default_rng(5)
    target = torch.from_numpy(rng.normal(scale=1e-3, size=shape).astype(np.float32)).cuda()
    finals = []
    for _ in range(2):
        sur = rk._lib.rkl_sur_create(nz, ny, nx, (1.0 / nx, 1.0 / ny, 1.0 / nz),
                                     torch.cuda.current_stream().cuda_stream)
        prng = np.random.default_rng(0)
        for l in range(6):
            co, ci = rk._lib.rkl_sur_layer_shape(l)
            w = prng.normal(scale=np.sqrt(2.0 / (27 * ci)), size=(27, co, ci)).astype(np.float32)
            rk._lib.rkl_sur_set_params(sur, l, w, np.zeros(co, dtype=np.float32))
        rk._lib.rkl_sur_features(sur, Td, bd, 0.01, True, 100.0)
        losses = [rk._lib.rkl_sur_train_step(sur, 2e-3, target, 1e-3) for _ in range(3)]
        finals.append((losses, [rk._lib.rkl_sur_get_params(sur, l) for l in range(6)]))
        rk._lib.rkl_sur_destroy(sur)
    assert finals[0][0] == finals[1][0]
    for (w0, b0), (w1, b1) in zip(finals[0][1], finals[1][1]):
        assert np.array_equal(w0, w1) and np.array_equal(b0, b1)
