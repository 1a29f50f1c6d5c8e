"""FP64 CPU oracle of the learned surrogate (TEST INFRASTRUCTURE ONLY).

The surrogate of the batched-conduction workloads is a 6-layer 3D
convolutional network on periodic patches: 3x3x3 kernels, 32 hidden
channels, ReLU between layers, inputs (T, b_x, b_y, b_z, log kappa_par,
dt/dt_expl).  Its head outputs three face-flux channels G_d, and the
predicted super-step increment is the conservative divergence
dT = -tau * sum_d (G_d[c] - G_d[c - e_d]) / dx_d — the same one-flux-per-face
form as the conduction operator (Section 3 of the paper), so the predicted
increment conserves energy exactly.  This module states every step with
plain numpy in FP64 (arrays are channels-first [C][z][y][x]):

* ``conv3d``            - periodic 3x3x3 cross-correlation plus bias,
* ``conv3d_grad_input`` - its adjoint with respect to the input,
* ``conv3d_grad_weight``- its gradient with respect to weights and bias,
* ``forward`` / ``backward`` - the network, MSE loss on dT, chain rule,
* ``adam``              - one Adam update (Kingma & Ba 2015),
* ``round_bf16``        - the nearest BF16 value (8 significant bits, ties to
  even): with ``store=round_bf16`` the forward and backward passes round
  every value at the points where the network keeps it in BF16 (inputs,
  weights, hidden activations, back-propagated gradients), so that the
  cost of BF16 storage itself can be measured in FP64.

Only the test suite loads it; it shares nothing with the CUDA library.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, dz, dy, dx):
    """x[..., z + dz, y + dy, x + dx] with periodic wrap (channels first)."""
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv3d(x, w, bias):
    """y[co, v] = bias[co] + sum_{off, ci} w[co, ci, off] x[ci, v + off].
    x: [Ci, D, H, W]; w: [Co, Ci, 3, 3, 3] indexed [dz+1, dy+1, dx+1]."""
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for dz, dy, dx in OFFSETS:
        xs = _shift(x, dz, dy, dx)
        y += np.einsum("oi,izyx->ozyx", w[:, :, dz + 1, dy + 1, dx + 1], xs)
    return y + bias[:, None, None, None]


def conv3d_grad_input(gy, w):
    """dL/dx for y = conv3d(x, w, b): gx[ci, v] = sum_{off, co} w[co, ci, off] gy[co, v - off]."""
    gx = np.zeros((w.shape[1],) + gy.shape[1:])
    for dz, dy, dx in OFFSETS:
        gys = _shift(gy, -dz, -dy, -dx)
        gx += np.einsum("oi,ozyx->izyx", w[:, :, dz + 1, dy + 1, dx + 1], gys)
    return gx


def conv3d_grad_weight(gy, x):
    """dL/dw[co, ci, off] = sum_v gy[co, v] x[ci, v + off]; dL/db[co] = sum_v gy[co, v]."""
    gw = np.zeros((gy.shape[0], x.shape[0], 3, 3, 3))
    for dz, dy, dx in OFFSETS:
        xs = _shift(x, dz, dy, dx)
        gw[:, :, dz + 1, dy + 1, dx + 1] = np.einsum("ozyx,izyx->oi", gy, xs)
    return gw, gy.sum(axis=(1, 2, 3))


def round_bf16(a):
    """Round FP64 values to the nearest BF16 value (1 sign, 8 exponent and 7
    stored fraction bits: the FP64 significand cut to its top 7 fraction
    bits, round to nearest, ties to even), returned as FP64.  Valid for
    values inside BF16's normal range and zero."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    bits = a.view(np.uint64)
    drop = np.uint64(52 - 7)
    lsb = (bits >> drop) & np.uint64(1)
    half = (np.uint64(1) << (drop - np.uint64(1))) - np.uint64(1)
    out = (bits + half + lsb) & ~((np.uint64(1) << drop) - np.uint64(1))
    return out.view(np.float64)


def _identity(a):
    return a


def features(T, b, kappa0, spitzer, ratio, flux=None):
    """Network input channels [6][z][y][x]: T - 1, b_x, b_y, b_z,
    log10(kappa_par(T) / 0.01), (dt / dt_expl) / 100; with flux ([3][z][y]
    [x], the face fluxes of T already scaled) three more channels."""
    kap = kappa0 * T ** 2.5 if spitzer else np.full_like(T, kappa0)
    ch = [T - 1.0, b[0], b[1], b[2], np.log10(kap) + 2.0, np.full_like(T, ratio / 100.0)]
    if flux is not None:
        ch += [flux[0], flux[1], flux[2]]
    return np.stack(ch)


def flux_divergence(G, tau, dx):
    """dT = -tau * sum_d (G_d[c] - G_d[c - e_d]) / dx_d for G = [Gx, Gy, Gz]
    (G_d at cell c is the flux on face c + e_d / 2), periodic."""
    dT = np.zeros(G.shape[1:])
    for d, axis in ((0, -1), (1, -2), (2, -3)):
        dT -= (G[d] - np.roll(G[d], 1, axis=axis)) / dx[d]
    return tau * dT


def flux_divergence_adjoint(gdT, tau, dx):
    """Adjoint of flux_divergence: dL/dG given dL/d(dT)."""
    gG = np.zeros((3,) + gdT.shape)
    for d, axis in ((0, -1), (1, -2), (2, -3)):
        gG[d] = -tau * (gdT - np.roll(gdT, -1, axis=axis)) / dx[d]
    return gG


def forward(params, x, tau, dx, store=None):
    """params: list of (w, b) per layer; x: [6, D, H, W].  Returns (dT, cache).
    store (default: none) is applied to the input, the weights and every
    hidden activation, the values a BF16 network keeps in BF16."""
    store = store or _identity
    h = store(x)
    acts = [h]
    pre = []
    for li, (w, b) in enumerate(params):
        z = conv3d(h, store(w), b)
        pre.append(z)
        h = store(np.maximum(z, 0.0)) if li < len(params) - 1 else z
        acts.append(h)
    dT = flux_divergence(h, tau, dx)
    return dT, (acts, pre)


def loss_and_grad(params, x, target, tau, dx, store=None):
    """MSE loss 0.5 * mean((dT - target)^2) and its gradients per layer.
    store as in forward, also applied to the gradients propagated back to
    each layer's output (after the ReLU mask)."""
    store = store or _identity
    dT, (acts, pre) = forward(params, x, tau, dx, store)
    n = dT.size
    r = dT - target
    loss = 0.5 * float(np.sum(r * r)) / n
    g = store(flux_divergence_adjoint(r / n, tau, dx))
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        gw, gb = conv3d_grad_weight(g, acts[li])
        grads[li] = (gw, gb)
        if li > 0:
            # through layer li to the output of layer li - 1, then its ReLU
            g = store(conv3d_grad_input(g, store(w)) * (pre[li - 1] > 0.0))
    return loss, grads, dT


def adam(param, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments); returns (param, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v
