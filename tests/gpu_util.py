"""Helpers shared by the GPU tests: device transfer, oracle comparison."""
import math

import numpy as np

# FP32 GPU path against the FP64 oracle.  The method's state is O(1); an
# FP32 stage rounds each cell to ~6e-8 relative, and the flux differences
# that form M lose a further factor |T| / |T_{i+1} - T_i| ~ 1e2 of relative
# precision, which the divergence then multiplies by dx: the normalised
# max-abs error of F and M stays below 1e-5 of their maximum.  One
# super-step of s <= 40 stages accumulates at most ~s such roundings on
# the O(1) state, far inside the 1e-5 relative L2 target.
F32_FLUX_TOL = 1e-5          # max |F_gpu - F_ref| / max |F_ref|
F32_STATE_REL_L2 = 1e-5      # ||T_gpu - T_ref||_2 / ||T_ref||_2 (the method's stated bound)
F32_STATE_MAX = 2e-5         # max |T_gpu - T_ref| / max |T_ref|
F64_TOL = 1e-12              # FP64 GPU against the FP64 oracle (rounding order only)
# With MC-limited transverse gradients the operator is piecewise linear in T:
# where FP32 rounding moves a cell across a kink of the limiter (two of its
# candidates equal, or two one-sided differences of opposite sign), that
# cell's gradient changes slope by up to a factor 2, so over a super-step the
# worst cell can drift several times 1e-5 while the L2 error stays below 1e-5.
F32_LIMITER_MAX = 2e-4


def torch_dev(a, dtype="f32"):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if dtype == "f32" else np.float64))
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rounded(a, dtype="f32"):
    """The input exactly as the GPU sees it, back in FP64 for the oracle."""
    return np.asarray(a, dtype=np.float32 if dtype == "f32" else np.float64).astype(np.float64)


def rel_l2(a, ref):
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))


def norm_max(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def window(a, center, half, axes_first=0):
    """Periodic window of an array [..., z, y, x] around center (z, y, x)
    with side 2*half (indices center - half .. center + half - 1)."""
    idx = [np.arange(c - half, c + half) % n for c, n in zip(center, a.shape[axes_first:])]
    return a[(Ellipsis,) + np.ix_(*idx)]
