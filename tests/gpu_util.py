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


# A priori bound on the FP32 error of a sequence of super-steps, for the
# change T - T0, whose norm can be two orders below the state's.
#
# Each stage stores Y_j rounded to FP32 and adds the FP32 rounding of its
# terms (the recurrence's fused multiply-adds, the flux arithmetic of
# tau M): model that as a perturbation of at most C_STAGE roundings of the
# stored value per cell, random in sign (u = 2^-24, rms u/sqrt(3) for a
# uniformly distributed rounding error), so its 2-norm is C_STAGE u/sqrt(3)
# ||T||.  A perturbation e of stage k reaches the super-step's result through
# the homogeneous part of Eq. rkl2scheme, e_j = mu_j e_{j-1} + nu_j e_{j-2}
# (e_{k-1} = 0, e_k = e): on the smoothest modes, which M does not damp,
# this multiplies it by A_k(s) (about 1 + k ln(s/k) for large s).  Rougher
# modes are damped by the tau M terms, so A_k bounds them too.  Independent
# perturbations add in quadrature over the stages and over the n
# super-steps (smooth modes pass later super-steps unchanged):
#     ||T_gpu - T_ref|| <= C_STAGE u/sqrt(3) sqrt(sum_steps sum_k A_k(s)^2) ||T_ref||
# and the same absolute error measured against ||T_ref - T0||.
C_STAGE = 2.0
U32 = 2.0 ** -24


def stage_amplification(orc, s: int) -> np.ndarray:
    """A_k(s), k = 1..s: the factor by which a perturbation of Y_k reaches
    Y_s through e_j = mu_j e_{j-1} + nu_j e_{j-2} (Appendix A coefficients)."""
    mu, nu, _, _ = orc.coeffs(s)
    out = np.zeros(s)
    for k in range(1, s + 1):
        e = np.zeros(s + 1)
        e[k] = 1.0
        for j in range(k + 1, s + 1):
            e[j] = mu[j] * e[j - 1] + nu[j] * e[j - 2]
        out[k - 1] = abs(e[s])
    return out


def f32_state_model(orc, stage_counts) -> float:
    """The model bound on ||T_gpu - T_ref|| / ||T_ref|| after super-steps
    with the given stage counts."""
    acc = sum(float((stage_amplification(orc, s) ** 2).sum()) for s in stage_counts)
    return C_STAGE * U32 / math.sqrt(3.0) * math.sqrt(acc)


def change_errors(Tg, Tref, T0):
    """(rel-L2, normalised L-inf) of the change T - T0 and of the state."""
    d_ref = Tref - T0
    err = Tg - Tref
    return dict(rel_l2_T=rel_l2(Tg, Tref), linf_T=norm_max(Tg, Tref),
                rel_l2_dT=float(np.linalg.norm(err.ravel()) / np.linalg.norm(d_ref.ravel())),
                linf_dT=float(np.max(np.abs(err)) / np.max(np.abs(d_ref))),
                change_over_state=float(np.linalg.norm(d_ref.ravel()) / np.linalg.norm(Tref.ravel())))


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
