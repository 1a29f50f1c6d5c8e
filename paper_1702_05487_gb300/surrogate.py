"""Training and use of the learned surrogate of one RKL2 super-step.

Every numerical step runs in the library (rkl_sur_* and rkl_super_step of
include/rkl.h): the training pairs are produced by the plain RKL2 super-step
on the GPU, the network is trained by the library's own forward, backward
and Adam kernels, and a surrogate super-step is accepted only when its
trapezoidal-rule residual is below a threshold calibrated on held-out
pairs; otherwise the plain super-step runs (the fallback).  This module only
orchestrates: it draws training fields from a pool of seeded tangled-field
patches transformed by the cube's symmetries (axis permutations and
reflections, applied to b as a vector) and cyclic shifts, with the
conductivity and super-step length drawn per pair.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from . import Plan


def _comp_of_axis(a: int) -> int:
    # array axes (z, y, x) <-> vector components (x, y, z)
    return 2 - a


def augment(T, b, rng):
    """Random symmetry of the periodic cube applied to T [D,H,W] and the
    vector field b [3,D,H,W] (torch tensors): axis permutation, reflections,
    cyclic shifts."""
    import torch
    perm = list(rng.permutation(3))
    Tn = T.permute(perm)
    bn = torch.stack([b[_comp_of_axis(perm[_comp_of_axis(c)])].permute(perm) for c in range(3)])
    for a in range(3):
        if rng.random() < 0.5:
            Tn = Tn.flip(a)
            bn = bn.flip(a + 1)
            bn[_comp_of_axis(a)] = -bn[_comp_of_axis(a)]
    shifts = tuple(int(v) for v in rng.integers(0, Tn.shape[0], 3))
    Tn = torch.roll(Tn, shifts, dims=(0, 1, 2))
    bn = torch.roll(bn, shifts, dims=(1, 2, 3))
    return Tn.contiguous(), bn.contiguous()


@dataclass
class SurrogateConfig:
    n: int = 128                      # periodic patch side (cells)
    pool: int = 16                    # seeded base fields
    seed0: int = 10000
    kappa_range: tuple = (5e-3, 2e-2)
    ratio_range: tuple = (50.0, 150.0)
    kappa_perp_ratio: float = 1e-4
    lr: float = 2e-3
    head_scale: float = 0.0           # 0: set from the first targets
    flux_c: float = 0.0625            # > 0: flux features scaled by flux_c dt / head_scale (0: none)


@dataclass
class Surrogate:
    """A trained (or training) surrogate for periodic n^3 patches."""
    cfg: SurrogateConfig = field(default_factory=SurrogateConfig)

    def __post_init__(self):
        import torch
        import workloads
        n = self.cfg.n
        self.dx = (1.0 / n,) * 3
        self.stream = torch.cuda.current_stream()
        self.handle = _lib.rkl_sur_create(n, n, n, self.dx, self.stream.cuda_stream)
        self.rng = np.random.default_rng(self.cfg.seed0)
        self._init_params()
        _lib.rkl_sur_set_flux_features(self.handle, self.cfg.flux_c)
        pool_T, pool_b = [], []
        for k in range(self.cfg.pool):
            T, b = workloads.tangled_box(n, n, n, self.cfg.seed0 + k)
            pool_T.append(torch.from_numpy(T.astype(np.float32)).cuda())
            pool_b.append(torch.from_numpy(b.astype(np.float32)).cuda())
        self.pool = list(zip(pool_T, pool_b))
        self.plans = {}
        self.threshold = None

    def _init_params(self):
        for l in range(6):
            co, ci = _lib.rkl_sur_layer_shape(l)
            rci = (9 if self.cfg.flux_c > 0 else 6) if l == 0 else ci
            rco = 3 if l == 5 else co
            w = np.zeros((27, co, ci), dtype=np.float32)
            scale = math.sqrt(2.0 / (27 * rci)) * (0.1 if l == 5 else 1.0)
            w[:, :rco, :rci] = self.rng.normal(scale=scale, size=(27, rco, rci))
            b = np.zeros(co, dtype=np.float32)
            _lib.rkl_sur_set_params(self.handle, l, w, b)

    def close(self):
        if getattr(self, "handle", None) is not None:
            _lib.rkl_sur_destroy(self.handle)
            self.handle = None

    def plan(self, kappa0):
        key = round(float(kappa0), 12)
        if key not in self.plans:
            if len(self.plans) > 8:
                self.plans.clear()
            self.plans[key] = Plan((self.cfg.n,) * 3, "f32", stream=self.stream,
                                   params=dict(dx=self.dx, kappa_model="spitzer", kappa_par0=kappa0,
                                               kappa_perp_ratio=self.cfg.kappa_perp_ratio))
        return self.plans[key]

    # ------------------------------------------------------------------
    def draw(self, pool_index=None):
        """One training sample: (T0, b, kappa0, ratio, dt, dT_target), the
        target from the plain RKL2 super-step on the GPU."""
        k = int(self.rng.integers(0, len(self.pool))) if pool_index is None else pool_index
        T0, b = augment(*self.pool[k], self.rng)
        kappa0 = float(math.exp(self.rng.uniform(*map(math.log, self.cfg.kappa_range))))
        ratio = float(self.rng.uniform(*self.cfg.ratio_range))
        plan = self.plan(kappa0)
        dt = ratio * plan.dt_expl(T0)
        T1 = T0.clone()
        plan.super_step(dt, T1, b)
        return T0, b, kappa0, ratio, dt, (T1 - T0).contiguous()

    def train(self, n_pairs, log_every=0):
        """Train on n_pairs freshly drawn RKL2 pairs (one Adam step each)."""
        losses = []
        for i in range(n_pairs):
            T0, b, kappa0, ratio, dt, target = self.draw()
            if self.cfg.head_scale <= 0.0:
                rms = float(target.double().pow(2).mean().sqrt())
                self.cfg.head_scale = rms * self.dx[0]
            self._features(T0, b, kappa0, ratio, dt)
            lr = self.cfg.lr * (0.5 * (1 + math.cos(math.pi * i / max(1, n_pairs))) * 0.9 + 0.1)
            losses.append(_lib.rkl_sur_train_step(self.handle, self.cfg.head_scale, target, lr))
            if log_every and (i + 1) % log_every == 0:
                print(f"pair {i + 1}/{n_pairs}: loss {np.mean(losses[-log_every:]):.4e}", flush=True)
        return losses

    def _features(self, T0, b, kappa0, ratio, dt):
        if self.cfg.flux_c > 0.0:
            _lib.rkl_sur_features_flux(self.handle, self.plan(kappa0).handle, T0, b, ratio,
                                       self.cfg.flux_c * dt / self.cfg.head_scale)
        else:
            _lib.rkl_sur_features(self.handle, T0, b, kappa0, True, ratio)

    def predict(self, T0, b, kappa0, ratio):
        import torch
        dT = torch.empty_like(T0)
        dt = ratio * self.plan(kappa0).dt_expl(T0)
        self._features(T0, b, kappa0, ratio, dt)
        _lib.rkl_sur_forward(self.handle, self.cfg.head_scale, dT)
        return dT

    def heldout_pool(self, count=4):
        """Tangled-field patches of seeds the training pool does not use."""
        import torch
        import workloads
        n = self.cfg.n
        out = []
        for k in range(count):
            T, b = workloads.tangled_box(n, n, n, self.cfg.seed0 + 2000 + k)
            out.append((torch.from_numpy(T.astype(np.float32)).cuda(), torch.from_numpy(b.astype(np.float32)).cuda()))
        return out

    def calibrate(self, n_pairs, accuracy=1e-3):
        """Held-out pairs (fields outside the training pool, their own seeded
        draws): the true state error ||T_pred - T_rkl2|| / ||T_rkl2|| and the
        residual of each prediction; the threshold is the largest residual
        below which every held-out prediction met `accuracy`."""
        rows = []
        train_pool, train_rng = self.pool, self.rng
        self.pool, self.rng = self.heldout_pool(), np.random.default_rng(self.cfg.seed0 + 3000)
        for _ in range(n_pairs):
            T0, b, kappa0, ratio, dt, target = self.draw()
            plan = self.plan(kappa0)
            Tp = T0.clone()
            acc, rho, _ = _lib.rkl_sur_super_step(self.handle, plan.handle, dt, Tp, b, self.cfg.head_scale,
                                                  float("inf"))
            Tt = T0 + target
            err = float((Tp - Tt).double().norm() / Tt.double().norm())
            rows.append((rho, err))
        self.pool, self.rng = train_pool, train_rng
        rows.sort()
        thr = 0.0
        for rho, err in rows:
            if err > accuracy:
                break
            thr = rho
        self.threshold = thr
        return thr, rows

    def time_to_solution(self, n_steps, kappa0=0.01, ratio=100.0, seed=None, accuracy=1e-3):
        """n_steps super-steps from one held-out field (tangled-field seed
        outside the training pool; default seed0 + 1000), plain RKL2 against
        the surrogate with fallback; wall times on the GPU (CUDA events) and
        the surrogate run's final relative L2 error against the plain run."""
        import torch
        import workloads
        n = self.cfg.n
        Th, bh = workloads.tangled_box(n, n, n, self.cfg.seed0 + 1000 if seed is None else seed)
        T0 = torch.from_numpy(Th.astype(np.float32)).cuda()
        b = torch.from_numpy(bh.astype(np.float32)).cuda()
        plan = self.plan(kappa0)
        dt = ratio * plan.dt_expl(T0)
        thr = self.threshold if self.threshold is not None else 0.0

        def run(use_sur, threshold=thr):
            T = T0.clone()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            accepted = 0
            torch.cuda.synchronize()
            ev0.record(self.stream)
            for _ in range(n_steps):
                if use_sur:
                    acc, _, _ = _lib.rkl_sur_super_step(self.handle, plan.handle, dt, T, b, self.cfg.head_scale,
                                                        threshold)
                    accepted += int(acc)
                else:
                    plan.super_step(dt, T, b)
            ev1.record(self.stream)
            torch.cuda.synchronize()
            return T, ev0.elapsed_time(ev1), accepted

        run(False)
        run(True)                                   # warm-up of both paths
        Tr, ms_r, _ = run(False)
        Ts, ms_s, acc = run(True)
        err = float((Ts - Tr).double().norm() / Tr.double().norm())
        # the same run with every prediction accepted: what a step of the
        # surrogate costs against one of RKL2, and the error it would carry
        Ta, ms_a, _ = run(True, float("inf"))
        err_a = float((Ta - Tr).double().norm() / Tr.double().norm())
        return dict(steps=n_steps, rkl2_ms=ms_r, surrogate_ms=ms_s, accepted=acc, rel_l2_vs_rkl2=err,
                    threshold=thr, accuracy_target=accuracy, speedup=ms_r / ms_s,
                    all_accepted=dict(surrogate_ms=ms_a, speedup=ms_r / ms_a, rel_l2_vs_rkl2=err_a))
