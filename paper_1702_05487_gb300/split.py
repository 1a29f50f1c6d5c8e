"""Operator-split driver (Section 3): each step advances the hyperbolic part
over dt_h (Eq. dt_h) without the conduction flux, then the conduction part
over the same dt_h.  The hyperbolic part is the library's passive donor-cell
advection of the energy density (`rkl_advect`); the conduction part is one
of the strategies whose cost Table 1 compares:

* ``"rkl2"``      one RKL2 super-step of length dt_h (s from dt_h / dt_expl);
* ``"subcycle"``  N = ceil(dt_h / dt_expl) forward-Euler steps of dt_h / N;
* ``"explicit"``  the whole system at the explicit step: N advection steps
                  of dt_h / N, each followed by one Euler conduction step.

Every step runs in the library's kernels; this module only sequences the
C-ABI calls.  The state alternates between two caller-owned device arrays
(the advection cannot run in place): ``step`` returns the one that holds it.
"""
from __future__ import annotations

import math

from . import Plan

STRATEGIES = ("rkl2", "subcycle", "explicit")


class SplitDriver:
    """Operator splitting on one grid.  ``params`` are the make_grid /
    make_phys keyword arguments of the conduction problem."""

    def __init__(self, shape, dtype="f32", params=None, stream=None, ch=0.8, strategy="rkl2"):
        if strategy not in STRATEGIES:
            raise ValueError(f"strategy must be one of {STRATEGIES}")
        self.ch = float(ch)
        self.strategy = strategy
        self.plan = Plan(shape, dtype, stream=stream, params=params)
        self.euler = None
        if strategy != "rkl2":
            # forward Euler = the one-stage RKL1 super-step
            self.euler = Plan(shape, dtype, stream=stream, params=params)
            self.euler.set_method("rkl1")

    def close(self):
        self.plan.close()
        if self.euler is not None:
            self.euler.close()

    def dt_h(self, u):
        return self.plan.dt_hyperbolic(u, self.ch)

    def substeps(self, dt, T):
        """Explicit steps needed to cover dt: ceil(dt / dt_expl(T))."""
        return max(1, math.ceil(dt / self.plan.dt_expl(T) - 1e-12))

    def step(self, T, T_other, b, u, dt=None, n=None):
        """One split step of length dt (default dt_h).  Returns (array holding
        the new state, dt, conduction stages run).  n fixes the number of
        explicit sub-steps of the "subcycle" / "explicit" strategies."""
        if dt is None:
            dt = self.dt_h(u)
        if self.strategy == "rkl2":
            self.plan.advect(dt, u, T, T_other)
            s = self.plan.super_step(dt, T_other, b)
            return T_other, dt, s
        n = n if n is not None else self.substeps(dt, T)
        if self.strategy == "subcycle":
            self.plan.advect(dt, u, T, T_other)
            for _ in range(n):
                self.euler.super_step_s(dt / n, 1, T_other, b)
            return T_other, dt, n
        cur, nxt = T, T_other
        for _ in range(n):
            self.plan.advect(dt / n, u, cur, nxt)
            self.euler.super_step_s(dt / n, 1, nxt, b)
            cur, nxt = nxt, cur
        return cur, dt, n


def table1_costs(t_hyp, t_stage, n, s):
    """Run-time model of one dt_h step per strategy (Table 1), from the
    measured time of one hyperbolic step (t_hyp) and of one conduction stage
    (t_stage), with n explicit steps per dt_h and s RKL2 stages."""
    return {"explicit": n * (t_hyp + t_stage), "subcycle": t_hyp + n * t_stage, "rkl2": t_hyp + s * t_stage}
