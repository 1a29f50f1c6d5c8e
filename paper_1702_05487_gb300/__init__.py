"""GB300 (sm_103a) RKL2 super-time-stepping of anisotropic thermal conduction.

The compute path is the CUDA library ``librkl.so`` (C ABI in
``include/rkl.h``); this package is its thin Python binding.  Device memory
and streams come from PyTorch; every step of the method runs in the
library's kernels.  There is no CPU fallback: without the built library (or
without a GPU) the calls raise.

``Plan`` wraps one ``rkl_plan`` for a grid, physics and stream.
"""
from __future__ import annotations

from dataclasses import dataclass

from ._lib import (  # noqa: F401  (the C ABI, same names)
    RKL_DIRICHLET, RKL_F32, RKL_F64, RKL_KAPPA_CONST, RKL_KAPPA_SPITZER, RKL_METHOD_RKL1, RKL_METHOD_RKL2,
    RKL_METHOD_STS, RKL_OK, RKL_PERIODIC, RklError, load, library_path, rkl_apply_M, rkl_coeffs,
    rkl_coeffs_method, rkl_dt_expl, rkl_energy, rkl_flux, rkl_grid, rkl_num_stages, rkl_num_stages_method,
    rkl_phys, rkl_plan_check, rkl_plan_create, rkl_plan_destroy, rkl_plan_set_method, rkl_plan_set_timing,
    rkl_plan_set_variant, rkl_plan_timing, rkl_run_host, rkl_run_host_batch, rkl_stage, rkl_super_step,
    rkl_super_step_s, rkl_advect, rkl_dt_hyperbolic,
)

__all__ = ["Plan", "make_grid", "make_phys", "RklError"]


def make_grid(shape, dx=None, bc="periodic", bc_value=0.0, dtype="f32") -> rkl_grid:
    """rkl_grid for an array of the given C-order shape ([z][y][x], [y][x] or [x])."""
    g = rkl_grid()
    nd = len(shape)
    g.ndim = nd
    nxyz = list(reversed([int(v) for v in shape])) + [1] * (3 - nd)
    dx = list(dx) if dx is not None else [1.0 / n for n in nxyz[:nd]]
    dx = dx + [1.0] * (3 - len(dx))
    for d in range(3):
        g.n[d] = nxyz[d]
        g.dx[d] = float(dx[d])
    g.bc = {"periodic": RKL_PERIODIC, "dirichlet": RKL_DIRICHLET}[bc]
    g.bc_value = float(bc_value)
    g.dtype = {"f32": RKL_F32, "f64": RKL_F64}[dtype]
    return g


def make_phys(kappa_model="const", kappa_par0=1.0, kappa_perp_ratio=0.0, saturate=False, phi=0.3,
              rho=1.0, sat_upwind=False, cp=0.5, limiter="none", limiter_floor=float("inf")) -> rkl_phys:
    p = rkl_phys()
    p.kappa_model = {"const": RKL_KAPPA_CONST, "spitzer": RKL_KAPPA_SPITZER}[kappa_model]
    p.kappa_par0 = float(kappa_par0)
    p.kappa_perp_ratio = float(kappa_perp_ratio)
    p.saturate = int(bool(saturate))
    p.phi = float(phi)
    p.rho = float(rho)
    p.sat_upwind = int(bool(sat_upwind))
    p.cp = float(cp)
    p.limiter = {"none": 0, "mc": 1}[limiter]
    p.limiter_floor = float(limiter_floor)
    return p


@dataclass
class Plan:
    """One rkl_plan.  ``params`` are make_grid / make_phys keyword arguments."""
    shape: tuple
    dtype: str = "f32"
    stream: object = None
    params: dict = None

    def __post_init__(self):
        import torch
        prm = dict(self.params or {})
        gkeys = {"dx", "bc", "bc_value"}
        grid = make_grid(self.shape, dtype=self.dtype, **{k: v for k, v in prm.items() if k in gkeys})
        phys = make_phys(**{k: v for k, v in prm.items() if k not in gkeys})
        if self.stream is None:
            self.stream = torch.cuda.current_stream()
        self.handle = rkl_plan_create(grid, phys, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            rkl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # thin forwarding methods (same semantics as the C ABI)
    def dt_expl(self, T):
        return rkl_dt_expl(self.handle, T)

    def flux(self, T, b, Fx, Fy=None, Fz=None):
        rkl_flux(self.handle, T, b, Fx, Fy, Fz)

    def apply_M(self, T, b, MT):
        rkl_apply_M(self.handle, T, b, MT)

    def stage(self, j, s, dt, b, Y0, MY0, Yjm1, Yjm2, Yj):
        rkl_stage(self.handle, j, s, dt, b, Y0, MY0, Yjm1, Yjm2, Yj)

    def super_step(self, dt, T, b, energies=False):
        return rkl_super_step(self.handle, dt, T, b, energies)

    def super_step_s(self, dt, s, T, b, energies=False):
        return rkl_super_step_s(self.handle, dt, s, T, b, energies)

    def energy(self, T):
        return rkl_energy(self.handle, T)

    def check(self):
        return rkl_plan_check(self.handle)

    def set_variant(self, variant, nzchunk=0):
        rkl_plan_set_variant(self.handle, variant, nzchunk)

    def dt_hyperbolic(self, u, ch=0.8):
        """Eq. dt_h for the advection velocity u ([3][cells] device array)."""
        return rkl_dt_hyperbolic(self.handle, u, ch)

    def advect(self, dt, u, T_in, T_out):
        """One donor-cell advection step of T_in into T_out (asynchronous)."""
        rkl_advect(self.handle, dt, u, T_in, T_out)

    def set_method(self, method, sts_nu=1e-3):
        """"rkl2" (default), "rkl1" or "sts" (AAG-STS with damping sts_nu)."""
        m = {"rkl2": RKL_METHOD_RKL2, "rkl1": RKL_METHOD_RKL1, "sts": RKL_METHOD_STS}.get(method, method)
        rkl_plan_set_method(self.handle, m, sts_nu)

    def autotune(self, dt, T, b):
        from . import _lib
        return _lib.rkl_plan_autotune(self.handle, dt, T, b)

    def set_timing(self, on):
        rkl_plan_set_timing(self.handle, on)

    def timing(self):
        return rkl_plan_timing(self.handle)

    def run_host(self, dt, n_super, T_host, b_host):
        return rkl_run_host(self.handle, dt, n_super, T_host, b_host)

    def run_host_batch(self, dt, n_super, T_hosts, b_hosts):
        return rkl_run_host_batch(self.handle, dt, n_super, T_hosts, b_hosts)


class Ensemble:
    """One rkl_ensemble: ``problems`` is a list of (shape, params) pairs with
    C-order 3D shapes and make_grid / make_phys keyword arguments."""

    def __init__(self, problems, stream=None):
        import torch
        from . import _lib
        gkeys = {"dx", "bc", "bc_value"}
        grids, physs = [], []
        for shape, prm in problems:
            prm = dict(prm or {})
            grids.append(make_grid(shape, dtype="f32", **{k: v for k, v in prm.items() if k in gkeys}))
            physs.append(make_phys(**{k: v for k, v in prm.items() if k not in gkeys}))
        self.shapes = [tuple(s) for s, _ in problems]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._lib = _lib
        self.handle = _lib.rkl_ensemble_create(grids, physs, self.stream.cuda_stream)
        self.offsets = _lib.rkl_ensemble_layout(self.handle, len(problems))

    def close(self):
        if getattr(self, "handle", None) is not None:
            self._lib.rkl_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def views(self, T_all, b_all):
        """Per-problem views (T_p, b_p) into the concatenated arrays."""
        out = []
        for p, shape in enumerate(self.shapes):
            o0, o1 = self.offsets[p], self.offsets[p + 1]
            out.append((T_all[o0:o1].view(shape), b_all[3 * o0:3 * o1].view((3,) + shape)))
        return out

    def set_schedule(self, persistent, nzchunk=0):
        self._lib.rkl_ensemble_set_schedule(self.handle, persistent, nzchunk)

    def super_step(self, dt, T_all, b_all):
        return self._lib.rkl_ensemble_super_step(self.handle, dt, T_all, b_all)

    def check(self):
        return self._lib.rkl_ensemble_check(self.handle)

    def autotune(self, dt, T_all, b_all):
        return self._lib.rkl_ensemble_autotune(self.handle, dt, T_all, b_all)

    def selftest_timeout(self):
        return self._lib.rkl_ensemble_selftest_timeout(self.handle)
