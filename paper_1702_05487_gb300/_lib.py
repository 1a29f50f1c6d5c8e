"""ctypes binding of librkl.so: the C ABI of include/rkl.h, one Python function
per entry point with the same name.  Argument marshalling only; every step of
the computation runs in the library's CUDA kernels.

Device arrays are passed as torch CUDA tensors (their data pointers are
handed to the library); host arrays for ``rkl_run_host`` are numpy arrays or
CPU tensors.  Errors raise ``RklError`` carrying the status and the plan's
message.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RKL_OK = 0
RKL_ERR_INVALID_ARG = 1
RKL_ERR_CUDA = 2
RKL_ERR_NONFINITE = 3
RKL_ERR_NONPOSITIVE_T = 4
RKL_ERR_TIMEOUT = 5
RKL_ERR_UNSUPPORTED = 6
RKL_ERR_NOMEM = 7

RKL_PERIODIC, RKL_DIRICHLET = 0, 1
RKL_F32, RKL_F64 = 0, 1
RKL_METHOD_RKL2, RKL_METHOD_RKL1, RKL_METHOD_STS = 0, 1, 2
RKL_KAPPA_CONST, RKL_KAPPA_SPITZER = 0, 1


class RklError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


class rkl_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int), ("bc_value", ctypes.c_double), ("dtype", ctypes.c_int)]


class rkl_phys(ctypes.Structure):
    _fields_ = [("kappa_model", ctypes.c_int), ("kappa_par0", ctypes.c_double),
                ("kappa_perp_ratio", ctypes.c_double), ("saturate", ctypes.c_int),
                ("phi", ctypes.c_double), ("rho", ctypes.c_double), ("sat_upwind", ctypes.c_int),
                ("cp", ctypes.c_double), ("limiter", ctypes.c_int), ("limiter_floor", ctypes.c_double)]


# Every symbol include/rkl.h declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "rkl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rkl_last_error": (ctypes.c_char_p, [_vp]),
    "rkl_num_stages": (ctypes.c_int, [ctypes.c_double, _ip]),
    "rkl_coeffs": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp, _dp]),
    "rkl_num_stages_method": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip]),
    "rkl_coeffs_method": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]),
    "rkl_plan_set_method": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double]),
    "rkl_dt_hyperbolic": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _dp]),
    "rkl_advect": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, _vp]),
    "rkl_plan_create": (ctypes.c_int, [ctypes.POINTER(rkl_grid), ctypes.POINTER(rkl_phys), _vp,
                                       ctypes.POINTER(_vp)]),
    "rkl_plan_destroy": (ctypes.c_int, [_vp]),
    "rkl_dt_expl": (ctypes.c_int, [_vp, _vp, _dp]),
    "rkl_flux": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "rkl_apply_M": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "rkl_stage": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp,
                                 _vp, _vp, _vp]),
    "rkl_super_step": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, _ip, _dp, _dp]),
    "rkl_super_step_s": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp, _vp, _dp, _dp]),
    "rkl_energy": (ctypes.c_int, [_vp, _vp, _dp]),
    "rkl_plan_check": (ctypes.c_int, [_vp]),
    "rkl_plan_set_variant": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "rkl_plan_autotune": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, _ip, _ip, _dp]),
    "rkl_plan_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rkl_plan_timing": (ctypes.c_int, [_vp, _dp, _i64p]),
    "rkl_run_host": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp, _vp, _ip]),
    "rkl_run_host_batch": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip]),
    "rkl_dt_expl_energy_noalloc": (ctypes.c_int, [ctypes.POINTER(rkl_grid), ctypes.POINTER(rkl_phys), _vp,
                                                  _vp, _dp, _dp]),
    "rkl_ensemble_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(rkl_grid), ctypes.POINTER(rkl_phys), _vp,
                                           ctypes.POINTER(_vp)]),
    "rkl_ensemble_destroy": (ctypes.c_int, [_vp]),
    "rkl_ensemble_last_error": (ctypes.c_char_p, [_vp]),
    "rkl_ensemble_layout": (ctypes.c_int, [_vp, _i64p]),
    "rkl_ensemble_set_schedule": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "rkl_ensemble_super_step": (ctypes.c_int, [_vp, _dp, _vp, _vp, _ip]),
    "rkl_ensemble_check": (ctypes.c_int, [_vp]),
    "rkl_ensemble_autotune": (ctypes.c_int, [_vp, _dp, _vp, _vp, _ip, _ip, _dp]),
    "rkl_ensemble_selftest_timeout": (ctypes.c_int, [_vp, _ip]),
    "rkl_sur_layer_shape": (ctypes.c_int, [ctypes.c_int, _ip, _ip]),
    "rkl_sur_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _vp, ctypes.POINTER(_vp)]),
    "rkl_sur_destroy": (ctypes.c_int, [_vp]),
    "rkl_sur_last_error": (ctypes.c_char_p, [_vp]),
    "rkl_sur_set_params": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "rkl_sur_get_params": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "rkl_sur_get_grads": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "rkl_sur_features": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_double]),
    "rkl_sur_set_backend": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rkl_sur_check": (ctypes.c_int, [_vp]),
    "rkl_sur_forward": (ctypes.c_int, [_vp, ctypes.c_double, _vp]),
    "rkl_sur_backward": (ctypes.c_int, [_vp, _vp, _dp]),
    "rkl_sur_adam": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "rkl_sur_train_step": (ctypes.c_int, [_vp, ctypes.c_double, _vp, ctypes.c_double, _dp]),
    "rkl_sur_super_step": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                          _ip, _dp, _ip]),
    "rkl_sur_features_flux": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double]),
    "rkl_sur_set_flux_features": (ctypes.c_int, [_vp, ctypes.c_double]),
    "rkl_sur_layer_forward": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "rkl_sur_layer_backward_data": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "rkl_sur_layer_weight_grad": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load librkl.so (building it first if missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing: build it with paper_1702_05487_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(st: int) -> str:
    return load().rkl_status_string(int(st)).decode()


def _ptr(t):
    """Data pointer of a torch tensor / numpy array (None passes NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _check(st: int, plan=None):
    if st != RKL_OK:
        msg = load().rkl_last_error(plan).decode() if plan is not None or st else ""
        raise RklError(st, msg)


def rkl_num_stages(ratio: float) -> int:
    s = ctypes.c_int(0)
    _check(load().rkl_num_stages(float(ratio), ctypes.byref(s)))
    return s.value


def rkl_coeffs(s: int):
    import numpy as np
    arrs = [np.zeros(s + 1) for _ in range(4)]
    _check(load().rkl_coeffs(int(s), *[a.ctypes.data_as(_dp) for a in arrs]))
    return tuple(arrs)


def rkl_num_stages_method(method: int, ratio: float, sts_nu: float = 1e-3) -> int:
    s = ctypes.c_int(0)
    _check(load().rkl_num_stages_method(int(method), float(ratio), float(sts_nu), ctypes.byref(s)))
    return s.value


def rkl_coeffs_method(method: int, s: int, sts_nu: float = 1e-3):
    import numpy as np
    arrs = [np.zeros(s + 1) for _ in range(4)]
    _check(load().rkl_coeffs_method(int(method), int(s), float(sts_nu), *[a.ctypes.data_as(_dp) for a in arrs]))
    return tuple(arrs)


def rkl_plan_set_method(plan, method: int, sts_nu: float = 1e-3):
    _check(load().rkl_plan_set_method(plan, int(method), float(sts_nu)), plan)


def rkl_dt_hyperbolic(plan, u, ch: float) -> float:
    dt = ctypes.c_double(0.0)
    _check(load().rkl_dt_hyperbolic(plan, _ptr(u), float(ch), ctypes.byref(dt)), plan)
    return dt.value


def rkl_advect(plan, dt: float, u, T_in, T_out):
    _check(load().rkl_advect(plan, float(dt), _ptr(u), _ptr(T_in), _ptr(T_out)), plan)


def rkl_plan_create(grid: rkl_grid, phys: rkl_phys, stream=None):
    h = _vp()
    st = load().rkl_plan_create(ctypes.byref(grid), ctypes.byref(phys),
                                _vp(int(stream) if stream else 0), ctypes.byref(h))
    if st != RKL_OK:
        raise RklError(st, load().rkl_last_error(None).decode())
    return h


def rkl_plan_destroy(plan):
    _check(load().rkl_plan_destroy(plan))


def rkl_dt_expl(plan, T) -> float:
    out = ctypes.c_double(0.0)
    _check(load().rkl_dt_expl(plan, _ptr(T), ctypes.byref(out)), plan)
    return out.value


def rkl_flux(plan, T, b, Fx, Fy=None, Fz=None):
    _check(load().rkl_flux(plan, _ptr(T), _ptr(b), _ptr(Fx), _ptr(Fy), _ptr(Fz)), plan)


def rkl_apply_M(plan, T, b, MT):
    _check(load().rkl_apply_M(plan, _ptr(T), _ptr(b), _ptr(MT)), plan)


def rkl_stage(plan, j, s, dt, b, Y0, MY0, Yjm1, Yjm2, Yj):
    _check(load().rkl_stage(plan, int(j), int(s), float(dt), _ptr(b), _ptr(Y0), _ptr(MY0),
                            _ptr(Yjm1), _ptr(Yjm2), _ptr(Yj)), plan)


def rkl_super_step(plan, dt, T, b, energies: bool = False):
    """Returns s, or (s, energy_before, energy_after) with energies=True."""
    s = ctypes.c_int(0)
    eb, ea = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().rkl_super_step(plan, float(dt), _ptr(T), _ptr(b), ctypes.byref(s),
                                 ctypes.byref(eb) if energies else None,
                                 ctypes.byref(ea) if energies else None), plan)
    return (s.value, eb.value, ea.value) if energies else s.value


def rkl_super_step_s(plan, dt, s, T, b, energies: bool = False):
    eb, ea = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().rkl_super_step_s(plan, float(dt), int(s), _ptr(T), _ptr(b),
                                   ctypes.byref(eb) if energies else None,
                                   ctypes.byref(ea) if energies else None), plan)
    return (eb.value, ea.value) if energies else None


def rkl_energy(plan, T) -> float:
    out = ctypes.c_double(0.0)
    _check(load().rkl_energy(plan, _ptr(T), ctypes.byref(out)), plan)
    return out.value


def rkl_plan_check(plan) -> int:
    """Returns the device status (RKL_OK or an error code) without raising."""
    return load().rkl_plan_check(plan)


def rkl_plan_set_variant(plan, variant: int, nzchunk: int = 0):
    _check(load().rkl_plan_set_variant(plan, int(variant), int(nzchunk)), plan)


def rkl_plan_autotune(plan, dt, T, b):
    """Returns (variant, nzchunk, ms of one super-step) of the fastest kernel."""
    v, nz, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().rkl_plan_autotune(plan, float(dt), _ptr(T), _ptr(b), ctypes.byref(v), ctypes.byref(nz),
                                    ctypes.byref(ms)), plan)
    return v.value, nz.value, ms.value


def rkl_plan_set_timing(plan, on: bool):
    _check(load().rkl_plan_set_timing(plan, int(bool(on))), plan)


def rkl_plan_timing(plan):
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    _check(load().rkl_plan_timing(plan, ctypes.byref(ms), ctypes.byref(n)), plan)
    return ms.value, n.value


def rkl_run_host(plan, dt, n_super, T_host, b_host) -> int:
    s = ctypes.c_int(0)
    _check(load().rkl_run_host(plan, float(dt), int(n_super), _ptr(T_host), _ptr(b_host),
                               ctypes.byref(s)), plan)
    return s.value


def rkl_run_host_batch(plan, dt, n_super, T_hosts, b_hosts) -> list:
    """Jobs (T_hosts[i], b_hosts[i]) streamed through the GPU with copies
    overlapping compute; returns each job's last s."""
    n = len(T_hosts)
    if len(b_hosts) != n:
        raise ValueError("one b array per T array")
    Tp = (_vp * max(n, 1))(*[_ptr(t) for t in T_hosts])
    bp = (_vp * max(n, 1))(*[_ptr(b) for b in b_hosts])
    s = (ctypes.c_int * max(n, 1))()
    _check(load().rkl_run_host_batch(plan, float(dt), int(n_super), n, Tp, bp, s), plan)
    return list(s)[:n]


def rkl_dt_expl_energy_noalloc(grid: rkl_grid, phys: rkl_phys, T, stream=None):
    """(dt_expl, energy) of a device array without a plan and without any
    device allocation (scratch is a fixed array inside the library)."""
    dt, e = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().rkl_dt_expl_energy_noalloc(ctypes.byref(grid), ctypes.byref(phys), _ptr(T),
                                           _vp(int(stream) if stream else 0), ctypes.byref(dt),
                                           ctypes.byref(e))
    if st != RKL_OK:
        raise RklError(st, load().rkl_last_error(None).decode())
    return dt.value, e.value


def _echeck(st: int, ens):
    if st != RKL_OK:
        raise RklError(st, load().rkl_ensemble_last_error(ens).decode())


def rkl_ensemble_create(grids, physs, stream=None):
    n = len(grids)
    ga = (rkl_grid * n)(*grids)
    pa = (rkl_phys * n)(*physs)
    h = _vp()
    st = load().rkl_ensemble_create(n, ga, pa, _vp(int(stream) if stream else 0), ctypes.byref(h))
    if st != RKL_OK:
        raise RklError(st, load().rkl_last_error(None).decode())
    return h


def rkl_ensemble_destroy(ens):
    _echeck(load().rkl_ensemble_destroy(ens), None)


def rkl_ensemble_layout(ens, nprob: int):
    out = (ctypes.c_int64 * (nprob + 1))()
    _echeck(load().rkl_ensemble_layout(ens, out), ens)
    return list(out)


def rkl_ensemble_set_schedule(ens, persistent: int, nzchunk: int = 0):
    _echeck(load().rkl_ensemble_set_schedule(ens, int(persistent), int(nzchunk)), ens)


def rkl_ensemble_super_step(ens, dt, T_all, b_all):
    """dt: sequence of per-problem super-steps; returns the list of s used."""
    n = len(dt)
    dts = (ctypes.c_double * n)(*[float(v) for v in dt])
    s = (ctypes.c_int * n)()
    _echeck(load().rkl_ensemble_super_step(ens, dts, _ptr(T_all), _ptr(b_all), s), ens)
    return list(s)


def rkl_ensemble_check(ens) -> int:
    return load().rkl_ensemble_check(ens)


def rkl_ensemble_autotune(ens, dt, T_all, b_all):
    n = len(dt)
    dts = (ctypes.c_double * n)(*[float(v) for v in dt])
    pers, nz, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _echeck(load().rkl_ensemble_autotune(ens, dts, _ptr(T_all), _ptr(b_all), ctypes.byref(pers),
                                         ctypes.byref(nz), ctypes.byref(ms)), ens)
    return pers.value, nz.value, ms.value


def rkl_ensemble_selftest_timeout(ens) -> int:
    out = ctypes.c_int(0)
    _echeck(load().rkl_ensemble_selftest_timeout(ens, ctypes.byref(out)), ens)
    return out.value


def _scheck(st: int, sur):
    if st != RKL_OK:
        raise RklError(st, load().rkl_sur_last_error(sur).decode())


def rkl_sur_layer_shape(layer: int):
    co, ci = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().rkl_sur_layer_shape(int(layer), ctypes.byref(co), ctypes.byref(ci)))
    return co.value, ci.value


def rkl_sur_create(D, H, W, dx, stream=None):
    dxa = (ctypes.c_double * 3)(*[float(v) for v in dx])
    h = _vp()
    st = load().rkl_sur_create(int(D), int(H), int(W), dxa, _vp(int(stream) if stream else 0), ctypes.byref(h))
    if st != RKL_OK:
        raise RklError(st, load().rkl_last_error(None).decode())
    return h


def rkl_sur_destroy(sur):
    _scheck(load().rkl_sur_destroy(sur), None)


def rkl_sur_set_params(sur, layer, w, b):
    """w, b: contiguous float32 numpy arrays ([27][cout][cin], [cout])."""
    _scheck(load().rkl_sur_set_params(sur, int(layer), _ptr(w), _ptr(b)), sur)


def rkl_sur_get_params(sur, layer):
    import numpy as np
    co, ci = rkl_sur_layer_shape(layer)
    w = np.zeros((27, co, ci), dtype=np.float32)
    b = np.zeros(co, dtype=np.float32)
    _scheck(load().rkl_sur_get_params(sur, int(layer), _ptr(w), _ptr(b)), sur)
    return w, b


def rkl_sur_get_grads(sur, layer):
    import numpy as np
    co, ci = rkl_sur_layer_shape(layer)
    w = np.zeros((27, co, ci), dtype=np.float32)
    b = np.zeros(co, dtype=np.float32)
    _scheck(load().rkl_sur_get_grads(sur, int(layer), _ptr(w), _ptr(b)), sur)
    return w, b


def rkl_sur_layer_forward(sur, layer, x, out):
    """One layer's forward convolution on device tensors (bf16 [V][cin] in)."""
    _scheck(load().rkl_sur_layer_forward(sur, int(layer), _ptr(x), _ptr(out)), sur)


def rkl_sur_layer_backward_data(sur, layer, dz, mask, out):
    """One layer's backward-data convolution, masked by mask > 0."""
    _scheck(load().rkl_sur_layer_backward_data(sur, int(layer), _ptr(dz), _ptr(mask), _ptr(out)), sur)


def rkl_sur_layer_weight_grad(sur, layer, dz, x):
    """One layer's weight and bias gradients (read them with rkl_sur_get_grads)."""
    _scheck(load().rkl_sur_layer_weight_grad(sur, int(layer), _ptr(dz), _ptr(x)), sur)


def rkl_sur_features(sur, T, b, kappa_par0, spitzer, ratio):
    _scheck(load().rkl_sur_features(sur, _ptr(T), _ptr(b), float(kappa_par0), int(bool(spitzer)), float(ratio)), sur)


def rkl_sur_features_flux(sur, plan, T, b, ratio, flux_scale):
    """Features with flux_scale times T's face fluxes (as the plan evaluates
    them) in channels 6, 7, 8."""
    _scheck(load().rkl_sur_features_flux(sur, plan, _ptr(T), _ptr(b), float(ratio), float(flux_scale)), sur)


def rkl_sur_set_flux_features(sur, c):
    """c > 0: rkl_sur_super_step uses flux features scaled by c dt / head_scale."""
    _scheck(load().rkl_sur_set_flux_features(sur, float(c)), sur)


def rkl_sur_set_backend(sur, backend: int):
    """0: warp-level mma.sync convolutions, 1: tcgen05 convolutions."""
    _scheck(load().rkl_sur_set_backend(sur, int(backend)), sur)


def rkl_sur_check(sur):
    _scheck(load().rkl_sur_check(sur), sur)


def rkl_sur_forward(sur, head_scale, dT_out=None):
    _scheck(load().rkl_sur_forward(sur, float(head_scale), _ptr(dT_out)), sur)


def rkl_sur_backward(sur, target) -> float:
    loss = ctypes.c_double(0.0)
    _scheck(load().rkl_sur_backward(sur, _ptr(target), ctypes.byref(loss)), sur)
    return loss.value


def rkl_sur_adam(sur, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _scheck(load().rkl_sur_adam(sur, float(lr), float(beta1), float(beta2), float(eps)), sur)


def rkl_sur_train_step(sur, head_scale, target, lr) -> float:
    loss = ctypes.c_double(0.0)
    _scheck(load().rkl_sur_train_step(sur, float(head_scale), _ptr(target), float(lr), ctypes.byref(loss)), sur)
    return loss.value


def rkl_sur_super_step(sur, plan, dt, T, b, head_scale, threshold):
    """Returns (accepted, residual, s_used)."""
    acc, res, s = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
    _scheck(load().rkl_sur_super_step(sur, plan, float(dt), _ptr(T), _ptr(b), float(head_scale), float(threshold),
                                      ctypes.byref(acc), ctypes.byref(res), ctypes.byref(s)), sur)
    return bool(acc.value), res.value, s.value
