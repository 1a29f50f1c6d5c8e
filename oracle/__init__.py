"""FP64 CPU oracle for the RKL2 super-step (Vaidya et al. 2017, arXiv:1702.05487).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow statement of what the
GPU library computes; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library (``paper_1702_05487_gb300``) and imports nothing from it.

The arithmetic lives in ``rkl_oracle.c`` (plain loops, FP64), compiled with
gcc on first use.  This module only marshals numpy arrays into it.  Function
by function, the paper passage each one follows:

* ``face_flux`` / ``flux``  - Eqs. Fclass, Fclass_HD, Fc, Fsat with the normal
  gradient across the face and the transverse gradients of Eqs. qN, qT
  (Appendix B) averaged to the face.
* ``apply_M``               - the conservative divergence of Section 3.
* ``dt_expl``               - Eq. dt_exp.
* ``num_stages``            - Eq. RKL-s (RKL2 row) with s -> 1 + floor(s)
  (Section 4.1).
* ``coeffs``                - Appendix A (b_j, a_j, w_1, mu_j, nu_j, mu~_j,
  gamma~_j).
* ``stage`` / ``super_step``- Eq. rkl2scheme.
* ``rkl2_scalar``           - Eq. rkl2scheme applied to dY/dt = lambda Y, i.e.
  the stability polynomial R_s(z) of Eq. stabpara.
* ``euler_step``            - forward Euler, the s = 1 case (Section 3.3).
* ``energy``                - sum of T dV (E = T for rho = 1, gamma = 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rkl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liborc.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_long * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", ctypes.c_int),
        ("bc_value", ctypes.c_double),
        ("kappa_model", ctypes.c_int),
        ("kappa_par0", ctypes.c_double),
        ("kappa_perp_ratio", ctypes.c_double),
        ("saturate", ctypes.c_int),
        ("phi", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("sat_upwind", ctypes.c_int),
        ("cp", ctypes.c_double),
        ("limiter", ctypes.c_int),
        ("limiter_floor", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_face_flux.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_long]
        lib.orc_face_flux.restype = ctypes.c_double
        lib.orc_flux.argtypes = [P, dp, dp, dp, dp, dp]
        lib.orc_apply_M.argtypes = [P, dp, dp, dp]
        lib.orc_dt_expl.argtypes = [P, dp]
        lib.orc_dt_expl.restype = ctypes.c_double
        lib.orc_num_stages.argtypes = [ctypes.c_double]
        lib.orc_num_stages.restype = ctypes.c_int
        lib.orc_coeffs.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        lib.orc_stage.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp, dp]
        lib.orc_super_step.argtypes = [P, ctypes.c_double, ctypes.c_int, dp, dp, dp]
        lib.orc_super_step.restype = ctypes.c_int
        lib.orc_euler_step.argtypes = [P, ctypes.c_double, dp, dp]
        lib.orc_energy.argtypes = [P, dp]
        lib.orc_energy.restype = ctypes.c_double
        lib.orc_rkl2_scalar.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_rkl2_scalar.restype = ctypes.c_double
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_num_stages_rkl1.argtypes = [ctypes.c_double]
        lib.orc_num_stages_rkl1.restype = ctypes.c_int
        lib.orc_rkl1_super_step.argtypes = [P, ctypes.c_double, ctypes.c_int, dp, dp]
        lib.orc_rkl1_super_step.restype = ctypes.c_int
        lib.orc_rkl1_scalar.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_rkl1_scalar.restype = ctypes.c_double
        lib.orc_sts_gain.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_sts_gain.restype = ctypes.c_double
        lib.orc_num_stages_sts.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_num_stages_sts.restype = ctypes.c_int
        lib.orc_sts_substeps.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_sts_super_step.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.orc_sts_super_step.restype = ctypes.c_int
        lib.orc_dt_hyp.argtypes = [P, dp, ctypes.c_double]
        lib.orc_dt_hyp.restype = ctypes.c_double
        lib.orc_advect.argtypes = [P, ctypes.c_double, dp, dp, dp]
        _lib = lib
        return lib


@dataclass
class Problem:
    """Grid and physics of one conduction problem (arrays are [z][y][x])."""
    shape: tuple                     # (nz, ny, nx) for 3D, (ny, nx) for 2D, (nx,) for 1D
    dx: tuple = None                 # spacing per axis in (x, y, z) order
    bc: str = "periodic"             # "periodic" | "dirichlet"
    bc_value: float = 0.0
    kappa_model: str = "const"       # "const" | "spitzer"
    kappa_par0: float = 1.0
    kappa_perp_ratio: float = 0.0
    saturate: bool = False
    phi: float = 0.3
    rho: float = 1.0
    sat_upwind: bool = False
    cp: float = 0.5
    limiter: str = "none"            # "none" (arithmetic mean, Eq. qT) | "mc" (Appendix C)
    limiter_floor: float = float("inf")
    _c: _Problem = field(default=None, repr=False)

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.shape))

    def cstruct(self) -> _Problem:
        p = _Problem()
        p.ndim = self.ndim
        nxyz = list(reversed(self.shape)) + [1] * (3 - self.ndim)
        dx = list(self.dx) if self.dx is not None else [1.0 / n for n in nxyz[: self.ndim]]
        dx = dx + [1.0] * (3 - len(dx))
        for d in range(3):
            p.n[d] = int(nxyz[d])
            p.dx[d] = float(dx[d])
        p.bc = {"periodic": 0, "dirichlet": 1}[self.bc]
        p.bc_value = float(self.bc_value)
        p.kappa_model = {"const": 0, "spitzer": 1}[self.kappa_model]
        p.kappa_par0 = float(self.kappa_par0)
        p.kappa_perp_ratio = float(self.kappa_perp_ratio)
        p.saturate = int(bool(self.saturate))
        p.phi = float(self.phi)
        p.rho = float(self.rho)
        p.sat_upwind = int(bool(self.sat_upwind))
        p.cp = float(self.cp)
        p.limiter = {"none": 0, "mc": 1}[self.limiter]
        p.limiter_floor = float(self.limiter_floor)
        return p


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _bfield(P: Problem, b) -> np.ndarray:
    """b as a [3][cells] FP64 array (missing components are zero)."""
    b = _f64(b).reshape(-1, P.ncell)
    out = np.zeros((3, P.ncell))
    out[: b.shape[0]] = b
    return out


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads the oracle uses."""
    return _load().orc_set_threads(int(n))


def face_flux(P: Problem, T, b, d: int, cell_xyz) -> float:
    """Flux component d on the face between cell (i,j,k) and its +e_d neighbour."""
    T = _f64(T)
    bb = _bfield(P, b)
    c = P.cstruct()
    i, j, k = (list(cell_xyz) + [0, 0])[:3]
    return _load().orc_face_flux(ctypes.byref(c), _ptr(T), _ptr(bb), d, i, j, k)


def flux(P: Problem, T, b):
    """Face fluxes F_d (one array per active axis, F_d[c] on face c + e_d/2)."""
    T = _f64(T)
    bb = _bfield(P, b)
    F = [np.zeros(P.shape) for _ in range(P.ndim)]
    ptrs = [_ptr(f) for f in F] + [None] * (3 - P.ndim)
    c = P.cstruct()
    _load().orc_flux(ctypes.byref(c), _ptr(T), _ptr(bb), *ptrs)
    return F


def apply_M(P: Problem, T, b) -> np.ndarray:
    """M(T) = -div F."""
    T = _f64(T)
    bb = _bfield(P, b)
    out = np.zeros(P.shape)
    c = P.cstruct()
    _load().orc_apply_M(ctypes.byref(c), _ptr(T), _ptr(bb), _ptr(out))
    return out


def dt_expl(P: Problem, T) -> float:
    T = _f64(T)
    c = P.cstruct()
    return _load().orc_dt_expl(ctypes.byref(c), _ptr(T))


def num_stages(ratio: float) -> int:
    return _load().orc_num_stages(float(ratio))


def coeffs(s: int):
    """(mu, nu, mu~, gamma~) as FP64 arrays of length s + 1 indexed by stage j."""
    arrs = [np.zeros(s + 1) for _ in range(4)]
    _load().orc_coeffs(int(s), *[_ptr(a) for a in arrs])
    return tuple(arrs)


def stage(P: Problem, j: int, s: int, dt: float, b, Y0, MY0, Yjm1, Yjm2):
    """One stage of Eq. rkl2scheme; returns (Y_j, MY0) (MY0 is written at j = 1)."""
    bb = _bfield(P, b)
    Y0 = _f64(Y0)
    MY0 = np.zeros(P.shape) if MY0 is None else _f64(MY0).copy()
    Yjm1 = Y0 if Yjm1 is None else _f64(Yjm1)
    Yjm2 = Y0 if Yjm2 is None else _f64(Yjm2)
    Yj = np.zeros(P.shape)
    c = P.cstruct()
    _load().orc_stage(ctypes.byref(c), int(j), int(s), float(dt), _ptr(bb), _ptr(Y0),
                      _ptr(MY0), _ptr(Yjm1), _ptr(Yjm2), _ptr(Yj))
    return Yj, MY0


def super_step(P: Problem, T, b, dt: float, s: int = 0, return_stage_min: bool = False):
    """One RKL2 super-step of length dt.  s = 0 picks s from dt / dt_expl(T)."""
    T = _f64(T).copy().reshape(P.shape)
    bb = _bfield(P, b)
    if s <= 0:
        s = num_stages(dt / dt_expl(P, T))
    mn = ctypes.c_double(0.0)
    c = P.cstruct()
    _load().orc_super_step(ctypes.byref(c), float(dt), int(s), _ptr(T), _ptr(bb),
                           ctypes.cast(ctypes.addressof(mn), ctypes.POINTER(ctypes.c_double)))
    if return_stage_min:
        return T, s, mn.value
    return T, s


def euler_step(P: Problem, T, b, dt: float) -> np.ndarray:
    T = _f64(T).copy().reshape(P.shape)
    bb = _bfield(P, b)
    c = P.cstruct()
    _load().orc_euler_step(ctypes.byref(c), float(dt), _ptr(T), _ptr(bb))
    return T


def energy(P: Problem, T) -> float:
    T = _f64(T)
    c = P.cstruct()
    return _load().orc_energy(ctypes.byref(c), _ptr(T))


def rkl2_scalar(s: int, z: float) -> float:
    """R_s(z): Eq. rkl2scheme applied to the scalar ODE dY/dt = lambda Y, z = tau lambda."""
    return _load().orc_rkl2_scalar(int(s), float(z))


# --- first-order super-time-steppers (Section 3.3) -------------------------

def num_stages_rkl1(ratio: float) -> int:
    """Eq. RKL-s for RKL1 (dt/dt_expl = (s^2 + s)/2), s -> 1 + floor(s)."""
    return _load().orc_num_stages_rkl1(float(ratio))


def rkl1_super_step(P: Problem, T, b, dt: float, s: int = 0):
    """One RKL1 super-step (Legendre recursion at 1 + w1 tau M, w1 = 2/(s^2+s))."""
    T = _f64(T).copy().reshape(P.shape)
    bb = _bfield(P, b)
    if s <= 0:
        s = num_stages_rkl1(dt / dt_expl(P, T))
    c = P.cstruct()
    _load().orc_rkl1_super_step(ctypes.byref(c), float(dt), int(s), _ptr(T), _ptr(bb))
    return T, s


def rkl1_scalar(s: int, z: float) -> float:
    """RKL1 amplification factor R_s(z) for dY/dt = lambda Y, z = tau lambda."""
    return _load().orc_rkl1_scalar(int(s), float(z))


def sts_gain(N: int, nu: float) -> float:
    """Eq. AAG-STS: super-step over explicit step for N sub-steps, damping nu."""
    return _load().orc_sts_gain(int(N), float(nu))


def num_stages_sts(ratio: float, nu: float) -> int:
    """Smallest N with sts_gain(N, nu) >= ratio."""
    return _load().orc_num_stages_sts(float(ratio), float(nu))


def sts_substeps(N: int, nu: float, dt: float) -> np.ndarray:
    """The N AAG-STS sub-steps of a super-step of length dt (they sum to dt)."""
    tau = np.zeros(N)
    _load().orc_sts_substeps(int(N), float(nu), float(dt), _ptr(tau))
    return tau


def sts_super_step(P: Problem, T, b, dt: float, nu: float = 1e-3, N: int = 0):
    """One AAG-STS super-step: N forward-Euler sub-steps summing to dt."""
    T = _f64(T).copy().reshape(P.shape)
    bb = _bfield(P, b)
    if N <= 0:
        N = num_stages_sts(dt / dt_expl(P, T), nu)
    c = P.cstruct()
    _load().orc_sts_super_step(ctypes.byref(c), float(dt), int(N), float(nu), _ptr(T), _ptr(bb))
    return T, N


# --- operator splitting (Section 3): passive advection, then conduction ----

def dt_hyp(P: Problem, u, ch: float = 0.8) -> float:
    """Eq. dt_h with lambda_d = |u_d|: C_h / max sum_d |u_d| / dx_d."""
    uu = _bfield(P, u)
    c = P.cstruct()
    return _load().orc_dt_hyp(ctypes.byref(c), _ptr(uu), float(ch))


def advect(P: Problem, T, u, dt: float) -> np.ndarray:
    """One conservative donor-cell step of dT/dt = -div(u T)."""
    T = _f64(T).reshape(P.shape)
    uu = _bfield(P, u)
    out = np.zeros(P.shape)
    c = P.cstruct()
    _load().orc_advect(ctypes.byref(c), float(dt), _ptr(T), _ptr(uu), _ptr(out))
    return out


def split_step(P: Problem, T, b, u, ch: float = 0.8, conduction: str = "rkl2", sub: int = 0):
    """One operator-split step of length dt_h: advection, then conduction over
    dt_h by one RKL2 super-step ("rkl2"), or by sub-cycled forward-Euler steps
    of at most dt_expl ("subcycle"; sub = their number, 0: ceil(dt_h/dt_expl)).
    Returns (T, dt_h, conduction stages)."""
    dth = dt_hyp(P, u, ch)
    T1 = advect(P, T, u, dth)
    if conduction == "rkl2":
        T2, s = super_step(P, T1, b, dth)
        return T2, dth, s
    n = sub if sub > 0 else int(np.ceil(dth / dt_expl(P, T1) - 1e-12))
    for _ in range(n):
        T1 = euler_step(P, T1, b, dth / n)
    return T1, dth, n
