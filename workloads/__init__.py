"""Seeded synthetic inputs for the RKL2 conduction workloads.

This module only makes input fields (temperature and unit magnetic field
arrays, problem parameters).  It holds none of the conduction method's
arithmetic, so both the FP64 oracle and the GPU library can be fed from it.

All arrays are C-ordered [z][y][x] (3D) or [y][x] (2D), cell-centred, FP64.
The field generators follow the workload recipes:

* ``ring``     - 2D ring diffusion on [-1,1]^2 with the azimuthal unit field
  b = (-y, x)/r and a hot sector (Section 4.1.3, with the sector, conductivity
  and boundary of the 100x100 Dirichlet workload).
* ``tangled``  - 3D periodic box [0,1)^3; b is the normalised curl of a random
  vector potential with Gaussian Fourier amplitudes, |A_k|^2 ~ k^(-17/3) on
  integer shells 2 <= |k| <= 8; T = 1 + 0.2 S with S a scalar field of the
  same spectrum scaled to max|S| = 1.
* ``blob``     - the tangled b with T = 1 + 9 exp(-r^2/0.01) about the centre
  (minimum-image distance).
* ``gaussian`` - the Gaussian profile exp(-x^2 / 2 sigma^2) of Section 4.1.1
  (1D, or a product in 2D/3D).
* ``ensemble_specs`` - the seeded list of uneven periodic problems of the
  batched workload.

The random Fourier modes are drawn once per seed from the shell alone, so
the same seed gives the same continuous field at every resolution.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.fft

KMIN, KMAX = 2, 8
SPECTRAL_SLOPE = -17.0 / 3.0     # |A_k|^2 ~ k^slope


def _shell_modes(seed: int, ncomp: int):
    """Integer wavevectors with KMIN <= |k| <= KMAX in the half space used by
    a real FFT (kz > 0, or kz == 0 and (ky > 0 or ky == 0 and kx > 0)), and
    complex Gaussian amplitudes with |A_k|^2 ~ |k|^slope for ncomp components."""
    ks = []
    for kz in range(0, KMAX + 1):
        for ky in range(-KMAX, KMAX + 1):
            for kx in range(-KMAX, KMAX + 1):
                if kz == 0 and (ky < 0 or (ky == 0 and kx <= 0)):
                    continue
                k2 = kx * kx + ky * ky + kz * kz
                if KMIN * KMIN <= k2 <= KMAX * KMAX:
                    ks.append((kx, ky, kz))
    ks = np.array(ks, dtype=np.int64)
    kmag = np.sqrt((ks ** 2).sum(1).astype(np.float64))
    rng = np.random.default_rng(seed)
    amp = kmag ** (SPECTRAL_SLOPE / 2.0)
    re = rng.standard_normal((ncomp, len(ks)))
    im = rng.standard_normal((ncomp, len(ks)))
    return ks, amp[None, :] * (re + 1j * im) / math.sqrt(2.0)


def _synth(nx: int, ny: int, nz: int, ks: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """Real field f(x) = sum_k 2 Re(coef_k exp(2 pi i k.x)) over half-space
    modes, evaluated at the cell centres ((i + 1/2)/nx, ...) of a periodic
    nx*ny*nz grid on the unit cube; returned as [z][y][x]."""
    # fold every mode onto the grid's own (aliased) frequencies
    kx = ks[:, 0] % nx
    ky = ks[:, 1] % ny
    kz = ks[:, 2] % nz
    fx = np.where(kx > nx // 2, kx - nx, kx)
    fy = np.where(ky > ny // 2, ky - ny, ky)
    fz = np.where(kz > nz // 2, kz - nz, kz)
    # cell-centre phase exp(i pi (kx/nx + ky/ny + kz/nz)) of the folded mode
    ph = np.exp(1j * math.pi * (fx / nx + fy / ny + fz / nz))
    c = coef * ph
    spec = np.zeros((nz, ny, nx), dtype=np.complex128)
    np.add.at(spec, (kz, ky, kx), c)
    np.add.at(spec, ((-ks[:, 2]) % nz, (-ks[:, 1]) % ny, (-ks[:, 0]) % nx), np.conj(c))
    return scipy.fft.ifftn(spec, workers=-1).real * (nx * ny * nz)


def tangled_b(n: int, seed: int = 2) -> np.ndarray:
    """Unit field b = curl A / |curl A| on an n^3 periodic grid, shape (3, n, n, n)."""
    ks, A = _shell_modes(seed, 3)
    kvec = ks.astype(np.float64) * 2.0 * math.pi
    # curl in Fourier space: B_k = i k x A_k
    B = 1j * np.cross(kvec, A.T).T                         # (3, nmodes)
    comps = [_synth(n, n, n, ks, B[c]) for c in range(3)]        # bx, by, bz with [z][y][x]
    b = np.stack(comps)
    mag = np.sqrt((b ** 2).sum(0))
    rms = math.sqrt(float((mag ** 2).mean()))
    b /= np.maximum(mag, 1e-12 * rms)[None]
    return b


def tangled_scalar(n: int, seed: int = 2) -> np.ndarray:
    """Scalar field of the same spectrum, scaled to max |S| = 1."""
    ks, S = _shell_modes(seed + 7919, 1)
    f = _synth(n, n, n, ks, S[0])
    return f / np.abs(f).max()


@dataclass
class Workload:
    name: str
    T: np.ndarray                  # initial temperature, FP64
    b: np.ndarray                  # unit field, (ndim, ...) FP64
    params: dict                   # grid / physics keyword arguments
    ratio: float                   # super-step dt / dt_expl(T at t = 0)
    n_super: int                   # super-steps in the run


def ring(n: int = 100) -> Workload:
    """2D ring: [-1,1]^2, b = (-y, x)/r, T = 12 in 0.5 < r < 0.7 with
    |atan2(y,x) - pi/12| < pi/12, else 10; Dirichlet T = 10; kappa_par = 0.01;
    super-step 50 dt_expl to t = 200."""
    dx = 2.0 / n
    c = -1.0 + (np.arange(n) + 0.5) * dx
    y, x = np.meshgrid(c, c, indexing="ij")
    r = np.sqrt(x * x + y * y)
    th = np.arctan2(y, x)
    T = np.where((r > 0.5) & (r < 0.7) & (np.abs(th - math.pi / 12) < math.pi / 12), 12.0, 10.0)
    b = np.stack([-y / r, x / r])
    params = dict(dx=(dx, dx), bc="dirichlet", bc_value=10.0, kappa_model="const",
                  kappa_par0=0.01, kappa_perp_ratio=0.0, saturate=False)
    dt_expl = 0.5 / (2 * 0.01 / dx ** 2)
    n_super = int(round(200.0 / (50 * dt_expl)))
    return Workload("ring2d", T, b, params, 50.0, n_super)


def tangled(n: int = 256, seed: int = 2) -> Workload:
    """3D tangled-field conduction: Spitzer kappa_par = 0.01 T^(5/2),
    kappa_perp = 1e-4 kappa_par, 10 super-steps at 100 dt_expl."""
    b = tangled_b(n, seed)
    T = 1.0 + 0.2 * tangled_scalar(n, seed)
    params = dict(dx=(1.0 / n,) * 3, bc="periodic", kappa_model="spitzer",
                  kappa_par0=0.01, kappa_perp_ratio=1e-4, saturate=False)
    return Workload(f"tangled{n}", T, b, params, 100.0, 10)


def blob(n: int = 512, seed: int = 2) -> Workload:
    """3D saturated conduction: tangled b, T = 1 + 9 exp(-r^2/0.01) about the
    box centre; Spitzer kappa_par, kappa_perp = 0, harmonic blend with
    q = 5 phi rho c^3, phi = 0.3, rho = 1; 20 super-steps at 200 dt_expl."""
    b = tangled_b(n, seed)
    c = (np.arange(n) + 0.5) / n - 0.5
    r2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    T = 1.0 + 9.0 * np.exp(-r2 / 0.01)
    params = dict(dx=(1.0 / n,) * 3, bc="periodic", kappa_model="spitzer",
                  kappa_par0=0.01, kappa_perp_ratio=0.0, saturate=True, phi=0.3, rho=1.0)
    return Workload(f"blob{n}", T, b, params, 200.0, 20)


def gaussian(n: int, ndim: int = 1, sigma: float = 0.1, L: float = 4.0):
    """Gaussian exp(-|x|^2 / 2 sigma^2) on [-L/2, L/2]^ndim at cell centres."""
    dx = L / n
    c = -L / 2 + (np.arange(n) + 0.5) * dx
    grids = np.meshgrid(*([c] * ndim), indexing="ij")
    r2 = sum(g * g for g in grids)
    return np.exp(-r2 / (2 * sigma * sigma)), dx, c


ENSEMBLE_SIZES = (32, 48, 64, 96, 128, 192)


def ensemble_specs(count: int = 64, seed: int = 4):
    """Seeded uneven periodic problems: per-axis sizes drawn from
    ENSEMBLE_SIZES, kappa_par0 uniform in [1e-3, 1e-1], dt/dt_expl uniform in
    [20, 400].  Cells are cubes of side h = 1 / max(nx, ny, nz) (the box is
    an nx*ny*nz brick of them).  Returns a list of dicts (nx, ny, nz, h,
    kappa_par0, ratio, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        nx, ny, nz = (int(v) for v in rng.choice(ENSEMBLE_SIZES, 3))
        out.append(dict(nx=nx, ny=ny, nz=nz, h=1.0 / max(nx, ny, nz),
                        kappa_par0=float(rng.uniform(1e-3, 1e-1)),
                        ratio=float(rng.uniform(20.0, 400.0)),
                        seed=int(1000 + p)))
    return out


def tangled_box(nx: int, ny: int, nz: int, seed: int):
    """Tangled b and T on an uneven nx*ny*nz periodic box (cells of unit
    aspect 1/nx, 1/ny, 1/nz on the unit cube), for the ensemble."""
    ks, A = _shell_modes(seed, 3)
    ksT, S = _shell_modes(seed + 7919, 1)
    kvec = ks.astype(np.float64) * 2.0 * math.pi
    B = 1j * np.cross(kvec, A.T).T
    b = np.stack([_synth(nx, ny, nz, ks, B[c]) for c in range(3)])
    mag = np.sqrt((b ** 2).sum(0))
    rms = math.sqrt(float((mag ** 2).mean()))
    b /= np.maximum(mag, 1e-12 * rms)[None]
    f = _synth(nx, ny, nz, ksT, S[0])
    T = 1.0 + 0.2 * f / np.abs(f).max()
    return T, b
