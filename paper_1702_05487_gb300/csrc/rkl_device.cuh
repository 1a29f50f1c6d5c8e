// Device-side building blocks shared by the RKL2 conduction kernels:
// kernel argument structs, boundary handling and the face-flux formula.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rkl {

// Status bits a kernel may raise in the plan's device status word.
enum : unsigned { ST_NONFINITE = 1u, ST_NONPOSITIVE = 2u, ST_TIMEOUT = 4u };

// Grid geometry as the kernels see it.
template <typename R>
struct KGrid {
    int n[3];            // cells along x, y, z (1 on inactive axes)
    int ndim;
    int bc;              // 0 periodic, 1 Dirichlet
    R bcv;               // Dirichlet ghost temperature
    R inv_dx[3];         // 1/dx_d  (normal gradient and divergence)
    R inv_4dx[3];        // 1/(4 dx_d)  (transverse gradient, Eq. qT)
    int64_t plane;       // n[0] * n[1]
    int64_t ncell;
};

// Conduction physics as the kernels see it (rho = 1, gamma = 2).
template <typename R>
struct KPhys {
    R kappa0;            // kappa_par0
    R kperp;             // kappa_perp / kappa_par
    R q0;                // 5 phi rho: q = q0 * c_iso^3 (Eq. Fsat)
    int upwind;          // c_iso from the donor cell of the normal flux
    int limiter;         // MC-limited transverse gradients (generic kernel)
    R lfloor;            // ... at faces with min(T_L, T_R) below this
};

// Per-stage recurrence coefficients in the kernel's type.  The update is
// evaluated about Y0 (mu + nu + c0 = 1 exactly):
//   Yj = Y0 + mu (Yjm1 - Y0) + nu (Yjm2 - Y0) + mt M(Yjm1) + gt MY0
// with mt = mut_j tau and gt = gt_j tau, which keeps the rounding of mu and
// nu from acting on the (large) base value.
template <typename R>
struct KCoef {
    R mu, nu, mt, gt;
};

// Square root and quotient of the flux formula.  FP64 uses the correctly
// rounded operations; FP32 uses the hardware approximations of the PTX ISA
// (sqrt.approx.f32 and div.full.f32, a few ulp), which keeps the stencil's
// instruction count down and stays far inside the FP32 tolerance.
template <typename R>
__device__ __forceinline__ R dsqrt(R x);
template <>
__device__ __forceinline__ float dsqrt<float>(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

template <typename R>
__device__ __forceinline__ R ddiv(R a, R b);
template <>
__device__ __forceinline__ float ddiv<float>(float a, float b) { return __fdividef(a, b); }
template <>
__device__ __forceinline__ double ddiv<double>(double a, double b) { return a / b; }

// Parallel conductivity at temperature T.
template <typename R, bool SPITZER>
__device__ __forceinline__ R kappa_par(R T, const KPhys<R>& p)
{
    if (SPITZER) return p.kappa0 * (T * T) * dsqrt<R>(T);
    return p.kappa0;
}

// Normal component of the conduction flux on one face.
//   TL, TR   : cell temperatures on the low / high side of the face
//   gn       : normal gradient (TR - TL)/dx_d              (Eq. qN)
//   g1, g2   : transverse gradients averaged to the face   (Eq. qT)
//   bn,b1,b2 : face b (mean of the two cells), normal / transverse parts
// Classical flux F = -kappa_par b (b . grad T) - kappa_perp grad T
// (Eqs. Fclass, Fclass_HD); with SAT the harmonic blend q/(q + |F|) F
// (Eqs. Fc, Fsat) with q = 5 phi rho c_iso^3.
template <typename R, bool SPITZER, bool SAT>
__device__ __forceinline__ R face_flux(R TL, R TR, R gn, R g1, R g2,
                                       R bn, R b1, R b2, const KPhys<R>& p)
{
    const R half = R(0.5);
    R Tf = half * (TL + TR);
    R kpar = kappa_par<R, SPITZER>(Tf, p);
    R kperp = p.kperp * kpar;
    R bdg = bn * gn + b1 * g1 + b2 * g2;
    R Fn = -kpar * bn * bdg - kperp * gn;
    if (SAT) {
        R F1 = -kpar * b1 * bdg - kperp * g1;
        R F2 = -kpar * b2 * bdg - kperp * g2;
        R Fmag = dsqrt<R>(Fn * Fn + F1 * F1 + F2 * F2);
        R Tq = p.upwind ? (Fn >= R(0) ? TL : TR) : Tf;
        R q = p.q0 * Tq * dsqrt<R>(Tq);
        Fn = ddiv<R>(q, q + Fmag) * Fn;
    }
    return Fn;
}

// Monotonised-central limiter: 0 if a and b differ in sign, else the one of
// 2a, 2b, (a + b)/2 smallest in magnitude.
template <typename R>
__device__ __forceinline__ R mc_limit(R a, R b)
{
    if (a * b <= R(0)) return R(0);
    R m = fabs(R(0.5) * (a + b));
    m = fmin(m, R(2) * fabs(a));
    m = fmin(m, R(2) * fabs(b));
    return a > R(0) ? m : -m;
}
// FP32: the same value without branches (2 min(|a|, |b|) = min(2|a|, 2|b|)
// exactly; the sign of a when a b > 0).
template <>
__device__ __forceinline__ float mc_limit<float>(float a, float b)
{
    const float m = fminf(0.5f * fabsf(a + b), 2.f * fminf(fabsf(a), fabsf(b)));
    return a * b > 0.f ? copysignf(m, a) : 0.f;
}

// Wrap or clamp an index that is at most a few cells outside [0, n).
__device__ __forceinline__ int wrap(int i, int n)
{
    i = (i < 0) ? i + n : i;
    return (i >= n) ? i - n : i;
}
__device__ __forceinline__ int clampi(int i, int n)
{
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Record a bad stage value in the device status word.
template <typename R, bool SPITZER>
__device__ __forceinline__ void check_value(R y, unsigned* status)
{
    bool bad_nf = !(y == y) || (y - y != R(0));      // NaN or +-Inf
    bool bad_np = SPITZER && !(y > R(0));
    if (bad_nf || bad_np) {
        atomicOr(status, (bad_nf ? ST_NONFINITE : 0u) | (bad_np ? ST_NONPOSITIVE : 0u));
    }
}

}  // namespace rkl
