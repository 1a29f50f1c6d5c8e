// Generic RKL2 conduction kernels: one thread per cell, any dtype (float /
// double), 1-3 active axes, periodic or Dirichlet boundaries.  These serve
// the FP64 and low-dimensional configurations and every case the tiled FP32
// kernel does not cover; each cell evaluates the fluxes on all of its faces
// straight from global memory (L1/L2 absorb the neighbour re-reads).
#include "rkl_launch.h"

namespace rkl {
namespace {

template <typename R>
struct Field {
    const R* T;
    const R* b;
    KGrid<R> g;

    // T at a cell that may lie one cell outside the grid on active axes.
    __device__ __forceinline__ R t(int i, int j, int k) const
    {
        if (g.bc == 1) {
            if (i < 0 || i >= g.n[0] || j < 0 || j >= g.n[1] || k < 0 || k >= g.n[2]) return g.bcv;
        } else {
            i = wrap(i, g.n[0]);
            j = wrap(j, g.n[1]);
            k = wrap(k, g.n[2]);
        }
        return T[((int64_t)k * g.n[1] + j) * g.n[0] + i];
    }
    // Component e of b; ghosts copy the nearest interior cell (Dirichlet).
    __device__ __forceinline__ R bc(int e, int i, int j, int k) const
    {
        if (g.bc == 1) {
            i = clampi(i, g.n[0]);
            j = clampi(j, g.n[1]);
            k = clampi(k, g.n[2]);
        } else {
            i = wrap(i, g.n[0]);
            j = wrap(j, g.n[1]);
            k = wrap(k, g.n[2]);
        }
        return b[(int64_t)e * g.ncell + ((int64_t)k * g.n[1] + j) * g.n[0] + i];
    }
};

// Flux component d on the face between P = (i,j,k) and P + e_d.
template <typename R, int NDIM, bool SPITZER, bool SAT>
__device__ __forceinline__ R face(const Field<R>& f, const KPhys<R>& p, int d, int i, int j, int k)
{
    int P[3] = {i, j, k};
    int Q[3] = {i, j, k};
    Q[d] += 1;
    R TL = f.t(P[0], P[1], P[2]);
    R TR = f.t(Q[0], Q[1], Q[2]);
    R gn = (TR - TL) * f.g.inv_dx[d];
    R gt[2] = {R(0), R(0)};
    R bt[2] = {R(0), R(0)};
    // Appendix C: MC-limited transverse gradients where the face's lower
    // temperature is below the floor (an infinite floor limits everywhere)
    const bool limit = p.limiter && fmin(TL, TR) < p.lfloor;
    int m = 0;
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        if (e == d) continue;
        int Pp[3] = {P[0], P[1], P[2]}, Pm[3] = {P[0], P[1], P[2]};
        int Qp[3] = {Q[0], Q[1], Q[2]}, Qm[3] = {Q[0], Q[1], Q[2]};
        Pp[e] += 1; Qp[e] += 1; Pm[e] -= 1; Qm[e] -= 1;
        if (limit) {
            const R upL = f.t(Pp[0], Pp[1], Pp[2]) - TL, downL = TL - f.t(Pm[0], Pm[1], Pm[2]);
            const R upR = f.t(Qp[0], Qp[1], Qp[2]) - TR, downR = TR - f.t(Qm[0], Qm[1], Qm[2]);
            gt[m] = mc_limit(mc_limit(upL, downL), mc_limit(upR, downR)) * f.g.inv_dx[e];
        } else {
            gt[m] = (f.t(Pp[0], Pp[1], Pp[2]) + f.t(Qp[0], Qp[1], Qp[2])
                   - f.t(Pm[0], Pm[1], Pm[2]) - f.t(Qm[0], Qm[1], Qm[2])) * f.g.inv_4dx[e];
        }
        bt[m] = R(0.5) * (f.bc(e, P[0], P[1], P[2]) + f.bc(e, Q[0], Q[1], Q[2]));
        ++m;
    }
    R bn = R(0.5) * (f.bc(d, P[0], P[1], P[2]) + f.bc(d, Q[0], Q[1], Q[2]));
    return face_flux<R, SPITZER, SAT>(TL, TR, gn, gt[0], gt[1], bn, bt[0], bt[1], p);
}

template <typename R>
struct StageArgs {
    const R* Y0;
    R* MY0;
    const R* Yjm1;
    const R* Yjm2;
    R* Yj;
    const R* coef_tab;
    int j;
    int mode;
};

template <typename R, int NDIM, bool SPITZER, bool SAT>
__global__ void __launch_bounds__(256) stage_generic_kernel(KGrid<R> g, KPhys<R> p, StageArgs<R> a,
                                                            const R* __restrict__ b, KCoef<R> cf,
                                                            unsigned* status)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    int i = (int)(c % g.n[0]);
    int64_t r = c / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);

    // the field whose M is taken: Y0 for stage 1 / Euler, Yjm1 otherwise
    Field<R> f{a.mode == 2 || a.mode == 0 ? a.Yjm1 : a.Y0, b, g};
    R div = R(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        int lo[3] = {i, j, k};
        lo[d] -= 1;
        R Fhi = face<R, NDIM, SPITZER, SAT>(f, p, d, i, j, k);
        R Flo = face<R, NDIM, SPITZER, SAT>(f, p, d, lo[0], lo[1], lo[2]);
        div += (Fhi - Flo) * g.inv_dx[d];
    }
    R M = -div;
    if (a.mode == 0) {
        a.Yj[c] = M;
        return;
    }
    if (a.coef_tab) {
        const R* t = a.coef_tab + 4 * a.j;
        cf.mu = t[0]; cf.nu = t[1]; cf.mt = t[2]; cf.gt = t[3];
    }
    R y0 = a.Y0[c];
    R y;
    if (a.mode == 1) {
        if (a.MY0) a.MY0[c] = M;
        y = y0 + cf.mt * M;
    } else {
        R inc = cf.mu * (a.Yjm1[c] - y0) + cf.nu * (a.Yjm2[c] - y0) + cf.mt * M + cf.gt * a.MY0[c];
        y = y0 + inc;
    }
    check_value<R, SPITZER>(y, status);
    a.Yj[c] = y;
}

template <typename R, int NDIM, bool SPITZER, bool SAT>
__global__ void __launch_bounds__(256) flux_generic_kernel(KGrid<R> g, KPhys<R> p, const R* __restrict__ T,
                                                           const R* __restrict__ b, R* Fx, R* Fy, R* Fz)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    int i = (int)(c % g.n[0]);
    int64_t r = c / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    Field<R> f{T, b, g};
    R* F[3] = {Fx, Fy, Fz};
#pragma unroll
    for (int d = 0; d < NDIM; ++d) F[d][c] = face<R, NDIM, SPITZER, SAT>(f, p, d, i, j, k);
}

// Threads per block: 256, halved (down to one warp) while the grid would
// leave SMs idle -- small FP64 grids (the 100 x 100 ring) are bound by the
// per-SM FP64 rate, so they need every SM more than full blocks.
int generic_block(int64_t ncell)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
            nsm = 152;
    }
    int tpb = 256;
    while (tpb > 32 && (ncell + tpb - 1) / tpb < 2 * (int64_t)nsm) tpb /= 2;
    return tpb;
}

template <typename R, int NDIM, bool SPITZER, bool SAT>
cudaError_t stage_impl(const void* grid, const void* phys, const StageIO& io, const void* coef,
                       unsigned* status, cudaStream_t st)
{
    const KGrid<R>& g = *static_cast<const KGrid<R>*>(grid);
    const KPhys<R>& p = *static_cast<const KPhys<R>*>(phys);
    StageArgs<R> a{static_cast<const R*>(io.Y0), static_cast<R*>(io.MY0),
                   static_cast<const R*>(io.Yjm1), static_cast<const R*>(io.Yjm2),
                   static_cast<R*>(io.Yj), static_cast<const R*>(io.coef_tab), io.j, io.mode};
    KCoef<R> cf = coef ? *static_cast<const KCoef<R>*>(coef) : KCoef<R>{R(0), R(0), R(0), R(0)};
    const int tpb = generic_block(g.ncell);
    const int64_t blocks = (g.ncell + tpb - 1) / tpb;
    stage_generic_kernel<R, NDIM, SPITZER, SAT><<<(unsigned)blocks, tpb, 0, st>>>(
        g, p, a, static_cast<const R*>(io.b), cf, status);
    return cudaGetLastError();
}

template <typename R, int NDIM, bool SPITZER, bool SAT>
cudaError_t flux_impl(const void* grid, const void* phys, const void* T, const void* b, void* F[3],
                      cudaStream_t st)
{
    const KGrid<R>& g = *static_cast<const KGrid<R>*>(grid);
    const KPhys<R>& p = *static_cast<const KPhys<R>*>(phys);
    const int tpb = generic_block(g.ncell);
    const int64_t blocks = (g.ncell + tpb - 1) / tpb;
    flux_generic_kernel<R, NDIM, SPITZER, SAT><<<(unsigned)blocks, tpb, 0, st>>>(
        g, p, static_cast<const R*>(T), static_cast<const R*>(b), static_cast<R*>(F[0]),
        static_cast<R*>(F[1]), static_cast<R*>(F[2]));
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Operator splitting (Section 3): the hyperbolic step as the passive
// advection dT/dt = -div(u T) of the energy density by a cell-centred
// velocity u ([3][ncell], ghosts copy the nearest interior cell as b does),
// conservative donor cell: face velocity = mean of the two cells, face flux
// = u_f T(upwind cell).

template <typename R>
__device__ __forceinline__ R adv_flux(const Field<R>& f, int d, int i, int j, int k)
{
    int Q[3] = {i, j, k};
    Q[d] += 1;
    const R uf = R(0.5) * (f.bc(d, i, j, k) + f.bc(d, Q[0], Q[1], Q[2]));
    return uf * (uf >= R(0) ? f.t(i, j, k) : f.t(Q[0], Q[1], Q[2]));
}

template <typename R, int NDIM>
__global__ void __launch_bounds__(256) advect_kernel(KGrid<R> g, const R* __restrict__ T, const R* __restrict__ u,
                                                     R* __restrict__ Tout, R dt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int i = (int)(c % g.n[0]);
    const int64_t r = c / g.n[0];
    const int j = (int)(r % g.n[1]);
    const int k = (int)(r / g.n[1]);
    const Field<R> f{T, u, g};
    R div = R(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        int lo[3] = {i, j, k};
        lo[d] -= 1;
        div += (adv_flux(f, d, i, j, k) - adv_flux(f, d, lo[0], lo[1], lo[2])) * g.inv_dx[d];
    }
    Tout[c] = T[c] - dt * div;
}

// lambda(c) = sum_d |u_d| / dx_d (the denominator of Eq. dt_h)
template <typename R, int NDIM>
__global__ void __launch_bounds__(256) hyp_rate_kernel(KGrid<R> g, const R* __restrict__ u, R* __restrict__ lam)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    R v = R(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) v += fabs(u[(int64_t)d * g.ncell + c]) * g.inv_dx[d];
    lam[c] = v;
}

template <typename R>
cudaError_t advect_impl(const LaunchCfg& c, const void* grid, const void* T, const void* u, void* Tout, double dt,
                        cudaStream_t st)
{
    const KGrid<R>& g = *static_cast<const KGrid<R>*>(grid);
    const int tpb = generic_block(g.ncell);
    const unsigned blocks = (unsigned)((g.ncell + tpb - 1) / tpb);
    const R* Tp = static_cast<const R*>(T);
    const R* up = static_cast<const R*>(u);
    R* op = static_cast<R*>(Tout);
    if (c.ndim == 1) advect_kernel<R, 1><<<blocks, tpb, 0, st>>>(g, Tp, up, op, (R)dt);
    else if (c.ndim == 2) advect_kernel<R, 2><<<blocks, tpb, 0, st>>>(g, Tp, up, op, (R)dt);
    else advect_kernel<R, 3><<<blocks, tpb, 0, st>>>(g, Tp, up, op, (R)dt);
    return cudaGetLastError();
}

template <typename R>
cudaError_t hyp_rate_impl(const LaunchCfg& c, const void* grid, const void* u, void* lam, cudaStream_t st)
{
    const KGrid<R>& g = *static_cast<const KGrid<R>*>(grid);
    const unsigned blocks = (unsigned)((g.ncell + 255) / 256);
    const R* up = static_cast<const R*>(u);
    R* lp = static_cast<R*>(lam);
    if (c.ndim == 1) hyp_rate_kernel<R, 1><<<blocks, 256, 0, st>>>(g, up, lp);
    else if (c.ndim == 2) hyp_rate_kernel<R, 2><<<blocks, 256, 0, st>>>(g, up, lp);
    else hyp_rate_kernel<R, 3><<<blocks, 256, 0, st>>>(g, up, lp);
    return cudaGetLastError();
}

template <typename R, int NDIM>
cudaError_t stage_dispatch_phys(const LaunchCfg& c, const void* grid, const void* phys,
                                const StageIO& io, const void* coef, unsigned* status, cudaStream_t st)
{
    if (c.spitzer) {
        if (c.saturate) return stage_impl<R, NDIM, true, true>(grid, phys, io, coef, status, st);
        return stage_impl<R, NDIM, true, false>(grid, phys, io, coef, status, st);
    }
    if (c.saturate) return stage_impl<R, NDIM, false, true>(grid, phys, io, coef, status, st);
    return stage_impl<R, NDIM, false, false>(grid, phys, io, coef, status, st);
}

template <typename R>
cudaError_t stage_dispatch_ndim(const LaunchCfg& c, const void* grid, const void* phys,
                                const StageIO& io, const void* coef, unsigned* status, cudaStream_t st)
{
    switch (c.ndim) {
        case 1: return stage_dispatch_phys<R, 1>(c, grid, phys, io, coef, status, st);
        case 2: return stage_dispatch_phys<R, 2>(c, grid, phys, io, coef, status, st);
        case 3: return stage_dispatch_phys<R, 3>(c, grid, phys, io, coef, status, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R, int NDIM>
cudaError_t flux_dispatch_phys(const LaunchCfg& c, const void* grid, const void* phys, const void* T,
                               const void* b, void* F[3], cudaStream_t st)
{
    if (c.spitzer) {
        if (c.saturate) return flux_impl<R, NDIM, true, true>(grid, phys, T, b, F, st);
        return flux_impl<R, NDIM, true, false>(grid, phys, T, b, F, st);
    }
    if (c.saturate) return flux_impl<R, NDIM, false, true>(grid, phys, T, b, F, st);
    return flux_impl<R, NDIM, false, false>(grid, phys, T, b, F, st);
}

template <typename R>
cudaError_t flux_dispatch_ndim(const LaunchCfg& c, const void* grid, const void* phys, const void* T,
                               const void* b, void* F[3], cudaStream_t st)
{
    switch (c.ndim) {
        case 1: return flux_dispatch_phys<R, 1>(c, grid, phys, T, b, F, st);
        case 2: return flux_dispatch_phys<R, 2>(c, grid, phys, T, b, F, st);
        case 3: return flux_dispatch_phys<R, 3>(c, grid, phys, T, b, F, st);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// FP64 statistics (max, min, sum) in a fixed reduction order.

template <typename R>
__device__ __forceinline__ void acc(double v, double& mx, double& mn, double& sm)
{
    // NaN propagates into max and min so that callers can detect it
    mx = (v > mx || v != v) ? v : mx;
    mn = (v < mn || v != v) ? v : mn;
    sm += v;
}

// Max and min are exact in the data's own type; the sum (energy) is
// accumulated in FP64 and only when asked for (FP64 arithmetic is scarce on
// this GPU, and dt_expl needs only the extrema).  Each block leaves its
// partial {max, min, sum}; the block that finishes last (ticket counter at
// partials[3 * gridDim.x], reset by that block) folds all partials in a
// fixed order, so the result does not depend on which block is last.
__device__ __forceinline__ void fold_mm(double vmx, double vmn, double& mx, double& mn)
{
    mx = (vmx > mx || vmx != vmx) ? vmx : mx;
    mn = (vmn < mn || vmn != vmn) ? vmn : mn;
}

template <bool SUM>
__device__ __forceinline__ void block_fold(double& mx, double& mn, double& sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fold_mm(__shfl_xor_sync(0xffffffffu, mx, o), __shfl_xor_sync(0xffffffffu, mn, o), mx, mn);
        if (SUM) sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    __shared__ double s[3][8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { s[0][w] = mx; s[1][w] = mn; s[2][w] = sm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) {
            fold_mm(s[0][q], s[1][q], mx, mn);
            sm += s[2][q];
        }
    }
}

template <typename R, bool SUM>
__global__ void __launch_bounds__(256) stats_kernel(const R* __restrict__ T, int64_t n, double* partials,
                                                    double* out, unsigned* status)
{
    R mx = -INFINITY, mn = INFINITY;
    double sm = 0.0;
    auto fold = [&](R v) {
        mx = (v > mx || v != v) ? v : mx;
        mn = (v < mn || v != v) ? v : mn;
        if (SUM) sm += (double)v;
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sizeof(R) == 4 && (n & 3) == 0 && (reinterpret_cast<uintptr_t>(T) & 15) == 0) {
        const float4* T4 = reinterpret_cast<const float4*>(T);
        const int64_t n4 = n / 4;
        int64_t c = t0;
        // four independent 16-byte loads in flight per thread
        for (; c + 3 * stride < n4; c += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = T4[c + u * stride];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                fold((R)v[u].x); fold((R)v[u].y); fold((R)v[u].z); fold((R)v[u].w);
            }
        }
        for (; c < n4; c += stride) {
            const float4 v = T4[c];
            fold((R)v.x); fold((R)v.y); fold((R)v.z); fold((R)v.w);
        }
    } else {
        for (int64_t c = t0; c < n; c += stride) fold(T[c]);
    }
    double dmx = (double)mx, dmn = (double)mn;
    block_fold<SUM>(dmx, dmn, sm);
    __shared__ bool last;
    unsigned* ticket = reinterpret_cast<unsigned*>(partials + 3 * gridDim.x);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = dmx;
        partials[3 * blockIdx.x + 1] = dmn;
        partials[3 * blockIdx.x + 2] = sm;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    dmx = -INFINITY; dmn = INFINITY; sm = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
        fold_mm(__ldcg(&partials[3 * q]), __ldcg(&partials[3 * q + 1]), dmx, dmn);
        sm += __ldcg(&partials[3 * q + 2]);
    }
    block_fold<SUM>(dmx, dmn, sm);
    if (threadIdx.x == 0) {
        out[0] = dmx;
        out[1] = dmn;
        out[2] = sm;
        unsigned st = status ? *status : 0u;
        out[3] = (double)st;
        if (status) *status = 0u;
        *ticket = 0u;
    }
}

}  // namespace

cudaError_t launch_stage_generic(const LaunchCfg& c, const void* grid, const void* phys,
                                 const StageIO& io, const void* coef, unsigned* status, cudaStream_t st)
{
    if (c.dtype == 1) return stage_dispatch_ndim<double>(c, grid, phys, io, coef, status, st);
    return stage_dispatch_ndim<float>(c, grid, phys, io, coef, status, st);
}

cudaError_t launch_advect(const LaunchCfg& c, const void* grid, const void* T, const void* u, void* Tout, double dt,
                          cudaStream_t st)
{
    if (c.dtype == 1) return advect_impl<double>(c, grid, T, u, Tout, dt, st);
    return advect_impl<float>(c, grid, T, u, Tout, dt, st);
}

cudaError_t launch_hyp_rate(const LaunchCfg& c, const void* grid, const void* u, void* lam, cudaStream_t st)
{
    if (c.dtype == 1) return hyp_rate_impl<double>(c, grid, u, lam, st);
    return hyp_rate_impl<float>(c, grid, u, lam, st);
}

cudaError_t launch_flux_generic(const LaunchCfg& c, const void* grid, const void* phys, const void* T,
                                const void* b, void* F[3], cudaStream_t st)
{
    if (c.dtype == 1) return flux_dispatch_ndim<double>(c, grid, phys, T, b, F, st);
    return flux_dispatch_ndim<float>(c, grid, phys, T, b, F, st);
}

cudaError_t launch_stats(int dtype, const void* T, int64_t n, double* partials, double* out,
                         unsigned* status, cudaStream_t st, bool need_sum)
{
    const int nb = kStatsBlocks;
    if (dtype == 1) {
        const double* Td = static_cast<const double*>(T);
        if (need_sum) stats_kernel<double, true><<<nb, 256, 0, st>>>(Td, n, partials, out, status);
        else stats_kernel<double, false><<<nb, 256, 0, st>>>(Td, n, partials, out, status);
    } else {
        const float* Tf = static_cast<const float*>(T);
        if (need_sum) stats_kernel<float, true><<<nb, 256, 0, st>>>(Tf, n, partials, out, status);
        else stats_kernel<float, false><<<nb, 256, 0, st>>>(Tf, n, partials, out, status);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Segmented FP64 statistics of the problems of an ensemble: block c folds
// chunk c (cells [cstart[c], cstart[c] + clen[c]) of one problem), then one
// warp per problem folds that problem's chunks pchunk[p] .. pchunk[p+1]-1.

namespace {

__global__ void __launch_bounds__(256) seg_stats_kernel(const float* __restrict__ T, const int64_t* cstart,
                                                        const int* clen, double* partials)
{
    double mx = -INFINITY, mn = INFINITY, sm = 0.0;
    const int64_t s0 = cstart[blockIdx.x];
    const int len = clen[blockIdx.x];
    for (int i = threadIdx.x; i < len; i += blockDim.x) acc<float>((double)T[s0 + i], mx, mn, sm);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double omx = __shfl_xor_sync(0xffffffffu, mx, o);
        double omn = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = (omx > mx || omx != omx) ? omx : mx;
        mn = (omn < mn || omn != omn) ? omn : mn;
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    __shared__ double s[3][8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = mx; s[1][w] = mn; s[2][w] = sm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < 8; ++q) {
            mx = (s[0][q] > mx || s[0][q] != s[0][q]) ? s[0][q] : mx;
            mn = (s[1][q] < mn || s[1][q] != s[1][q]) ? s[1][q] : mn;
            sm += s[2][q];
        }
        partials[3 * blockIdx.x + 0] = mx;
        partials[3 * blockIdx.x + 1] = mn;
        partials[3 * blockIdx.x + 2] = sm;
    }
}

__global__ void seg_stats_final_kernel(const double* partials, const int* pchunk, int nprob, double* out)
{
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int l = threadIdx.x & 31;
    if (p >= nprob) return;
    double mx = -INFINITY, mn = INFINITY, sm = 0.0;
    for (int q = pchunk[p] + l; q < pchunk[p + 1]; q += 32) {
        double a = partials[3 * q], b = partials[3 * q + 1];
        mx = (a > mx || a != a) ? a : mx;
        mn = (b < mn || b != b) ? b : mn;
        sm += partials[3 * q + 2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double omx = __shfl_xor_sync(0xffffffffu, mx, o);
        double omn = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = (omx > mx || omx != omx) ? omx : mx;
        mn = (omn < mn || omn != omn) ? omn : mn;
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if (l == 0) {
        out[3 * p + 0] = mx;
        out[3 * p + 1] = mn;
        out[3 * p + 2] = sm;
    }
}

}  // namespace

cudaError_t launch_stats_segmented(const float* T, const int64_t* cstart, const int* clen, int nchunk,
                                   const int* pchunk, int nprob, double* partials, double* out, cudaStream_t st)
{
    seg_stats_kernel<<<nchunk, 256, 0, st>>>(T, cstart, clen, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seg_stats_final_kernel<<<(nprob + 7) / 8, 256, 0, st>>>(partials, pchunk, nprob, out);
    return cudaGetLastError();
}

}  // namespace rkl
