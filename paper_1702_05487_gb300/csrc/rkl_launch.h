// Host-side launchers of the RKL2 kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rkl_device.cuh"

namespace rkl {

// Pointers of one stage launch.  mode: 0 -> out = M(in); 1 -> stage 1 /
// forward Euler (Yj = Y0 + mt M(Y0), MY0 written if non-null); 2 -> stage j.
struct StageIO {
    const void* Y0;
    void* MY0;
    const void* Yjm1;
    const void* Yjm2;
    void* Yj;
    const void* b;
    const void* coef_tab;   // if non-null: coefficients at coef_tab[4 j .. 4 j + 3]
    int j;
    int mode;
};

struct LaunchCfg {
    int dtype;              // 0 float, 1 double
    int ndim;
    int spitzer;
    int saturate;
    int limiter;            // MC-limited transverse gradients (generic, tiled and paired-cell kernels)
    int lim_all;            // the limiter at every face (floor +inf): the paired-cell kernel's only form
};

// Generic kernels: one thread per cell, any dtype / ndim / boundary.
cudaError_t launch_stage_generic(const LaunchCfg& c, const void* grid, const void* phys,
                                 const StageIO& io, const void* coef, unsigned* status,
                                 cudaStream_t st);
cudaError_t launch_flux_generic(const LaunchCfg& c, const void* grid, const void* phys,
                                const void* T, const void* b, void* F[3], cudaStream_t st);

// Operator splitting: one donor-cell advection step T_out = T - dt div(u T)
// (u: [3][ncell] cell-centred velocity), and the per-cell rate
// sum_d |u_d| / dx_d of Eq. dt_h into lam (grid-sized scratch).
cudaError_t launch_advect(const LaunchCfg& c, const void* grid, const void* T, const void* u, void* Tout, double dt,
                          cudaStream_t st);
cudaError_t launch_hyp_rate(const LaunchCfg& c, const void* grid, const void* u, void* lam, cudaStream_t st);

// Tiled FP32 3D stage kernel (shared-memory halo planes, z-march).
// Returns cudaErrorNotSupported if the configuration is not covered.
bool fast_stage_supported(const LaunchCfg& c, const KGrid<float>& g);
cudaError_t launch_stage_fast(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p,
                              const StageIO& io, const KCoef<float>& coef, unsigned* status,
                              cudaStream_t st);

// Paired-cell FP32 3D stage kernel (packed f32x2 arithmetic, 64 x 4 tiles,
// nzchunk planes per CTA, occupancy 2 or 3 CTAs per SM).  Needs nx % 4 == 0
// and 16-byte aligned arrays.
// With bulk (and a periodic grid with nx >= 72) the plane bundles are
// copied by the TMA engine (cp.async.bulk, one row per copy, mbarrier
// completion) instead of per-thread 16-byte cp.async.
// A limiter plan (floor +inf only) always takes the MC-limited build (five
// CTAs per SM, per-thread copies), whatever occupancy, bulk and ytma say.
bool x2_stage_supported(const LaunchCfg& c, const KGrid<float>& g);
bool x2_bulk_supported(const LaunchCfg& c, const KGrid<float>& g);
// With ytma the Y0 / Y_{j-2} / M(Y0) bundles of stages j >= 2 are copied by
// the TMA engine from tensor maps (cp.async.bulk.tensor, one thread, mbarrier
// completion) instead of per-thread 16-byte copies.
bool x2_ytma_supported(const LaunchCfg& c, const KGrid<float>& g);
// With tmaps every plane bundle is copied by the TMA engine from tensor maps
// (periodic, nx >= 72, ny >= 6, no limiter); the zero-filled periodic images
// at the grid's edges are patched by per-thread 16-byte chunks.
bool x2_tmaps_supported(const LaunchCfg& c, const KGrid<float>& g);
cudaError_t launch_stage_x2(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p, const StageIO& io,
                            const KCoef<float>& coef, unsigned* status, int nzchunk, int occupancy,
                            cudaStream_t st, bool bulk = false, bool ytma = false, bool tmaps = false);

// Row-pair FP32 3D stage kernel: the paired-cell kernel's arithmetic with
// two cell pairs per thread (rows 2w, 2w + 1 of 64 x 8 tiles, three CTAs per
// SM; txw = 32: 32 x 16 tiles, two row pairs per warp), writing the same
// bits.  Periodic grids, nx % 4 == 0, no limiter, fewer than 2^31 cells,
// 16-byte aligned arrays; nzchunk <= 0 picks the chunk length.
bool xq_stage_supported(const LaunchCfg& c, const KGrid<float>& g);
cudaError_t launch_stage_xq(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p, const StageIO& io,
                            const KCoef<float>& coef, unsigned* status, int nzchunk, cudaStream_t st,
                            int txw = 64);

// Two-stage paired-cell FP32 3D kernel: stages j (io, coefficients at
// io.coef_tab[4 j]) and j + 1 (written to Yj1) in one pass, 60 x 7 tiles of
// nzchunk planes.  Periodic grids with nx % 4 == 0 only.  Neither output may
// alias an input: the pass reads Y_{j-1}, Y_{j-2} and Y0 around its tile.
bool pair_stage_supported(const LaunchCfg& c, const KGrid<float>& g);
cudaError_t launch_stage_pair(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p, const StageIO& io,
                              void* Yj1, unsigned* status, int nzchunk, cudaStream_t st);

// FP64 statistics of a grid array: max, min and sum (fixed-order, deterministic).
// partials must hold 3 * kStatsBlocks + 1 doubles, the last one zero before
// the first call (a ticket counter the pass leaves at zero); out receives {max, min, sum}
// followed by the status word (as a double), which is then cleared.
constexpr int kStatsBlocks = 1216;   // 8 x 152 SMs
cudaError_t launch_stats(int dtype, const void* T, int64_t n, double* partials, double* out,
                         unsigned* status, cudaStream_t st, bool need_sum = true);

// FP64 {max, min, sum} per problem of an ensemble (FP32 data), from a chunk
// table: chunk c covers cells [cstart[c], cstart[c] + clen[c]); problem p
// owns chunks pchunk[p] .. pchunk[p+1]-1.  out receives 3 doubles per problem.
cudaError_t launch_stats_segmented(const float* T, const int64_t* cstart, const int* clen, int nchunk,
                                   const int* pchunk, int nprob, double* partials, double* out, cudaStream_t st);

}  // namespace rkl
