// Paired-cell FP32 3D stage kernel: launches with the classical flux, the
// kernel choice and z-chunk of a launch, and the persistent ensemble kernel.
// The tile body and the kernel template are in rkl_x2_tile.cuh.
#include <algorithm>

#include <cudaTypedefs.h>

#include "rkl_x2_tile.cuh"

namespace rkl {

namespace {

template <int OCC, bool BULK>
cudaError_t launch_phys(const LaunchCfg& c, int mode, const KGrid<float>& g, const KPhys<float>& p,
                        const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk, cudaStream_t st,
                        const x2::YMaps* ym = nullptr, const x2::TMaps* tm = nullptr)
{
    if (c.saturate) return launch_x2_sat(c.spitzer, OCC, BULK, mode, g, p, a, cf, status, nzchunk, st, ym, tm);
    if (c.spitzer) return launch_mode<true, false, OCC, BULK>(mode, g, p, a, cf, status, nzchunk, st, ym, tm);
    return launch_mode<false, false, OCC, BULK>(mode, g, p, a, cf, status, nzchunk, st, ym, tm);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr if the driver does not offer it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// Tensor map of one grid-sized FP32 array: dims (nx, ny, nz), boxes of one
// tile's rows of one plane (TX x TY x 1); rows 16-byte multiples (nx % 4 == 0).
bool encode_ymap(CUtensorMap* m, const void* base, const KGrid<float>& g)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * 4u, (cuuint64_t)g.n[0] * (cuuint64_t)g.n[1] * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)x2::TX, (cuuint32_t)x2::TY, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of one grid-sized FP32 array with boxes of a tile's rows and
// their halo ring: SXS x (TY + 2) x 1 (columns from i0 - 4, rows from
// j0 - 1; cells outside the grid are filled with zeros).
bool encode_halo_map(CUtensorMap* m, const void* base, const KGrid<float>& g)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * 4u, (cuuint64_t)g.n[0] * (cuuint64_t)g.n[1] * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)x2::SXS, (cuuint32_t)x2::ROWS, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool x2_stage_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    return c.dtype == 0 && c.ndim == 3 && (!c.limiter || c.lim_all) && (g.n[0] % 4) == 0;
}

bool x2_bulk_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    return x2_stage_supported(c, g) && g.bc == 0 && g.n[0] >= x2::SXS;
}

bool x2_ytma_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    return x2_stage_supported(c, g) && tensor_map_encoder() != nullptr;
}
bool x2_tmaps_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    // boxes no larger than the grid: nx >= SXS (> TX) and ny >= TY + 2
    return x2_stage_supported(c, g) && !c.limiter && g.bc == 0 && g.n[0] >= x2::SXS && g.n[1] >= x2::ROWS &&
           tensor_map_encoder() != nullptr;
}

// Planes per CTA when none is given: the chunk length in [16, 48] that
// minimises (rounds of resident CTAs) x (planes + halo cost) per CTA, so that
// the last wave of CTAs is not left mostly empty, among the lengths that
// give at least 3.5 waves of CTAs where the grid has that many.  Measured
// on the 256^3 grid at five CTAs per SM: chunks of 20-24 planes (3.7-4.4
// waves) 113 us per stage, 28-37 planes (2.4-3.4 waves) 116 us.
static int auto_nzchunk(const KGrid<float>& g, int occupancy)
{
    const int64_t cols = (int64_t)((g.n[0] + x2::TX - 1) / x2::TX) * ((g.n[1] + x2::TY - 1) / x2::TY);
    const int64_t slots = (int64_t)ctas_per_sm(occupancy) * sm_count();
    const bool many = cols * ((g.n[2] + 15) / 16) * 2 >= 7 * slots;
    int best = 32;
    double cost = 1e300;
    for (int nzc = 16; nzc <= 48; ++nzc) {
        const int64_t chunks = (g.n[2] + nzc - 1) / nzc;
        if (many && cols * chunks * 2 < 7 * slots) continue;
        const int64_t rounds = (cols * chunks + slots - 1) / slots;
        const double c = (double)rounds * (std::min(nzc, g.n[2]) + 2.5);
        if (c < cost - 1e-9) {
            cost = c;
            best = nzc;
        }
    }
    return best;
}

x2::FastArgs x2_args(const StageIO& io)
{
    x2::FastArgs a;
    a.Tin = static_cast<const float*>(io.mode == 1 ? io.Y0 : io.Yjm1);
    a.b = static_cast<const float*>(io.b);
    a.Y0 = static_cast<const float*>(io.Y0);
    a.Yjm2 = static_cast<const float*>(io.Yjm2);
    a.MY0in = static_cast<const float*>(io.MY0);
    a.MY0out = io.mode == 1 ? static_cast<float*>(io.MY0) : nullptr;
    a.out = static_cast<float*>(io.Yj);
    a.coef_tab = static_cast<const float*>(io.coef_tab);
    a.j = io.j;
    return a;
}

cudaError_t launch_stage_x2(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p, const StageIO& io,
                            const KCoef<float>& coef, unsigned* status, int nzchunk, int occupancy, cudaStream_t st,
                            bool bulk, bool ytma, bool tmaps)
{
    const x2::FastArgs a = x2_args(io);
    if (c.limiter) {
        // the MC-limited build, whatever the variant asked for
        if (nzchunk == 0) nzchunk = auto_nzchunk(g, 4);
        else if (nzchunk < 0) nzchunk = 0;
        return launch_x2_lim(c.spitzer, c.saturate, io.mode, g, p, a, coef, status, nzchunk, st);
    }
    if (nzchunk == 0) nzchunk = auto_nzchunk(g, occupancy);
    else if (nzchunk < 0) nzchunk = 0;
    if (occupancy == 3) return launch_phys<3, false>(c, io.mode, g, p, a, coef, status, nzchunk, st);
    if (occupancy == 6) return launch_phys<6, false>(c, io.mode, g, p, a, coef, status, nzchunk, st);
    if (bulk && x2_bulk_supported(c, g)) return launch_phys<2, true>(c, io.mode, g, p, a, coef, status, nzchunk, st);
    if (tmaps && x2_tmaps_supported(c, g)) {
        x2::TMaps tm{};
        if (!encode_halo_map(&tm.m[0], a.Tin, g) || !encode_halo_map(&tm.m[1], a.b, g) ||
            !encode_halo_map(&tm.m[2], a.b + g.ncell, g) || !encode_halo_map(&tm.m[3], a.b + 2 * g.ncell, g))
            return cudaErrorInvalidValue;
        if (io.mode == 2 && (!encode_ymap(&tm.m[4], io.Y0, g) || !encode_ymap(&tm.m[5], io.Yjm2, g) ||
                             !encode_ymap(&tm.m[6], io.MY0, g)))
            return cudaErrorInvalidValue;
        return launch_phys<2, false>(c, io.mode, g, p, a, coef, status, nzchunk, st, nullptr, &tm);
    }
    if (ytma && io.mode == 2 && x2_ytma_supported(c, g)) {
        x2::YMaps ym;
        if (!encode_ymap(&ym.m[0], io.Y0, g) || !encode_ymap(&ym.m[1], io.Yjm2, g) ||
            !encode_ymap(&ym.m[2], io.MY0, g))
            return cudaErrorInvalidValue;
        return launch_phys<2, false>(c, io.mode, g, p, a, coef, status, nzchunk, st, &ym);
    }
    return launch_phys<2, false>(c, io.mode, g, p, a, coef, status, nzchunk, st);
}

// --------------------------------------------------------------------------
// Persistent ensemble kernel: one launch advances every problem of an
// ensemble by one super-step.  Work items (problem, stage, tile) are
// claimed in a fixed stage-major order from a global counter; before a tile
// of stage j of problem p runs, the CTA waits until all tiles of stage j-1
// of p are done (a per-problem counter).  Every item a CTA waits on was
// claimed earlier by a CTA that is already running and never waits on a
// later item, so the schedule cannot deadlock; each wait is still bounded
// and ends with ST_TIMEOUT and an abort flag that stops the other CTAs.

namespace {

template <bool SP, bool SAT>
__global__ void __launch_bounds__(x2::NTHREADS, x2::kCtasPerSm)
ensemble_x2_kernel(const x2::EnsProb* __restrict__ probs, const x2::EnsSeg* __restrict__ segs, int nseg,
                   int total, int* work, unsigned* done, unsigned* status, int* abort_flag, long long spin_limit)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    x2::Smem& sm = *reinterpret_cast<x2::Smem*>(smem_raw);                  // 64-column tiles
    x2::SmemT<x2::kPD, 32>& sm32 = *reinterpret_cast<x2::SmemT<x2::kPD, 32>*>(smem_raw);   // 32-column tiles
    __shared__ int s_go, s_p, s_j, s_tile;
    for (;;) {
        if (threadIdx.x == 0) {
            int p = 0, j = 0, tile = 0;
            s_go = x2::ens_claim(probs, segs, nseg, total, work, done, status, abort_flag, spin_limit, p, j, tile);
            s_p = p;
            s_j = j;
            s_tile = tile;
        }
        __syncthreads();
        if (!s_go) break;
        const x2::EnsProb& d = probs[s_p];
        const int j = s_j, tile = s_tile;
        const int bx = tile % d.tx, by = (tile / d.tx) % d.ty, bz = tile / (d.tx * d.ty);
        const bool narrow = d.txw == 32;
        const int i0 = bx * d.txw, j0 = by * (narrow ? x2::NTHREADS / 16 : x2::TY);
        const int z0 = bz * d.nzchunk;
        const int nzc = min(d.nzchunk, d.g.n[2] - z0);
        x2::FastArgs a;
        a.b = d.b;
        a.Y0 = d.T;
        a.coef_tab = d.coef;
        a.j = j;
        KCoef<float> cf{0.f, 0.f, 0.f, 0.f};
        if (j == 1) {
            a.Tin = d.T;
            a.Yjm2 = nullptr;
            a.MY0in = nullptr;
            a.MY0out = d.my0;
            a.out = d.buf[0];
            if (narrow)
                tile_x2<SP, SAT, 1, x2::kPD, false, false, false, false, 32>(sm32, d.g, d.p, a, cf, status, i0, j0,
                                                                            z0, nzc);
            else
                tile_x2<SP, SAT, 1, x2::kPD>(sm, d.g, d.p, a, cf, status, i0, j0, z0, nzc);
        } else {
            a.Tin = d.buf[(j - 2) % 3];
            a.Yjm2 = j == 2 ? d.T : d.buf[(j - 3) % 3];
            a.MY0in = d.my0;
            a.MY0out = nullptr;
            a.out = j == d.s ? d.T : d.buf[(j - 1) % 3];
            if (narrow)
                tile_x2<SP, SAT, 2, x2::kPD, false, false, false, false, 32>(sm32, d.g, d.p, a, cf, status, i0, j0,
                                                                            z0, nzc);
            else
                tile_x2<SP, SAT, 2, x2::kPD>(sm, d.g, d.p, a, cf, status, i0, j0, z0, nzc);
        }
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[s_p], 1u);
        }
    }
}

template <bool SP, bool SAT>
cudaError_t ensemble_launch_t(const x2::EnsProb* probs, const x2::EnsSeg* segs, int nseg, int total, int* work,
                              unsigned* done, unsigned* status, int* abort_flag, long long spin_limit, int grid,
                              cudaStream_t st)
{
    const int smem = (int)std::max(sizeof(x2::Smem), sizeof(x2::SmemT<x2::kPD, 32>));
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(ensemble_x2_kernel<SP, SAT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ensemble_x2_kernel<SP, SAT>,
                                                                      x2::NTHREADS, smem);
        if (e != cudaSuccess) return e;
        grid = sms * (per > 0 ? per : 1);
    }
    if (grid > total) grid = total > 0 ? total : 1;
    ensemble_x2_kernel<SP, SAT><<<grid, x2::NTHREADS, smem, st>>>(probs, segs, nseg, total, work, done, status,
                                                                   abort_flag, spin_limit);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ensemble_x2(bool spitzer, bool saturate, const x2::EnsProb* probs, const x2::EnsSeg* segs,
                               int nseg, int total, int* work, unsigned* done, unsigned* status, int* abort_flag,
                               long long spin_limit, int grid, cudaStream_t st)
{
    if (spitzer) {
        if (saturate)
            return ensemble_launch_t<true, true>(probs, segs, nseg, total, work, done, status, abort_flag, spin_limit,
                                                 grid, st);
        return ensemble_launch_t<true, false>(probs, segs, nseg, total, work, done, status, abort_flag, spin_limit,
                                              grid, st);
    }
    if (saturate)
        return ensemble_launch_t<false, true>(probs, segs, nseg, total, work, done, status, abort_flag, spin_limit,
                                              grid, st);
    return ensemble_launch_t<false, false>(probs, segs, nseg, total, work, done, status, abort_flag, spin_limit,
                                           grid, st);
}

}  // namespace rkl
