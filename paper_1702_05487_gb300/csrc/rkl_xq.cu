// Row-pair FP32 3D stage kernel (the tile body and kernel template are in
// rkl_xq.cuh): launches with the classical flux, the choice of build, the
// z-chunk of a launch, and the persistent ensemble kernel on the row-pair
// tile body.
#include "rkl_xq.cuh"

namespace rkl {
namespace xq {

// Persistent ensemble kernel on the row-pair tile body: the work list,
// dependency waits and completion counters of the paired-cell ensemble
// kernel (x2::ens_claim), each item a 64 x 8 tile (or 32 x 16 where the
// problem's txw is 32) of one stage of one problem.
template <bool SP, bool SAT>
__global__ void __launch_bounds__(NTHREADS, kCtasPerSm)
ensemble_q_kernel(const x2::EnsProb* __restrict__ probs, const x2::EnsSeg* __restrict__ segs, int nseg, int total,
                  int* work, unsigned* done, unsigned* status, int* abort_flag, long long spin_limit)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemQ<64>& sm = *reinterpret_cast<SmemQ<64>*>(smem_raw);
    SmemQ<32>& sm32 = *reinterpret_cast<SmemQ<32>*>(smem_raw);
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
        const int i0 = bx * d.txw, j0 = by * (narrow ? SmemQ<32>::TY : SmemQ<64>::TY);
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
            if (narrow) tile_q<SP, SAT, 1, 32>(sm32, d.g, d.p, a, cf, status, i0, j0, z0, nzc);
            else tile_q<SP, SAT, 1, 64>(sm, d.g, d.p, a, cf, status, i0, j0, z0, nzc);
        } else {
            a.Tin = d.buf[(j - 2) % 3];
            a.Yjm2 = j == 2 ? d.T : d.buf[(j - 3) % 3];
            a.MY0in = d.my0;
            a.MY0out = nullptr;
            a.out = j == d.s ? d.T : d.buf[(j - 1) % 3];
            if (narrow) tile_q<SP, SAT, 2, 32>(sm32, d.g, d.p, a, cf, status, i0, j0, z0, nzc);
            else tile_q<SP, SAT, 2, 64>(sm, d.g, d.p, a, cf, status, i0, j0, z0, nzc);
        }
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[s_p], 1u);
        }
    }
}

template <bool SP, bool SAT>
cudaError_t ensemble_launch_q(const x2::EnsProb* probs, const x2::EnsSeg* segs, int nseg, int total, int* work,
                              unsigned* done, unsigned* status, int* abort_flag, long long spin_limit, int grid,
                              cudaStream_t st)
{
    const int smem = (int)std::max(sizeof(SmemQ<64>), sizeof(SmemQ<32>));
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(ensemble_q_kernel<SP, SAT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (grid <= 0) {
        int per = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ensemble_q_kernel<SP, SAT>, NTHREADS, smem);
        if (e != cudaSuccess) return e;
        grid = sm_count() * (per > 0 ? per : 1);
    }
    if (grid > total) grid = total > 0 ? total : 1;
    ensemble_q_kernel<SP, SAT><<<grid, NTHREADS, smem, st>>>(probs, segs, nseg, total, work, done, status, abort_flag,
                                                             spin_limit);
    return cudaGetLastError();
}

// Planes per CTA: among 16 .. 64, the length that minimises (rounds of
// resident CTAs) x (planes + halo cost), keeping at least 3.5 waves of CTAs
// where the grid has that many (the paired-cell kernel's rule with this
// kernel's tile and occupancy).
int auto_nzchunk_q(const KGrid<float>& g, int tx, int ty)
{
    const int64_t cols = (int64_t)((g.n[0] + tx - 1) / tx) * ((g.n[1] + ty - 1) / ty);
    const int64_t slots = (int64_t)kCtasPerSm * sm_count();
    const bool many = cols * ((g.n[2] + 15) / 16) * 2 >= 7 * slots;
    int best = 32;
    double cost = 1e300;
    for (int nzc = 16; nzc <= 64; ++nzc) {
        const int64_t chunks = (g.n[2] + nzc - 1) / nzc;
        if (many && cols * chunks * 2 < 7 * slots) continue;
        const int64_t rounds = (cols * chunks + slots - 1) / slots;
        const double cst = (double)rounds * (std::min(nzc, g.n[2]) + 2.5);
        if (cst < cost - 1e-9) {
            cost = cst;
            best = nzc;
        }
    }
    return best;
}

}  // namespace xq

x2::FastArgs x2_args(const StageIO& io);      // rkl_x2.cu

bool xq_stage_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    return c.dtype == 0 && c.ndim == 3 && (!c.limiter || c.lim_all) && g.bc == 0 && (g.n[0] % 4) == 0 &&
           g.ncell < ((int64_t)1 << 31);
}

cudaError_t launch_stage_xq(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p, const StageIO& io,
                            const KCoef<float>& coef, unsigned* status, int nzchunk, cudaStream_t st, int txw)
{
    if (!xq_stage_supported(c, g) || (txw != 64 && txw != 32)) return cudaErrorNotSupported;
    const x2::FastArgs a = x2_args(io);
    // the limited build comes with 64-column tiles only
    if (c.limiter) txw = 64;
    if (nzchunk <= 0) nzchunk = xq::auto_nzchunk_q(g, txw, txw == 64 ? xq::SmemQ<64>::TY : xq::SmemQ<32>::TY);
    if (c.limiter) return xq::launch_q_lim(c.spitzer != 0, c.saturate != 0, io.mode, g, p, a, coef, status, nzchunk, st);
    if (c.saturate)
        return xq::launch_q_sat(c.spitzer != 0, p.kperp == 0.f, txw, io.mode, g, p, a, coef, status, nzchunk, st);
    if (c.spitzer) {
        if (txw == 32) return xq::launch_q_mode<true, false, 32, false>(io.mode, g, p, a, coef, status, nzchunk, st);
        return xq::launch_q_mode<true, false, 64, false>(io.mode, g, p, a, coef, status, nzchunk, st);
    }
    if (txw == 32) return xq::launch_q_mode<false, false, 32, false>(io.mode, g, p, a, coef, status, nzchunk, st);
    return xq::launch_q_mode<false, false, 64, false>(io.mode, g, p, a, coef, status, nzchunk, st);
}

cudaError_t launch_ensemble_xq(bool spitzer, bool saturate, const x2::EnsProb* probs, const x2::EnsSeg* segs,
                               int nseg, int total, int* work, unsigned* done, unsigned* status, int* abort_flag,
                               long long spin_limit, int grid, cudaStream_t st)
{
    if (spitzer) {
        if (saturate)
            return xq::ensemble_launch_q<true, true>(probs, segs, nseg, total, work, done, status, abort_flag,
                                                     spin_limit, grid, st);
        return xq::ensemble_launch_q<true, false>(probs, segs, nseg, total, work, done, status, abort_flag,
                                                  spin_limit, grid, st);
    }
    if (saturate)
        return xq::ensemble_launch_q<false, true>(probs, segs, nseg, total, work, done, status, abort_flag,
                                                  spin_limit, grid, st);
    return xq::ensemble_launch_q<false, false>(probs, segs, nseg, total, work, done, status, abort_flag, spin_limit,
                                               grid, st);
}

}  // namespace rkl
