// Paired-cell FP32 3D stage kernel: the saturated-flux instantiations (a
// translation unit of their own so that they compile in parallel with
// rkl_x2.cu).
#include "rkl_x2_tile.cuh"

namespace rkl {

cudaError_t launch_x2_sat(bool spitzer, int occ, bool bulk, int mode, const KGrid<float>& g, const KPhys<float>& p,
                          const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                          cudaStream_t st, const x2::YMaps* ym, const x2::TMaps* tm)
{
    if (occ == 3) {
        if (spitzer) return launch_mode<true, true, 3, false>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_mode<false, true, 3, false>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (occ == 6) {
        if (spitzer) return launch_mode<true, true, 6, false>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_mode<false, true, 6, false>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (bulk) {
        if (spitzer) return launch_mode<true, true, 2, true>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_mode<false, true, 2, true>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (spitzer) return launch_mode<true, true, 2, false>(mode, g, p, a, cf, status, nzchunk, st, ym, tm);
    return launch_mode<false, true, 2, false>(mode, g, p, a, cf, status, nzchunk, st, ym, tm);
}

}  // namespace rkl
