// Paired-cell stage kernel with MC-limited transverse gradients at every
// face (Appendix C with the limiter floor at +inf): the instantiations of
// the LIM build (five CTAs per SM), in a translation unit of their own so
// that they compile in parallel with the others.
#include "rkl_x2_tile.cuh"

namespace rkl {

cudaError_t launch_x2_lim(bool spitzer, bool saturate, int mode, const KGrid<float>& g, const KPhys<float>& p,
                          const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                          cudaStream_t st)
{
    if (saturate) {
        if (spitzer) return launch_mode<true, true, 4, false>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_mode<false, true, 4, false>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (spitzer) return launch_mode<true, false, 4, false>(mode, g, p, a, cf, status, nzchunk, st);
    return launch_mode<false, false, 4, false>(mode, g, p, a, cf, status, nzchunk, st);
}

}  // namespace rkl
