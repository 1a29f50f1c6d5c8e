// MC-limited builds of the row-pair stage kernel (rkl_xq.cuh; the limiter
// at every face, Appendix C with the limiter floor at +inf): each cell's
// transverse slopes are half its limited slopes MC(T+ - T0, T0 - T-) / 2 and
// a face takes MC of its two cells' slopes, as in the paired-cell kernel's
// limited build, whose bits these builds write.  64-column tiles.
#include "rkl_xq.cuh"

namespace rkl {
namespace xq {

cudaError_t launch_q_lim(bool sp, bool sat, int mode, const KGrid<float>& g, const KPhys<float>& p,
                         const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                         cudaStream_t st)
{
    if (sp) {
        if (sat) return launch_q_mode<true, true, 64, false, true>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_q_mode<true, false, 64, false, true>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (sat) return launch_q_mode<false, true, 64, false, true>(mode, g, p, a, cf, status, nzchunk, st);
    return launch_q_mode<false, false, 64, false, true>(mode, g, p, a, cf, status, nzchunk, st);
}

}  // namespace xq
}  // namespace rkl
