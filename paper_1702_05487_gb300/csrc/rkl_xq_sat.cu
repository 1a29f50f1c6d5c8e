// Saturated-flux builds of the row-pair stage kernel (rkl_xq.cuh), in a
// translation unit of their own so that they compile beside the others.
#include "rkl_xq.cuh"

namespace rkl {
namespace xq {

// kp0: kappa_perp = 0, the perpendicular terms left out at compile time
cudaError_t launch_q_sat(bool sp, bool kp0, int txw, int mode, const KGrid<float>& g, const KPhys<float>& p,
                         const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                         cudaStream_t st)
{
    if (sp) {
        if (kp0) {
            if (txw == 32) return launch_q_mode<true, true, 32, true>(mode, g, p, a, cf, status, nzchunk, st);
            return launch_q_mode<true, true, 64, true>(mode, g, p, a, cf, status, nzchunk, st);
        }
        if (txw == 32) return launch_q_mode<true, true, 32, false>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_q_mode<true, true, 64, false>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (kp0) {
        if (txw == 32) return launch_q_mode<false, true, 32, true>(mode, g, p, a, cf, status, nzchunk, st);
        return launch_q_mode<false, true, 64, true>(mode, g, p, a, cf, status, nzchunk, st);
    }
    if (txw == 32) return launch_q_mode<false, true, 32, false>(mode, g, p, a, cf, status, nzchunk, st);
    return launch_q_mode<false, true, 64, false>(mode, g, p, a, cf, status, nzchunk, st);
}

}  // namespace xq
}  // namespace rkl
