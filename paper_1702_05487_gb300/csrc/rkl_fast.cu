// Tiled FP32 3D stage kernel (placeholder until the tiled kernel lands).
#include "rkl_launch.h"

namespace rkl {

bool fast_stage_supported(const LaunchCfg&, const KGrid<float>&) { return false; }

cudaError_t launch_stage_fast(const LaunchCfg&, const KGrid<float>&, const KPhys<float>&, const StageIO&,
                              const KCoef<float>&, unsigned*, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace rkl
