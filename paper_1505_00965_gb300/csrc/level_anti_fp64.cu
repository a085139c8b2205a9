// level_anti_fp64.cu -- antithetic level kernels, FP64 paths (a translation unit of their own so
// that they compile in parallel with the plain kernels).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_anti_kernel_fp64(int payoff, int mt, int scheme, bool long_lanes)
{
    return select_anti_kernel<double>(payoff, mt, scheme, long_lanes);
}
}  // namespace mlmcgb
