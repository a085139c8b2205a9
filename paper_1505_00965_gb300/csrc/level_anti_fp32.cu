// level_anti_fp32.cu -- antithetic level kernels, FP32 paths (a translation unit of their own so
// that they compile in parallel with the plain kernels).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_anti_kernel_fp32(int payoff, int mt, int scheme, bool long_lanes)
{
    return select_anti_kernel<float>(payoff, mt, scheme, long_lanes);
}
}  // namespace mlmcgb
