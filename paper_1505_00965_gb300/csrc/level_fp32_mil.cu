// level_fp32_mil.cu -- Milstein level kernels, FP32 paths (a translation unit of their own so that
// they compile in parallel with the Euler--Maruyama kernels of level_fp32.cu).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_kernel_fp32_milstein(int payoff, int mt, bool split, bool long_lanes, bool positive)
{
    return select_scheme<float, true>(payoff, mt, split, long_lanes, positive);
}
}  // namespace mlmcgb
