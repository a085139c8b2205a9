// level_fp64_mil.cu -- Milstein level kernels, FP64 paths (a translation unit of their own so that
// they compile in parallel with the Euler--Maruyama kernels of level_fp64.cu).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_kernel_fp64_milstein(int payoff, int mt, bool split, bool long_lanes, bool positive)
{
    return select_scheme<double, true>(payoff, mt, split, long_lanes, positive);
}
}  // namespace mlmcgb
