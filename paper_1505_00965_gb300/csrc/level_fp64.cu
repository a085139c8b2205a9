// level_fp64.cu -- FP64-path level kernels (FP64 normals, paths and moment sums).
#include "level_kernel.cuh"
#include "mlmc.h"

namespace mlmcgb {
// Euler--Maruyama kernels here; the Milstein ones in level_fp64_mil.cu (a translation unit of
// their own, compiled in parallel).
const void *level_kernel_fp64(int payoff, int mt, bool split, int scheme, bool long_lanes, bool positive)
{
    if (scheme == MLMC_MILSTEIN) return level_kernel_fp64_milstein(payoff, mt, split, long_lanes, positive);
    return select_scheme<double, false>(payoff, mt, split, long_lanes, positive);
}
const void *batch_kernel_fp64(int mt)
{
    return select_batch_kernel<double>(mt);
}
}  // namespace mlmcgb
