// level_fp32.cu -- FP32-path level kernels (FP32 normals and paths, FP64 moment sums).
#include "level_kernel.cuh"
#include "mlmc.h"

namespace mlmcgb {
// Euler--Maruyama kernels here; the Milstein ones in level_fp32_mil.cu (a translation unit of
// their own, compiled in parallel).
const void *level_kernel_fp32(int payoff, int mt, bool split, int scheme, bool long_lanes, bool positive)
{
    if (scheme == MLMC_MILSTEIN) return level_kernel_fp32_milstein(payoff, mt, split, long_lanes, positive);
    return select_scheme<float, false>(payoff, mt, split, long_lanes, positive);
}
const void *batch_kernel_fp32(int mt)
{
    return select_batch_kernel<float>(mt);
}
}  // namespace mlmcgb
