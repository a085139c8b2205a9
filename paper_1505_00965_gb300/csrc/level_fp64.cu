// level_fp64.cu -- FP64-path level kernels (FP64 normals, paths and moment sums).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_kernel_fp64(int payoff, int mt, bool split, int scheme, bool long_lanes)
{
    return select_level_kernel<double>(payoff, mt, split, scheme, long_lanes);
}
const void *batch_kernel_fp64(int mt)
{
    return select_batch_kernel<double>(mt);
}
}  // namespace mlmcgb
