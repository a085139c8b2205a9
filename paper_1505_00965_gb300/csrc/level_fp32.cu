// level_fp32.cu -- FP32-path level kernels (FP32 normals and paths, FP64 moment sums).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_kernel_fp32(int payoff, int mt, bool split, int scheme, bool long_lanes)
{
    return select_level_kernel<float>(payoff, mt, split, scheme, long_lanes);
}
const void *batch_kernel_fp32(int mt)
{
    return select_batch_kernel<float>(mt);
}
}  // namespace mlmcgb
