// level_fp32_ns2.cu -- FP32-path Euler--Maruyama level kernels with two samples per thread (a
// translation unit of their own, compiled in parallel with the one-sample kernels).
#include "level_kernel.cuh"

namespace mlmcgb {
const void *level_ns2_kernel_fp32(int payoff, int mt, bool long_lanes)
{
    return select_ns2_kernel<float>(payoff, mt, long_lanes);
}
}  // namespace mlmcgb
