// cv_level.cu -- the control variate's level-estimator kernels (a translation unit of their own,
// compiled in parallel with the rest of the control-variate code): one instance per payoff for a
// run-time M^l, and one per payoff and level size for levels 0..2 at M = 4.
#include "cv_level_kernel.cuh"

namespace mlmcgb {

// M^l of the control-variate kernels compiled for one level size (M = 4, levels 0..2), else 0.
static int cv_level_nf(int level, int M)
{
    if (M != 4) return 0;
    return level == 0 ? 1 : level == 1 ? 4 : level == 2 ? 16 : 0;
}

template <int NF> static const void *cv_level_kernel_nf(int payoff)
{
    switch (payoff) {
    case kEuropean: return (const void *)cv_level_tc_kernel<kEuropean, NF>;
    case kAsian: return (const void *)cv_level_tc_kernel<kAsian, NF>;
    case kLookback: return (const void *)cv_level_tc_kernel<kLookback, NF>;
    case kDigital: return (const void *)cv_level_tc_kernel<kDigital, NF>;
    case kLinear: return (const void *)cv_level_tc_kernel<kLinear, NF>;
    case kGeoAsian: return (const void *)cv_level_tc_kernel<kGeoAsian, NF>;
    default: return nullptr;
    }
}

const void *cv_level_kernel_fp32(int payoff, int level, int M)
{
    switch (cv_level_nf(level, M)) {
    case 1: return cv_level_kernel_nf<1>(payoff);
    case 4: return cv_level_kernel_nf<4>(payoff);
    case 16: return cv_level_kernel_nf<16>(payoff);
    default: return cv_level_kernel_nf<0>(payoff);
    }
}

}  // namespace mlmcgb
