// ode.cu -- level kernel of the counterexample cited in Sec. 5 (Eq. count): the random ODE
// dX = -X^5 dt with a standard normal X(0), quantity E[X(T)^2].
//
// Explicit Euler--Maruyama (Sec. 2, Eq. em with g = 0) X <- X + h f(X), f(x) = -x^5, blows up on
// paths with large X(0) (|1 - h X^4| > 1 grows the next value), and multilevel Monte Carlo with it
// diverges; the tamed step X <- X + h f(X) / (1 + h |f(X)|) keeps every increment below 1 in size.
// The coupling of the two grids is the shared X(0): the fine path takes M^l steps of h, the coarse
// path M^(l-1) steps of M h, and Y = X_f(T)^2 - X_c(T)^2 (Y = X_f(T)^2 on level 0).
//
// Sample s draws X(0) as normal (s mod 4) of Philox block 0 of counter index floor(s / 4), so a
// thread takes one Philox block and its four samples; their four paths are independent chains
// that the loop below interleaves.  Overflowing explicit paths give inf or NaN as in any IEEE
// program; the driver stops on non-finite sums.
#include "level_kernel.cuh"
#include "mlmc.h"

namespace mlmcgb {

template <typename R, bool TAMED>
__device__ __forceinline__ R quintic_step(R x, R h)
{
    const R x2 = x * x;
    const R f = -(x2 * x2) * x;
    if constexpr (TAMED) return x + h * f / (R(1) + h * fabs(f));
    else return x + h * f;
}

// NS paths of n steps of h from x[0..NS), in lockstep.
template <typename R, bool TAMED, int NS>
__device__ __forceinline__ void quintic_paths(R x[NS], R h, int n)
{
    for (int k = 0; k < n; ++k) {
#pragma unroll
        for (int i = 0; i < NS; ++i) x[i] = quintic_step<R, TAMED>(x[i], h);
    }
}

template <typename R, bool TAMED>
__global__ void __launch_bounds__(256) quintic_level_kernel(const LevelParams p)
{
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f;
    int nb = 0;
    const uint64_t first = p.first, end = p.first + p.N;
    const uint64_t q0 = first / 4, nq = (end - 1) / 4 - q0 + 1;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, T = (uint64_t)gridDim.x * blockDim.x;
    const R h = R(p.h), H = R(p.h * p.M);
    const int nf = p.nf, nc = p.nf / p.M;
    const bool coupled = p.level > 0 && !p.fine_only;
    const bool u23 = p.u23 != 0;
    for (uint64_t u = t; u < nq; u += T) {
        const uint64_t q = q0 + u;
        const uint4 w = philox4x32_10(make_uint4(p.ctr3, 0u, (uint32_t)(q >> 32), (uint32_t)q), p.rkey);
        R rho, c, s, x0[4];
        BoxMuller<R>::pair(w.x, w.y, rho, c, s, u23);
        x0[0] = rho * c;
        x0[1] = rho * s;
        BoxMuller<R>::pair(w.z, w.w, rho, c, s, u23);
        x0[2] = rho * c;
        x0[3] = rho * s;
        R xf[4], xc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) xf[r] = xc[r] = x0[r];
        quintic_paths<R, TAMED, 4>(xf, h, nf);
        if (coupled) quintic_paths<R, TAMED, 4>(xc, H, nc);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t sample = q * 4 + r;
            if (sample < first || sample >= end) continue;
            R Y = xf[r] * xf[r];
            if (coupled) Y -= xc[r] * xc[r];
            if (p.y_out) p.y_out[sample - first] = (double)Y;
            add_moments(Y, m, b1, b2, b3, b4, nb);
        }
    }
    fold_batch<R>(m, b1, b2, b3, b4);
    finish_sums(m, p);
}

const void *ode_level_kernel(int precision, int scheme)
{
    const bool tamed = scheme == MLMC_TAMED_EM;
    if (scheme != MLMC_TAMED_EM && scheme != MLMC_EULER_MARUYAMA) return nullptr;
    if (precision == MLMC_FP32_PATH)
        return tamed ? (const void *)quintic_level_kernel<float, true> : (const void *)quintic_level_kernel<float, false>;
    return tamed ? (const void *)quintic_level_kernel<double, true> : (const void *)quintic_level_kernel<double, false>;
}

}  // namespace mlmcgb
