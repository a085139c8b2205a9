// cv_level_kernel.cuh -- the learned control variate's samples and level estimator (FP32 paths).
//
// For a level-l sample the control variate needs Y = P_l - P_{l-1} (Sec. 5, Eq. Yldef) and the
// network inputs: the Brownian-bridge (Levy) coordinates of the path on the T/16 grid,
// x_0 = W(T) / sqrt(T), then stage by stage (intervals of 16, 8, 4, 2 grid steps) and left to
// right the standardised midpoint deviations (W(m) - (W(l) + W(r)) / 2) / sqrt((r - l) / 4).
// On levels with M^l >= 16 the grid values are running sums of the path's fine increments; on
// coarser levels the grid is refined from the path's own grid by Brownian-bridge midpoints whose
// normals come from the Philox blocks of the sample's counter after the path's own (from block
// max(1, M^l / 4) on; stage by stage, left to right), so the path itself is the one the plain
// estimator draws.
#pragma once
#include <cstdint>

#include "engine.h"
#include "level_kernel.cuh"
#include "mlmc.h"
#include "mlp.cuh"
#include "tc_mlp.cuh"
#include "rng.cuh"

namespace mlmcgb {

// The FP32 constants of a level's paths and payoff, converted once from the FP64 parameters (a
// conversion from FP64 runs on the FP64 pipe, 2 per SM per clock on GB300; kernels keep these in
// shared memory so the compiler reloads them instead of converting again in every sample).
// inv_tg = 1 / sqrt_tg is the FP32 quotient of the converted value (sqrt_tg = sqrt(T / 16), the
// scale of a grid increment).
struct CvConsts {
    float a, rh, S0, sqrt_h, sqrt_tg, inv_nf, inv_nc, K, disc, Q, inv_tg;
};
__device__ __forceinline__ CvConsts cv_consts(const LevelParams &p)
{
    const float sqrt_tg = (float)p.sqrt_tg;
    return {(float)p.a, (float)p.rh, (float)p.S0, (float)p.sqrt_h, sqrt_tg, (float)p.inv_nf, (float)p.inv_nc,
            (float)p.K, (float)p.disc, (float)p.Q, 1.0f / sqrt_tg};
}

// The Levy coordinates of grid[i] = W(i T / 16), i = 0..16 (grid[0] = 0); inv_tg = 1 / sqrt(T / 16).
// The midpoint of an interval of w grid steps has bridge standard deviation sqrt(T / 16) sqrt(w) / 2.
__device__ __forceinline__ void levy_coordinates(const float grid[17], float inv_tg, float x[kInputs])
{
    static_assert(kInputs == 16, "the coordinates of a 16-step grid");
    x[0] = 0.25f * inv_tg * grid[16];
    int idx = 1;
#pragma unroll
    for (int w = 16; w > 1; w /= 2) {
        const float s = inv_tg * (w == 16 ? 0.5f : w == 8 ? 0.70710678118654752f : w == 4 ? 1.0f : 1.41421356237309505f);
#pragma unroll
        for (int left = 0; left < 16; left += w) x[idx++] = (grid[left + w / 2] - 0.5f * (grid[left] + grid[left + w])) * s;
    }
}

// The Philox blocks use the round keys of the kernel's parameters (constant-bank operands).  NF,
// when nonzero, is M^l known at compile time with M = 4 (levels 0, 1, 2): the loops then unroll
// and the grid stays in registers (with a run-time M^l it is indexed at run time, in local memory).
__device__ __forceinline__ float pick4(const float z[4], uint32_t i)
{
    return i == 0 ? z[0] : i == 1 ? z[1] : i == 2 ? z[2] : z[3];
}
template <int PAY, int NF = 0>
__device__ __forceinline__ void cv_sample(const LevelParams &p, const CvConsts &k, uint64_t s, float &Y,
                                          float x[kInputs])
{
    static_assert(NF == 0 || NF == 1 || NF == 4 || NF == 16, "compile-time sizes of levels 0..2 at M = 4");
    const int nf = NF ? NF : p.nf, M = NF ? 4 : p.M;
    const bool level0 = NF ? NF == 1 : p.level == 0;
    const float a = k.a, rh = k.rh, S0 = k.S0;
    const float sqrt_h = k.sqrt_h, sqrt_tg = k.sqrt_tg;
    float fS = 1.f, fsum = 0.f, fhi = 1.f, flo = 1.f, fls = 0.f;
    float cS = 1.f, csum = 0.f, chi = 1.f, clo = 1.f, cls = 0.f;
    float dc = 0.f;
    int q = 0;
    float grid[17];  // W at i T / 16
    auto fine_step = [&](float z) {
        const float d = fmaf(a, z, rh);
        em_step<float, PAY, false>(fS, fsum, fhi, flo, fls, d);
        dc += d;
        if (++q == M) {
            em_step<float, PAY, false>(cS, csum, chi, clo, cls, dc);
            dc = 0.f;
            q = 0;
        }
    };
    if (nf < 4) {
        // 4 / nf samples share block 0 of counter index s / G (the packed small levels)
        const uint32_t G = 4u / (uint32_t)(nf < 4 ? nf : 4);
        const uint64_t qb = s / G;
        const uint32_t slot = (uint32_t)(s % G);
        const uint4 xb = philox4x32_10(make_uint4(p.ctr3, 0u, (uint32_t)(qb >> 32), (uint32_t)qb), p.rkey);
        float rho, c, sn, z[4];
        BoxMuller<float>::pair(xb.x, xb.y, rho, c, sn);
        z[0] = rho * c;
        z[1] = rho * sn;
        BoxMuller<float>::pair(xb.z, xb.w, rho, c, sn);
        z[2] = rho * c;
        z[3] = rho * sn;
        float W = 0.f;
        grid[0] = 0.f;
#pragma unroll
        for (int k = 0; k < nf; ++k) {
            float zk;
            if constexpr (NF != 0) zk = pick4(z, slot * nf + k);
            else zk = z[slot * nf + k];
            if (!level0) {
                fine_step(zk);
            } else {
                em_step<float, PAY, false>(fS, fsum, fhi, flo, fls, fmaf(a, zk, rh));
            }
            W = fmaf(sqrt_h, zk, W);
            grid[(k + 1) * (16 / nf)] = W;
        }
    } else {
        const uint32_t slo = (uint32_t)s, shi = (uint32_t)(s >> 32);
        const int per16 = nf >= 16 ? nf / 16 : 0, gstep = nf < 16 ? 16 / nf : 0;
        float acc = 0.f, W = 0.f;
        int f = 0, cnt = 0;
        grid[0] = 0.f;
#pragma unroll
        for (int j = 0; j < nf / 4; ++j) {
            const uint4 xb = philox4x32_10(make_uint4(p.ctr3, (uint32_t)j, shi, slo), p.rkey);
            float rho, c, sn, z[4];
            BoxMuller<float>::pair(xb.x, xb.y, rho, c, sn);
            z[0] = rho * c;
            z[1] = rho * sn;
            BoxMuller<float>::pair(xb.z, xb.w, rho, c, sn);
            z[2] = rho * c;
            z[3] = rho * sn;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                fine_step(z[k]);
                if (per16) {
                    acc += z[k];
                    if (++cnt == per16) {
                        W = fmaf(sqrt_h, acc, W);
                        grid[++f] = W;
                        acc = 0.f;
                        cnt = 0;
                    }
                } else {  // nf = 4 or 8: the path's own grid points
                    W = fmaf(sqrt_h, z[k], W);
                    grid[(4 * j + k + 1) * gstep] = W;
                }
            }
        }
    }
    if (nf < 16) {
        // Brownian-bridge midpoints: 16 - M^l normals from blocks b0, b0 + 1, ... of the sample's
        // own counter, b0 = max(1, M^l / 4) the first block its path does not read
        const uint32_t slo = (uint32_t)s, shi = (uint32_t)(s >> 32);
        const int b0 = nf >= 4 ? nf / 4 : 1, nblk = (19 - nf) / 4;
        float zb[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < nblk) {
                const uint4 xb = philox4x32_10(make_uint4(p.ctr3, (uint32_t)(b0 + j), shi, slo), p.rkey);
                float rho, c, sn;
                BoxMuller<float>::pair(xb.x, xb.y, rho, c, sn);
                zb[4 * j + 0] = rho * c;
                zb[4 * j + 1] = rho * sn;
                BoxMuller<float>::pair(xb.z, xb.w, rho, c, sn);
                zb[4 * j + 2] = rho * c;
                zb[4 * j + 3] = rho * sn;
            }
        }
        int next = 0;
#pragma unroll
        for (int width = 16 / nf; width > 1; width /= 2) {
            // midpoint variance: (width / 4) T / 16
            const float sd = sqrt_tg * sqrtf(0.25f * (float)width);
#pragma unroll
            for (int left = 0; left < 16; left += width) {
                const int mid = left + width / 2;
                grid[mid] = 0.5f * (grid[left] + grid[left + width]) + sd * zb[next++];
            }
        }
    }
    levy_coordinates(grid, k.inv_tg, x);
    const float logS0 = PAY == kGeoAsian ? logf(S0) : 0.f;
    const float Pf = payoff_from<float, PAY>(S0 * fS, S0 * fsum, S0 * fhi, lpost_of((float)nf, logS0, fls), k.inv_nf, k.K,
                                             k.disc, S0, k.Q);
    if (level0) {
        Y = Pf;
    } else {
        const float Pc = payoff_from<float, PAY>(S0 * cS, S0 * csum, S0 * chi, lpost_of((float)(nf / M), logS0, cls),
                                                 k.inv_nc, k.K, k.disc, S0, k.Q);
        Y = Pf - Pc;
    }
}

// Sum NV doubles over the grid: block partials into `partials`, the last block to finish adds
// them into out (every thread a fixed stride of blocks in block order, then the threads in a fixed
// tree), so the sums repeat bit for bit for a given grid.  The ticket is zero between launches.
template <int NV>
__device__ __forceinline__ void finish_sums_n(double m[NV], double *partials, unsigned *ticket, double *out)
{
    __shared__ double sm[32][NV];
    __shared__ bool is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) m[k] = warp_sum(m[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[warp][k] = m[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) m[k] = warp_sum(lane < nw ? sm[lane][k] : 0.0);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) partials[NV * blockIdx.x + k] = m[k];
            __threadfence();
            is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
#pragma unroll 4
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + NV * b + k);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[warp][k] = acc[k];  // sm's earlier values were read before the barrier above
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sm[w][k];
            out[k] = t;
        }
        *ticket = 0u;
    }
}

// Control-variate level estimator: per sample r = Y - g(x); sums
// [r, r^2, r^3, r^4, Y, Y^2, g, g^2] (FP64).  Each thread adds batches of kCvBatch samples in FP32
// and folds every batch into its FP64 sums (relative error of a batch sum at most
// (kCvBatch - 1) u of its sum of magnitudes, 4.2e-7): eight FP64 updates per sample kept GB300's
// FP64 pipe (2 operations per SM per clock) 47% busy.
constexpr int kCvBatch = 8;

// The network runs on the tcgen05 tensor cores (tc_mlp.cuh), the function the lattice mean kernel
// evaluates, so that the samples of Y - g and the estimate of E[g] use one g.
// 128 threads, one sample per thread and tile; each block strides over tiles of 128 samples (the
// stride is uniform over the block, so all its threads reach the tile's barriers; the lanes past
// N compute copies of sample N - 1 and add nothing).  A tile whose tensor-core wait ran out
// makes the sums NaN (the driver then stops on non-finite sums).
constexpr int kCvTcThreads = kTcRows;
template <int PAY, int NF = 0>
__global__ void __launch_bounds__(kCvTcThreads) cv_level_tc_kernel(const LevelParams p, const float *__restrict__ params,
                                                                   double *out8, float *r_out, float *g_out)
{
    __shared__ TcShared ts;
    __shared__ CvConsts kc;
    if (threadIdx.x == 0) kc = cv_consts(p);
    const uint32_t tmem = tc_setup(ts, params);  // ends with a block barrier
    double m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t phase = 0;
    bool ok = true;
    const uint64_t tile_stride = (uint64_t)gridDim.x * kCvTcThreads;
    uint64_t base = (uint64_t)blockIdx.x * kCvTcThreads;
    // batches of kCvBatch tiles, each folded into the FP64 sums after its loop (a fold inside the
    // tile loop was compiled as predicated FP64 work on every tile: FP64 pipe 42% busy)
#pragma unroll 1
    while (base < p.N) {
        float b[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int j = 0; j < kCvBatch && base < p.N; ++j, base += tile_stride) {
            const uint64_t idx = base + threadIdx.x;
            const bool valid = idx < p.N;
            float Y, x[kInputs];
            cv_sample<PAY, NF>(p, kc, p.first + (valid ? idx : p.N - 1), Y, x);
            const float gv = tc_mlp_tile(ts, tmem, x, phase, ok);
            if (valid) {
                const float r = Y - gv, r2 = r * r;
                b[0] += r;
                b[1] += r2;
                b[2] = fmaf(r2, r, b[2]);
                b[3] = fmaf(r2, r2, b[3]);
                b[4] += Y;
                b[5] = fmaf(Y, Y, b[5]);
                b[6] += gv;
                b[7] = fmaf(gv, gv, b[7]);
                if (r_out) r_out[idx] = r;
                if (g_out) g_out[idx] = gv;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) m[k] += (double)b[k];
    }
    tc_teardown(ts, tmem);
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = ok ? m[k] : __longlong_as_double(0x7FF8000000000000LL);
    finish_sums_n<8>(m, p.partials, p.ticket, out8);
}

}  // namespace mlmcgb
