// cv_kernels.cuh -- device code of the learned control variate (FP32 paths) beside its level
// estimator (cv_level_kernel.cuh): the lattice mean of the network, the training data and the
// standalone forward pass.
#pragma once
#include <cstdint>

#include "cv_level_kernel.cuh"

namespace mlmcgb {

// Independent sample that estimates E[g]: replicates of a randomly shifted rank-1 lattice rule
// (Sloan and Joe 1994; random shift after Cranley and Patterson 1976).  Replicate r is
// {frac(i z / n + Delta_r)}, i < n = MLMC_CV_LATTICE_POINTS, z_k = a^k mod n with the Korobov
// multiplier a = MLMC_CV_LATTICE_A, and Delta_r the sixteen words of Philox blocks 0..3 of
// counter r under the control-variate-mean tag, read as 32-bit fractions.  In fixed point a
// coordinate is v = (i z_k mod n) 2^16 + D_k mod 2^32, exact; the point keeps its top 23 bits,
// the baker's (tent) transform w = 2 v below one half, 2 (2^32 - 1 - v) above (Hickernell 2002;
// two to one onto the even fractions, so still uniform), keeps its top 23 bits, centred,
// u = (floor(w / 2^9) + 1/2) 2^-23 (exact in FP32), and x_k = Phi^{-1}(u_k).
constexpr uint32_t kLatticeN = MLMC_CV_LATTICE_POINTS;
constexpr uint32_t kLatticeChunk = 1024;                         // points per block
constexpr uint32_t kChunksPerReplicate = kLatticeN / kLatticeChunk;
static_assert(kLatticeN == 65536, "the fixed-point lattice coordinates assume n = 2^16");
static_assert(kLatticeChunk % kTcRows == 0, "whole tiles per chunk");

__host__ __device__ constexpr uint32_t lattice_z(int k)
{
    uint32_t z = 1;
    for (int j = 0; j < k; ++j) z = (z * (uint32_t)MLMC_CV_LATTICE_A) & (kLatticeN - 1);
    return z;
}

// Blocks [q * 64, q * 64 + 64) take replicate p.first + q (p.N replicates), 1024 points each:
// 128 threads, one point per thread and tile, 8 tiles, the network on the tcgen05 tensor cores
// (tc_mlp.cuh).  Each block writes the sum of g over its points to partials[block]; the last
// block forms every replicate's mean Q = (1/n) sum of its 64 partials (fixed order) and writes
// out2 = (sum Q, sum Q^2) over the launch's replicates, added to out2's old values when
// `accumulate` is set.  g_out [p.N][n] (or NULL) receives g of every point.  A tile whose
// tensor-core wait ran out makes the sums NaN (the driver then stops on non-finite sums).
constexpr int kMeanTcThreads = kTcRows;
__global__ void __launch_bounds__(kMeanTcThreads) cv_mean_tc_kernel(const LevelParams p,
                                                                    const float *__restrict__ params,
                                                                    double *out2, float *g_out, int accumulate)
{
    __shared__ TcShared s;
    __shared__ double sm[kMeanTcThreads / 32][2];
    __shared__ bool is_last;
    const uint32_t tmem = tc_setup(s, params);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t rep = blockIdx.x / kChunksPerReplicate;
    const uint32_t chunk = blockIdx.x % kChunksPerReplicate;
    const uint64_t r = p.first + rep;
    uint32_t D[kInputs];
#pragma unroll
    for (int j = 0; j < kInputs / 4; ++j) {
        const uint4 xb = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)r, (uint32_t)(r >> 32), p.ctr3),
                                       p.key0, p.key1);
        D[4 * j + 0] = xb.x;
        D[4 * j + 1] = xb.y;
        D[4 * j + 2] = xb.z;
        D[4 * j + 3] = xb.w;
    }
    double acc = 0.0;
    uint32_t phase = 0;
    bool ok = true;
#pragma unroll 1
    for (uint32_t tile = 0; tile < kLatticeChunk / kMeanTcThreads; ++tile) {
        const uint32_t i = chunk * kLatticeChunk + tile * kMeanTcThreads + threadIdx.x;
        float x[kInputs];
#pragma unroll
        for (int k = 0; k < kInputs; ++k) {
            const uint32_t v = (((i * lattice_z(k)) & (kLatticeN - 1)) << 16) + D[k];
            const uint32_t w = v < 0x80000000u ? v << 1 : (~v) << 1;  // tent: 2v, or 2 (2^32 - 1 - v)
            x[k] = normcdfinvf(((float)(w >> 9) + 0.5f) * 0x1p-23f);
        }
        const float gv = tc_mlp_tile(s, tmem, x, phase, ok);
        acc += (double)gv;
        if (g_out) g_out[rep * kLatticeN + i] = gv;
    }
    tc_teardown(s, tmem);
    if (!ok) acc = __longlong_as_double(0x7FF8000000000000LL);  // NaN: reported as non-finite sums
    acc = warp_sum(acc);
    if (lane == 0) sm[warp][0] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < kMeanTcThreads / 32; ++w) sum += sm[w][0];
        p.partials[blockIdx.x] = sum;
        __threadfence();
        is_last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const uint64_t nrep = gridDim.x / kChunksPerReplicate;
    double sq = 0.0, sqq = 0.0;
    for (uint64_t k = threadIdx.x; k < nrep; k += kMeanTcThreads) {
        double sum = 0.0;
        for (uint32_t c = 0; c < kChunksPerReplicate; ++c) sum += __ldcg(p.partials + k * kChunksPerReplicate + c);
        const double Q = sum / (double)kLatticeN;
        sq += Q;
        sqq = fma(Q, Q, sqq);
    }
    sq = warp_sum(sq);
    sqq = warp_sum(sqq);
    __syncthreads();
    if (lane == 0) {
        sm[warp][0] = sq;
        sm[warp][1] = sqq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kMeanTcThreads / 32; ++w) {
            a += sm[w][0];
            b += sm[w][1];
        }
        out2[0] = (accumulate ? out2[0] : 0.0) + a;
        out2[1] = (accumulate ? out2[1] : 0.0) + b;
        *p.ticket = 0u;
    }
}

// Training data: (x, Y) of samples [first, first + N) under the training tag.
template <int PAY>
__global__ void __launch_bounds__(256) cv_data_kernel(const LevelParams p, float *X, float *Yout)
{
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const CvConsts kc = cv_consts(p);
    for (uint64_t idx = tid; idx < p.N; idx += stride) {
        float Y, x[kInputs];
        cv_sample<PAY>(p, kc, p.first + idx, Y, x);
        Yout[idx] = Y;
#pragma unroll
        for (int k = 0; k < kInputs; ++k) X[kInputs * idx + k] = x[k];
    }
}

// g(x) for rows of X [N][16] (standalone forward, used for validation and tests).
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float *__restrict__ params, const float *X,
                                                          uint64_t N, float *G)
{
    __shared__ MlpShared net;
    __shared__ __align__(16) uint32_t xw_all[8][32 * kXStride];  // 16-byte aligned rows: warp_mlp stores uint4
    load_mlp(net, params);
    __syncthreads();
    uint32_t *xw = xw_all[threadIdx.x >> 5];
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t warp_first = tid & ~uint64_t(31);
    for (uint64_t base = 0; base + warp_first < N; base += stride) {
        const uint64_t idx = base + tid;
        const bool valid = idx < N;
        const uint64_t row = valid ? idx : N - 1;
        float x[kInputs];
#pragma unroll
        for (int k = 0; k < kInputs; ++k) x[k] = X[kInputs * row + k];
        const float gv = warp_mlp(net, xw, x);
        if (valid) G[idx] = gv;
    }
}

}  // namespace mlmcgb
