// train_kernel.cuh -- training of the control-variate network on the GPU: every mini-batch step
// (forward, backward, parameter gradient, Adam) of every epoch in one persistent launch.
//
// The network is g(x) = w3 . GELU(W2 GELU(W1 x + b1) + b2) + b3 (16 -> 64 -> 64 -> 1) with the
// numerics of the estimator's kernels: bfloat16 operands x, W1, W2 and GELU(z1), FP32 accumulation.
// The loss is the mean of (g - t)^2 over the B rows of a batch, t = (Y - mu) / sd the
// standardised target.  Its gradient by the chain rule (d = dL/dg = 2 (g - t) / B):
//   dw3 = sum_r d_r h2_r, db3 = sum_r d_r,
//   dz2 = d w3 * GELU'(z2),  dW2 = dz2^T h1,  db2 = sum_r dz2_r,
//   dz1 = (dz2 W2) * GELU'(z1),  dW1 = dz1^T x,  db1 = sum_r dz1_r.
// The four products (two forward, dz2 W2, and the batch contractions dz2^T h1 and dz1^T x) run on
// the tensor cores as mma.sync m16n8k16 with bfloat16 operands and FP32 accumulators; dz2 and dz1
// are rounded to bfloat16 as operands (relative 2^-9 per term), the bias and w3 sums stay FP32.
//
// Layout: one thread-block cluster of C CTAs (C = 16 where the GPU can place it, else 8) per
// network; several networks (the levels) train side by side, one cluster each.  A batch of B rows
// is split into C contiguous slices of B / C rows; a CTA of 8 warps takes its slice in chunks of
// 256 rows (16 tiles of 16 rows, two per warp), staged in shared memory together with the
// bfloat16 activations that the batch contractions read.  Each CTA's partial gradient goes by
// distributed shared memory (st.shared::cluster) to the CTA that owns that part of the parameter
// vector (C equal slices); after a cluster barrier each owner adds the C partials in rank order,
// applies Adam to its slice and writes the new values into every CTA's copy of the parameters;
// after a second barrier every CTA rebuilds its bfloat16 network.  Reductions run in a fixed
// order, so a training run repeats bit for bit.  Cluster barriers are the hardware's: no thread
// spins on memory.
#pragma once
#include <cstdint>

#include "mlmc.h"
#include "mlp.cuh"

namespace mlmcgb {

constexpr int kTrainThreads = 256;          // 8 warps
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr int kTrainChunk = 256;            // rows staged at a time (16 tiles)
constexpr int kActWords = 36;               // words per staged activation row: 64 bfloat16 + 8 pad
constexpr int kTrainMaxCluster = 16;
constexpr int kTrainMinClusterAdam = 8;     // training clusters (Adam slices of at most 601)
constexpr int kTrainMaxSlice = (kNumParams + kTrainMinClusterAdam - 1) / kTrainMinClusterAdam;
constexpr int kTrainPartCols = 3 * kHidden + 1;  // per-warp sums: db1, db2, dw3, db3

struct TrainJob {
    const float *X;   // [n][16] network inputs of the job's rows
    const float *Y;   // [n] targets (before standardisation)
    float *params;    // [kNumParams] in: initial values; out: trained values
    float mu, inv_sd; // target standardisation t = (Y - mu) inv_sd
};

struct TrainArgs {
    TrainJob job[MLMC_CV_MAX_LEVELS];
    int B;            // rows per batch, a multiple of 16 C
    int steps;        // batches per epoch (batch s: rows [s B, (s + 1) B))
    int epochs;
    float lr;         // Adam step size
    float *grad_out;  // gradient mode: [kNumParams] gradient of the loss on batch 0
    float *g_out;     // gradient mode: [B] network outputs on batch 0
};

struct TrainSmem {
    uint32_t W1[kHidden * kXStride];         // bfloat16 pairs, row o: (W1[o][2j], W1[o][2j+1]), j < 8, padded
    uint32_t W2[kHidden * kW2Stride];        // row o: (W2[o][2j], W2[o][2j+1]), j < 32
    uint32_t W2T[kHidden * kW2Stride];       // row i: (W2[2j][i], W2[2j+1][i]), j < 32
    float b1[kHidden], b2[kHidden], w3[kHidden];
    float b3, pad0[3];
    float pfull[kNumParams + 3];             // FP32 parameters; the owned slice is the master copy
    float gin[kTrainMaxCluster * ((kNumParams + kTrainMaxCluster - 1) / kTrainMaxCluster) + 16];  // pushed partials
    float m1[kTrainMaxSlice], m2[kTrainMaxSlice];  // Adam moments of the owned slice
    float grad[kNumParams + 3];              // this CTA's partial gradient
    float part[kTrainWarps][kTrainPartCols + 3];
    // ldmatrix reads rows of 16 bytes: the staged operands start on 16-byte boundaries
    alignas(16) uint32_t x[kTrainChunk * kXStride];      // staged rows: 16 bfloat16 inputs (32 bytes), padded
    float y[kTrainChunk];
    alignas(16) uint32_t h1[kTrainChunk * kActWords];    // bfloat16 GELU(z1) of the staged rows
    alignas(16) uint32_t dz2[kTrainChunk * kActWords];   // bfloat16 dL/dz2
    alignas(16) uint32_t dz1[kTrainChunk * kActWords];   // bfloat16 dL/dz1
};
static_assert(sizeof(TrainSmem) <= 227 * 1024, "training CTA exceeds the shared memory of an SM");
static_assert(kTrainMaxCluster * ((kNumParams + kTrainMaxCluster - 1) / kTrainMaxCluster) >=
                  2 * ((kNumParams + 1) / 2), "gin holds C slices for every cluster size");

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// All threads of every CTA of the cluster; orders shared::cluster stores before the barrier
// before loads after it.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t dsmem_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsmem_store(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" :: "r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void ldsm_x4_trans(const void *p, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
// GELU and its derivative from one hardware tanh, on both halves of a packed pair (packed FP32
// arithmetic): with u = sqrt(2/pi) (z + 0.044715 z^3) and t = tanh(u), GELU(z) = z (1 + t) / 2
// and GELU'(z) = (1 + t) / 2 + z (1 - t^2) u'(z) / 2.
__device__ __forceinline__ void gelu_and_grad2(f32x2 z, f32x2 &h, f32x2 &dh)
{
    const f32x2 z2 = f2_mul(z, z);
    const f32x2 u = f2_mul(z, f2_fma(z2, f2_splat(0.035677408136300125f), f2_splat(0.7978845608028654f)));
    const f32x2 du = f2_fma(z2, f2_splat(3.0f * 0.035677408136300125f), f2_splat(0.7978845608028654f));
    float u0, u1;
    f2_unpack(u, u0, u1);
    const f32x2 t = f2_pack(tanh_approx(u0), tanh_approx(u1));
    const f32x2 hz = f2_mul(z, f2_splat(0.5f));
    h = f2_fma(hz, t, hz);
    // (1 + t) / 2 + hz (1 - t^2) u' with 1 - t^2 = fma(t, -t, 1)
    const f32x2 q = f2_fma(t, f2_mul(t, f2_splat(-1.0f)), f2_splat(1.0f));
    dh = f2_fma(f2_mul(hz, q), du, f2_fma(t, f2_splat(0.5f), f2_splat(0.5f)));
}

// The bfloat16 network from the FP32 parameters in s.pfull (all threads; ends with a barrier).
__device__ __forceinline__ void train_build_net(TrainSmem &s)
{
    for (int i = threadIdx.x; i < kHidden * kInputs / 2; i += kTrainThreads)
        s.W1[(i >> 3) * kXStride + (i & 7)] = pack_bf16x2(s.pfull[kOffW1 + 2 * i], s.pfull[kOffW1 + 2 * i + 1]);
    for (int i = threadIdx.x; i < kHidden * kHidden / 2; i += kTrainThreads) {
        const int o = i >> 5, c = i & 31;
        s.W2[o * kW2Stride + c] = pack_bf16x2(s.pfull[kOffW2 + o * kHidden + 2 * c], s.pfull[kOffW2 + o * kHidden + 2 * c + 1]);
        // transposed copy: consecutive threads take consecutive rows i (consecutive words read)
        const int r = i & 63, c2 = i >> 6;
        s.W2T[r * kW2Stride + c2] = pack_bf16x2(s.pfull[kOffW2 + (2 * c2) * kHidden + r],
                                               s.pfull[kOffW2 + (2 * c2 + 1) * kHidden + r]);
    }
    for (int i = threadIdx.x; i < kHidden; i += kTrainThreads) {
        s.b1[i] = s.pfull[kOffB1 + i];
        s.b2[i] = s.pfull[kOffB2 + i];
        s.w3[i] = s.pfull[kOffW3 + i];
    }
    if (threadIdx.x == 0) s.b3 = s.pfull[kOffB3];
    __syncthreads();
}

// Per-lane sums over the rows a lane sees (columns 8 nt + 2 t, + 1 of each quantity).
struct TrainLaneSums {
    float db1[8][2], db2[8][2], dw3[8][2];
    float db3;
};

// Forward and backward pass of one tile of 16 staged rows (rows 16 tile .. 16 tile + 15 of the
// chunk) by one warp: writes bfloat16 GELU(z1), dz2 and dz1 of the rows into the staging area,
// adds the bias and w3 gradient terms into `acc`, and in gradient mode writes g of each row to
// g_row[row].
__device__ __forceinline__ void train_tile(TrainSmem &s, int tile, float dscale, float mu, float inv_sd,
                                           TrainLaneSums &acc, float *g_row)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = 16 * tile + g, r1 = r0 + 8;
    // layer 1: A = x (16 x 16), B[k][n] = W1[n][k]
    const uint32_t a[4] = {s.x[r0 * kXStride + t], s.x[r1 * kXStride + t], s.x[r0 * kXStride + t + 4],
                           s.x[r1 * kXStride + t + 4]};
    float gz1[8][4];
    uint32_t a2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int o = 8 * nt + 2 * t;
        float c[4] = {s.b1[o], s.b1[o + 1], s.b1[o], s.b1[o + 1]};
        mma_bf16(c, a, s.W1[(8 * nt + g) * kXStride + t], s.W1[(8 * nt + g) * kXStride + t + 4]);
        f32x2 h01, h23, d01, d23;
        gelu_and_grad2(f2_pack(c[0], c[1]), h01, d01);
        gelu_and_grad2(f2_pack(c[2], c[3]), h23, d23);
        f2_unpack(d01, gz1[nt][0], gz1[nt][1]);
        f2_unpack(d23, gz1[nt][2], gz1[nt][3]);
        const uint32_t w01 = pack_bf16x2_f2(h01), w23 = pack_bf16x2_f2(h23);
        a2[nt >> 1][(nt & 1) * 2] = w01;
        a2[nt >> 1][(nt & 1) * 2 + 1] = w23;
        s.h1[r0 * kActWords + 4 * nt + t] = w01;
        s.h1[r1 * kActWords + 4 * nt + t] = w23;
    }
    // layer 2 and the output
    float h2[8][4], gz2[8][4];
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int o = 8 * nt + 2 * t;
        float c[4] = {s.b2[o], s.b2[o + 1], s.b2[o], s.b2[o + 1]};
        const uint32_t *w = &s.W2[(8 * nt + g) * kW2Stride];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_bf16(c, a2[kt], w[8 * kt + t], w[8 * kt + t + 4]);
        f32x2 h01, h23, d01, d23;
        gelu_and_grad2(f2_pack(c[0], c[1]), h01, d01);
        gelu_and_grad2(f2_pack(c[2], c[3]), h23, d23);
        f2_unpack(h01, h2[nt][0], h2[nt][1]);
        f2_unpack(h23, h2[nt][2], h2[nt][3]);
        f2_unpack(d01, gz2[nt][0], gz2[nt][1]);
        f2_unpack(d23, gz2[nt][2], gz2[nt][3]);
        p0 = fmaf(s.w3[o], h2[nt][0], p0);
        p0 = fmaf(s.w3[o + 1], h2[nt][1], p0);
        p1 = fmaf(s.w3[o], h2[nt][2], p1);
        p1 = fmaf(s.w3[o + 1], h2[nt][3], p1);
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    const float gv0 = p0 + s.b3, gv1 = p1 + s.b3;
    if (g_row && t == 0) {
        g_row[r0] = gv0;
        g_row[r1] = gv1;
    }
    const float d0 = dscale * (gv0 - (s.y[r0] - mu) * inv_sd);
    const float d1 = dscale * (gv1 - (s.y[r1] - mu) * inv_sd);
    if (t == 0) acc.db3 += d0 + d1;
    // dz2 = d w3 GELU'(z2): FP32 sums, bfloat16 operands of the next products
    uint32_t a3[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int o = 8 * nt + 2 * t;
        acc.dw3[nt][0] = fmaf(d0, h2[nt][0], fmaf(d1, h2[nt][2], acc.dw3[nt][0]));
        acc.dw3[nt][1] = fmaf(d0, h2[nt][1], fmaf(d1, h2[nt][3], acc.dw3[nt][1]));
        const float e0 = d0 * s.w3[o], e1 = d0 * s.w3[o + 1], f0 = d1 * s.w3[o], f1 = d1 * s.w3[o + 1];
        const float z0 = e0 * gz2[nt][0], z1 = e1 * gz2[nt][1], z2 = f0 * gz2[nt][2], z3 = f1 * gz2[nt][3];
        acc.db2[nt][0] += z0 + z2;
        acc.db2[nt][1] += z1 + z3;
        const uint32_t w01 = pack_bf16x2(z0, z1), w23 = pack_bf16x2(z2, z3);
        a3[nt >> 1][(nt & 1) * 2] = w01;
        a3[nt >> 1][(nt & 1) * 2 + 1] = w23;
        s.dz2[r0 * kActWords + 4 * nt + t] = w01;
        s.dz2[r1 * kActWords + 4 * nt + t] = w23;
    }
    // dz1 = (dz2 W2) GELU'(z1): B[k = o][n = i] = W2[o][i] from the transposed copy
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t *w = &s.W2T[(8 * nt + g) * kW2Stride];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_bf16(c, a3[kt], w[8 * kt + t], w[8 * kt + t + 4]);
        const float z0 = c[0] * gz1[nt][0], z1 = c[1] * gz1[nt][1], z2 = c[2] * gz1[nt][2], z3 = c[3] * gz1[nt][3];
        acc.db1[nt][0] += z0 + z2;
        acc.db1[nt][1] += z1 + z3;
        s.dz1[r0 * kActWords + 4 * nt + t] = pack_bf16x2(z0, z1);
        s.dz1[r1 * kActWords + 4 * nt + t] = pack_bf16x2(z2, z3);
    }
}

// Batch contractions over the `nrows` staged rows (a multiple of 16), added into this warp's
// accumulators: warp w takes dW2 rows o in [16 (w / 2), +16) and columns u in [32 (w % 2), +32)
// (four n-tiles), warps 0..3 also dW1 rows u in [16 w, +16) (all 16 columns, two n-tiles).  Operands are read
// with ldmatrix.trans: the staged activations are row-major in the batch index r, which is the
// products' k.
__device__ __forceinline__ void train_contract(const TrainSmem &s, int nrows, float gw2[4][4], float gw1[2][4])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mi = lane >> 3, rr = lane & 7;
    const int mt = warp >> 1, n0 = 4 * (warp & 1);
    for (int kk = 0; kk < nrows; kk += 16) {
        // A = dz2^T: matrix mi holds rows r = kk + rr (+ 8 for mi >= 2), columns o = 16 mt (+ 8 for odd mi)
        const int ar = kk + rr + ((mi & 2) ? 8 : 0);
        uint32_t a[4];
        ldsm_x4_trans(&s.dz2[ar * kActWords + 8 * mt + ((mi & 1) ? 4 : 0)], a[0], a[1], a[2], a[3]);
#pragma unroll
        for (int jj = 0; jj < 4; jj += 2) {
            // B = h1 for n-tiles n0 + jj and n0 + jj + 1: matrix mi holds rows r = kk + rr (+ 8 for
            // odd mi), columns u = 8 (n0 + jj) (+ 8 for mi >= 2)
            const int br = kk + rr + ((mi & 1) ? 8 : 0);
            const int bc = 8 * (n0 + jj) + ((mi & 2) ? 8 : 0);
            uint32_t b[4];
            ldsm_x4_trans(&s.h1[br * kActWords + bc / 2], b[0], b[1], b[2], b[3]);
            mma_bf16(gw2[jj], a, b[0], b[1]);
            mma_bf16(gw2[jj + 1], a, b[2], b[3]);
        }
        if (warp < 4) {
            uint32_t a1[4];
            ldsm_x4_trans(&s.dz1[ar * kActWords + 8 * warp + ((mi & 1) ? 4 : 0)], a1[0], a1[1], a1[2], a1[3]);
            // B = x for n-tiles 0 and 1: matrix mi holds rows r = kk + rr (+ 8 for odd mi), columns
            // 0..7 (8..15 for mi >= 2)
            const int xr = kk + rr + ((mi & 1) ? 8 : 0);
            uint32_t b[4];
            ldsm_x4_trans(&s.x[xr * kXStride + ((mi & 2) ? 4 : 0)], b[0], b[1], b[2], b[3]);
            mma_bf16(gw1[0], a1, b[0], b[1]);
            mma_bf16(gw1[1], a1, b[2], b[3]);
        }
    }
}

// Training (TRAIN) or one gradient evaluation (!TRAIN) of the networks of a.job[cluster index].
template <bool TRAIN>
__global__ void __launch_bounds__(kTrainThreads, 1) train_cluster_kernel(const TrainArgs a)
{
    extern __shared__ __align__(128) uint8_t train_smem_raw[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(train_smem_raw);
    const int C = (int)cluster_nctarank(), rank = (int)cluster_ctarank();
    const TrainJob job = a.job[blockIdx.x / C];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = (kNumParams + C - 1) / C;              // parameters per owner
    const uint32_t inv_s = (uint32_t)((0x100000000ull + (uint64_t)S - 1) / (uint64_t)S);  // ceil(2^32 / S)
    const int lo = rank * S, nown = max(0, min(S, kNumParams - lo));
    const int rows = a.B / C;                            // this CTA's rows of every batch
    const int chunks = (rows + kTrainChunk - 1) / kTrainChunk;
    const float dscale = 2.0f / (float)a.B;

    for (int i = tid; i < kNumParams; i += kTrainThreads) s.pfull[i] = job.params[i];
    if (TRAIN) {
        for (int i = tid; i < nown; i += kTrainThreads) s.m1[i] = s.m2[i] = 0.f;
    }
    __syncthreads();
    train_build_net(s);
    cluster_sync();  // every CTA of the cluster is running before any distributed store

    // rows of (step, chunk) are prefetched into registers one chunk ahead
    float px[kInputs], py = 0.f;
    auto fetch = [&](int step, int chunk) {
        const int local = chunk * kTrainChunk + tid;
        if (local < rows) {
            const size_t row = (size_t)step * a.B + (size_t)rank * rows + local;
#pragma unroll
            for (int k = 0; k < kInputs; ++k) px[k] = __ldg(job.X + kInputs * row + k);
            py = __ldg(job.Y + row);
        } else {
#pragma unroll
            for (int k = 0; k < kInputs; ++k) px[k] = 0.f;
            py = 0.f;
        }
    };
    fetch(0, 0);
    const int total = TRAIN ? a.epochs * a.steps : 1;
    const float b1c = 0.9f, b2c = 0.999f;
    for (int it = 0; it < total; ++it) {
        const int step = it % a.steps;
        TrainLaneSums acc;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int e = 0; e < 2; ++e) acc.db1[nt][e] = acc.db2[nt][e] = acc.dw3[nt][e] = 0.f;
        }
        acc.db3 = 0.f;
        float gw2[4][4], gw1[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int j = 0; j < 4; ++j) gw2[j][0] = gw2[j][1] = gw2[j][2] = gw2[j][3] = 0.f;
        for (int ch = 0; ch < chunks; ++ch) {
            const int nrows = min(kTrainChunk, rows - ch * kTrainChunk);
            uint4 *xrow = reinterpret_cast<uint4 *>(&s.x[tid * kXStride]);
            xrow[0] = make_uint4(pack_bf16x2(px[0], px[1]), pack_bf16x2(px[2], px[3]), pack_bf16x2(px[4], px[5]),
                                 pack_bf16x2(px[6], px[7]));
            xrow[1] = make_uint4(pack_bf16x2(px[8], px[9]), pack_bf16x2(px[10], px[11]), pack_bf16x2(px[12], px[13]),
                                 pack_bf16x2(px[14], px[15]));
            s.y[tid] = py;
            if (ch + 1 < chunks) fetch(step, ch + 1);
            else if (it + 1 < total) fetch((it + 1) % a.steps, 0);
            __syncthreads();
            float *g_row = TRAIN ? nullptr : a.g_out + (size_t)rank * rows + (size_t)ch * kTrainChunk;
            for (int tile = warp; tile < nrows / 16; tile += kTrainWarps)
                train_tile(s, tile, dscale, job.mu, job.inv_sd, acc, g_row);
            __syncthreads();
            train_contract(s, nrows, gw2, gw1);
            __syncthreads();  // the staging area is rewritten by the next chunk
        }
        // this CTA's partial gradient: products from the accumulators (lane (g, t) holds rows
        // g and g + 8, columns 2 t and 2 t + 1 of its tiles), sums reduced over the warp's rows
        {
            const int g = lane >> 2, t = lane & 3, mt = warp >> 1, n0 = 4 * (warp & 1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = 16 * mt + g, u = 8 * (n0 + j) + 2 * t;
                s.grad[kOffW2 + o * kHidden + u] = gw2[j][0];
                s.grad[kOffW2 + o * kHidden + u + 1] = gw2[j][1];
                s.grad[kOffW2 + (o + 8) * kHidden + u] = gw2[j][2];
                s.grad[kOffW2 + (o + 8) * kHidden + u + 1] = gw2[j][3];
            }
            if (warp < 4) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int u = 16 * warp + g, k = 8 * j + 2 * t;
                    s.grad[kOffW1 + u * kInputs + k] = gw1[j][0];
                    s.grad[kOffW1 + u * kInputs + k + 1] = gw1[j][1];
                    s.grad[kOffW1 + (u + 8) * kInputs + k] = gw1[j][2];
                    s.grad[kOffW1 + (u + 8) * kInputs + k + 1] = gw1[j][3];
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float v1 = acc.db1[nt][e], v2 = acc.db2[nt][e], v3 = acc.dw3[nt][e];
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                        v3 += __shfl_xor_sync(0xffffffffu, v3, o);
                    }
                    if (g == 0) {
                        const int col = 8 * nt + 2 * t + e;
                        s.part[warp][col] = v1;
                        s.part[warp][kHidden + col] = v2;
                        s.part[warp][2 * kHidden + col] = v3;
                    }
                }
            }
            float v = acc.db3;
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s.part[warp][3 * kHidden] = v;
        }
        __syncthreads();
        if (tid < kTrainPartCols) {
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < kTrainWarps; ++w) v += s.part[w][tid];
            const int off = tid < kHidden ? kOffB1 + tid
                          : tid < 2 * kHidden ? kOffB2 + tid - kHidden
                          : tid < 3 * kHidden ? kOffW3 + tid - 2 * kHidden : kOffB3;
            s.grad[off] = v;
        }
        __syncthreads();
        // push the partial gradient to the owners: owner q keeps C slices, this CTA's at rank S.
        // q = i / S as a multiply-high by ceil(2^32 / S): for i < 5313 and S >= 333 the error
        // i (ceil(2^32 / S) - 2^32 / S) / 2^32 stays below 2e-6 while i / S is at least 1 / S below
        // the next integer, so the quotient is exact.
        for (int i = tid; i < kNumParams; i += kTrainThreads) {
            const int q = (int)__umulhi((uint32_t)i, inv_s);
            dsmem_store(dsmem_addr(&s.gin[rank * S + (i - q * S)], (uint32_t)q), s.grad[i]);
        }
        cluster_sync();
        // owner: the batch gradient of its slice (partials added in rank order)
        if (TRAIN) {
            const float step_t = (float)(it + 1);
            const float c1 = 1.0f / (1.0f - powf(b1c, step_t)), c2 = 1.0f / (1.0f - powf(b2c, step_t));
            for (int j = tid; j < nown; j += kTrainThreads) {
                float gsum = 0.f;
                for (int c = 0; c < C; ++c) gsum += s.gin[c * S + j];
                const float m = fmaf(b1c, s.m1[j], (1.f - b1c) * gsum);
                const float v = fmaf(b2c, s.m2[j], (1.f - b2c) * gsum * gsum);
                s.m1[j] = m;
                s.m2[j] = v;
                const float p = s.pfull[lo + j] - a.lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
                for (int c = 0; c < C; ++c) dsmem_store(dsmem_addr(&s.pfull[lo + j], (uint32_t)c), p);
            }
            cluster_sync();
            train_build_net(s);
        } else {
            for (int j = tid; j < nown; j += kTrainThreads) {
                float gsum = 0.f;
                for (int c = 0; c < C; ++c) gsum += s.gin[c * S + j];
                a.grad_out[lo + j] = gsum;
            }
        }
    }
    if (TRAIN) {
        for (int j = tid; j < nown; j += kTrainThreads) job.params[lo + j] = s.pfull[lo + j];
    }
    cluster_sync();  // no CTA leaves while another may still address its shared memory
}

}  // namespace mlmcgb
