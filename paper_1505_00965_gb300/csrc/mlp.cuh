// mlp.cuh -- the control-variate network g(x) = w3 . GELU(W2 GELU(W1 x + b1) + b2) + b3 on the
// tensor cores (8 -> 64 -> 64 -> 1), evaluated by whole warps on 32 samples at a time.
//
// The two matrix products run as mma.sync m16n8k16 with bfloat16 operands and FP32
// accumulation; biases, GELU and the last layer (a 64-term dot product) are FP32.  Layer-1
// accumulator fragments are rounded to bfloat16 and reused directly as layer-2 operand
// fragments (the m16n8 accumulator layout of two adjacent column tiles is the m16k16 operand
// layout), so hidden values never leave registers.
//
// GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), tanh from the hardware unit.
#pragma once
#include <cstdint>

namespace mlmcgb {

constexpr int kHidden = 64;
constexpr int kInputs = 8;
// Packed FP32 parameters: W1 [64][8] (row = output unit), b1 [64], W2 [64][64], b2 [64],
// w3 [64], b3.
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHidden * kInputs;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kHidden * kHidden;
constexpr int kOffW3 = kOffB2 + kHidden;
constexpr int kOffB3 = kOffW3 + kHidden;
constexpr int kNumParams = kOffB3 + 1;  // 4801

// Network in shared memory: weights as packed bfloat16 pairs, the rest FP32.  A W2 row takes
// kW2Stride = 36 words (32 used): the layer-2 operand loads of a warp read word 8 kt + t of rows
// g = 0..7, which a stride of 32 would put in the same four banks; with 36 the 32 lanes hit 32
// distinct banks.
constexpr int kW2Stride = kHidden / 2 + 4;
struct MlpShared {
    uint32_t W1[kHidden * kInputs / 2];   // row o: 4 words of pairs (W1[o][2t], W1[o][2t+1])
    uint32_t W2[kHidden * kW2Stride];     // row o: 32 words of pairs (W2[o][2j], W2[o][2j+1]), then 4 unused
    float b1[kHidden], b2[kHidden], w3[kHidden];
    float b3;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float gelu(float z)
{
    // sqrt(2/pi) (z + 0.044715 z^3) = z (sqrt(2/pi) + 0.044715 sqrt(2/pi) z^2)
    const float u = z * fmaf(0.035677408136300125f, z * z, 0.7978845608028654f);
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_approx(u), hz);
}

// Two FP32 values in one 64-bit register pair, for the packed FP32 arithmetic of sm_100 and
// later (fma / mul / add .rn.f32x2: each half rounds exactly as the scalar instruction would).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_splat(float v) { return f2_pack(v, v); }

// GELU of both halves: the operations of gelu() in the same order, two values per instruction
// (bit-identical to gelu() on each half).
__device__ __forceinline__ f32x2 gelu2(f32x2 z)
{
    const f32x2 p = f2_fma(f2_mul(z, z), f2_splat(0.035677408136300125f), f2_splat(0.7978845608028654f));
    float u0, u1;
    f2_unpack(f2_mul(z, p), u0, u1);
    const f32x2 hz = f2_mul(z, f2_splat(0.5f));
    return f2_fma(hz, f2_pack(tanh_approx(u0), tanh_approx(u1)), hz);
}

// The bfloat16 pair of a packed pair (low half in the low 16 bits).
__device__ __forceinline__ uint32_t pack_bf16x2_f2(f32x2 v)
{
    float lo, hi;
    f2_unpack(v, lo, hi);
    return pack_bf16x2(lo, hi);
}

// d += a * b for one m16n8k16 tile, bfloat16 operands, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Copy packed FP32 parameters into shared memory (all threads of the block take part).
__device__ __forceinline__ void load_mlp(MlpShared &s, const float *__restrict__ params)
{
    for (int i = threadIdx.x; i < kHidden * kInputs / 2; i += blockDim.x)
        s.W1[i] = pack_bf16x2(params[kOffW1 + 2 * i], params[kOffW1 + 2 * i + 1]);
    for (int i = threadIdx.x; i < kHidden * kHidden / 2; i += blockDim.x)
        s.W2[(i >> 5) * kW2Stride + (i & 31)] = pack_bf16x2(params[kOffW2 + 2 * i], params[kOffW2 + 2 * i + 1]);
    for (int i = threadIdx.x; i < kHidden; i += blockDim.x) {
        s.b1[i] = params[kOffB1 + i];
        s.b2[i] = params[kOffB2 + i];
        s.w3[i] = params[kOffW3 + i];
    }
    if (threadIdx.x == 0) s.b3 = params[kOffB3];
}

// g for the 16 samples of one tile.  xw: the warp's staging area, xw[row * 4 + t] holds the
// bfloat16 pair (x[2t], x[2t+1]) of tile row `row`.  Returns g for rows g and g + 8 of this
// lane's group (every lane of the group gets both).
__device__ __forceinline__ void mlp_tile(const MlpShared &s, const uint32_t *xw, float &out0, float &out1)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 1: A = x (16 x 16, columns 8..15 zero), B[k][n] = W1[n][k]
    uint32_t a[4] = {xw[g * 4 + t], xw[(g + 8) * 4 + t], 0u, 0u};
    // layer 1, then A = GELU(z1) as bfloat16 (k-tile kt = n-tiles 2kt and 2kt + 1); GELU on the
    // accumulator pairs (columns 2t, 2t + 1 of rows g and g + 8) with packed FP32 arithmetic
    uint32_t a2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int o = 8 * nt + 2 * t;
        float c[4] = {s.b1[o], s.b1[o + 1], s.b1[o], s.b1[o + 1]};
        mma_bf16(c, a, s.W1[(8 * nt + g) * 4 + t], 0u);
        a2[nt >> 1][(nt & 1) * 2] = pack_bf16x2_f2(gelu2(f2_pack(c[0], c[1])));
        a2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16x2_f2(gelu2(f2_pack(c[2], c[3])));
    }
    // layer 2, B[k][n] = W2[n][k]; layer 3: the dot product with w3 over this lane's units, rows g
    // and g + 8, in packed pairs (units o and o + 1 summed at the end)
    f32x2 q0 = f2_splat(0.f), q1 = f2_splat(0.f);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int o = 8 * nt + 2 * t;
        float c[4] = {s.b2[o], s.b2[o + 1], s.b2[o], s.b2[o + 1]};
        const uint32_t *w = &s.W2[(8 * nt + g) * kW2Stride];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_bf16(c, a2[kt], w[8 * kt + t], w[8 * kt + t + 4]);
        const f32x2 w3 = f2_pack(s.w3[o], s.w3[o + 1]);
        q0 = f2_fma(w3, gelu2(f2_pack(c[0], c[1])), q0);
        q1 = f2_fma(w3, gelu2(f2_pack(c[2], c[3])), q1);
    }
    float p0, p1, e0, e1;
    f2_unpack(q0, p0, e0);
    f2_unpack(q1, p1, e1);
    p0 += e0;
    p1 += e1;
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    out0 = p0 + s.b3;
    out1 = p1 + s.b3;
}

// g(x) for the 32 samples of a warp, one per lane (all 32 lanes must call).  xw: 128 words of
// warp-private shared memory.
__device__ __forceinline__ float warp_mlp(const MlpShared &s, uint32_t *xw, const float x[8])
{
    const int lane = threadIdx.x & 31;
    // one 16-byte store per lane (four 4-byte stores at a stride of 4 words conflicted 4 ways)
    *reinterpret_cast<uint4 *>(&xw[lane * 4]) = make_uint4(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]),
                                                           pack_bf16x2(x[4], x[5]), pack_bf16x2(x[6], x[7]));
    __syncwarp();
    float mine = 0.f;
#pragma unroll 1
    for (int tile = 0; tile < 2; ++tile) {
        float r0, r1;
        mlp_tile(s, xw + tile * 64, r0, r1);
        // sample (tile * 16 + row) is lane tile * 16 + row; row < 8 holds r0 of group row
        const int row = lane & 15;
        const float v0 = __shfl_sync(0xffffffffu, r0, (row & 7) * 4);
        const float v1 = __shfl_sync(0xffffffffu, r1, (row & 7) * 4);
        if ((lane >> 4) == tile) mine = row < 8 ? v0 : v1;
    }
    __syncwarp();
    return mine;
}

}  // namespace mlmcgb
