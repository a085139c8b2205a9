// mlp.cuh -- the control-variate network g(x) = w3 . GELU(W2 GELU(W1 x + b1) + b2) + b3 on the
// tensor cores (16 -> 64 -> 64 -> 1), evaluated by whole warps on 32 samples at a time.
//
// The two matrix products run as mma.sync m16n8k16 with bfloat16 operands and FP32
// accumulation; biases, GELU and the last layer (a 64-term dot product) are FP32.  Layer-1
// accumulator fragments are rounded to bfloat16 and reused directly as layer-2 operand
// fragments (the m16n8 accumulator layout of two adjacent column tiles is the m16k16 operand
// layout), so hidden values never leave registers.
//
// GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), tanh from the hardware unit.  The
// kernels evaluate 2 GELU(z) = z + z tanh(.) and take the factor 1/2 into the weights that
// consume it (W2 and w3 halved when they are loaded).  Scaling by a power of two commutes with
// every rounding involved (FP32 fma, bfloat16 conversion, the exact bfloat16 products of the
// tensor cores) for values outside the subnormal range, so g is bit-identical to the plain form.
#pragma once
#include <cstdint>

namespace mlmcgb {

constexpr int kHidden = 64;
constexpr int kInputs = 16;
// Packed FP32 parameters: W1 [64][16] (row = output unit), b1 [64], W2 [64][64], b2 [64],
// w3 [64], b3.
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHidden * kInputs;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kHidden * kHidden;
constexpr int kOffW3 = kOffB2 + kHidden;
constexpr int kOffB3 = kOffW3 + kHidden;
constexpr int kNumParams = kOffB3 + 1;  // 5313
// A staged row of 16 bfloat16 inputs (8 words) takes kXStride = 12 words: the rows g = 0..7 that
// one operand fetch (word t or t + 4 of each) or one ldmatrix (16 bytes of each) reads then fall in
// distinct banks.
constexpr int kXStride = 12;

// Network in shared memory, laid out so that each lane fetches its operand fragments with
// 16-byte loads:
// - L1[32 nt + lane] = {W1 pairs of row 8 nt + g at columns (2t, 2t + 1) and (8 + 2t, 9 + 2t)
//   (lane = 4 g + t); b1[8 nt + 2t]; b1[8 nt + 2t + 1]}: one load gives a layer-1 column tile's B
//   fragment and bias pair.
// - W2: row o holds the 32 bfloat16 pairs (W2[o][2j], W2[o][2j+1]) / 2 in the order a lane of
//   quad index t reads them, words 8 kt + t and 8 kt + t + 4 for kt = 0..3 at positions
//   8 t + 2 kt and 8 t + 2 kt + 1, so its eight words are two 16-byte loads.  A row takes
//   kW2Stride = 36 words: a quarter warp (rows g, g + 1 at t = 0..3) then covers all 32 banks.
// - b2w3[i] = {b2[2i], b2[2i+1], w3[2i] / 2, w3[2i+1] / 2}.
constexpr int kW2Stride = kHidden / 2 + 4;
struct MlpShared {
    uint4 L1[8 * 32];
    uint32_t W2[kHidden * kW2Stride];
    float4 b2w3[kHidden / 2];
    float b3;
};

// Position within a W2 row of the pair word w = 8 kt + 4 half + t (see MlpShared).
__host__ __device__ constexpr int w2_slot(int w) { return 8 * (w & 3) + 2 * (w >> 3) + ((w >> 2) & 1); }

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

// 2 GELU(z) of both halves: u = z (sqrt(2/pi) + 0.044715 sqrt(2/pi) z^2), then z + z tanh(u)
// (each half equals twice the scalar z/2 + (z/2) tanh(u) exactly).
__device__ __forceinline__ f32x2 twice_gelu2(f32x2 z)
{
    const f32x2 p = f2_fma(f2_mul(z, z), f2_splat(0.035677408136300125f), f2_splat(0.7978845608028654f));
    float u0, u1;
    f2_unpack(f2_mul(z, p), u0, u1);
    return f2_fma(z, f2_pack(tanh_approx(u0), tanh_approx(u1)), z);
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
    for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) {
        const int nt = i >> 5, g = (i & 31) >> 2, t = i & 3, row = 8 * nt + g, o = 8 * nt + 2 * t;
        const float *w = params + kOffW1 + row * kInputs;
        s.L1[i] = make_uint4(pack_bf16x2(w[2 * t], w[2 * t + 1]), pack_bf16x2(w[8 + 2 * t], w[9 + 2 * t]),
                             __float_as_uint(params[kOffB1 + o]), __float_as_uint(params[kOffB1 + o + 1]));
    }
    for (int i = threadIdx.x; i < kHidden * kHidden / 2; i += blockDim.x)
        s.W2[(i >> 5) * kW2Stride + w2_slot(i & 31)] =
            pack_bf16x2(0.5f * params[kOffW2 + 2 * i], 0.5f * params[kOffW2 + 2 * i + 1]);
    for (int i = threadIdx.x; i < kHidden / 2; i += blockDim.x)
        s.b2w3[i] = make_float4(params[kOffB2 + 2 * i], params[kOffB2 + 2 * i + 1], 0.5f * params[kOffW3 + 2 * i],
                                0.5f * params[kOffW3 + 2 * i + 1]);
    if (threadIdx.x == 0) s.b3 = params[kOffB3];
}

// g for the 16 samples of one tile.  xw: the warp's staging area, xw[row * kXStride + j] holds the
// bfloat16 pair (x[2j], x[2j+1]) of tile row `row`, j < 8.  Returns g for rows g and g + 8 of this
// lane's group (every lane of the group gets both).
__device__ __forceinline__ void mlp_tile(const MlpShared &s, const uint32_t *xw, float &out0, float &out1)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 1: A = x (16 x 16), B[k][n] = W1[n][k]
    const uint32_t a[4] = {xw[g * kXStride + t], xw[(g + 8) * kXStride + t], xw[g * kXStride + t + 4],
                           xw[(g + 8) * kXStride + t + 4]};
    // layer 1, then A = 2 GELU(z1) as bfloat16 (k-tile kt = n-tiles 2kt and 2kt + 1); GELU on the
    // accumulator pairs (columns 2t, 2t + 1 of rows g and g + 8) with packed FP32 arithmetic
    uint32_t a2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const uint4 l1 = s.L1[32 * nt + lane];
        const float b1a = __uint_as_float(l1.z), b1b = __uint_as_float(l1.w);
        float c[4] = {b1a, b1b, b1a, b1b};
        mma_bf16(c, a, l1.x, l1.y);
        a2[nt >> 1][(nt & 1) * 2] = pack_bf16x2_f2(twice_gelu2(f2_pack(c[0], c[1])));
        a2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16x2_f2(twice_gelu2(f2_pack(c[2], c[3])));
    }
    // layer 2, B[k][n] = W2[n][k] / 2; layer 3: the dot product with w3 / 2 over this lane's
    // units, rows g and g + 8, in packed pairs (units o and o + 1 summed at the end)
    f32x2 q0 = f2_splat(0.f), q1 = f2_splat(0.f);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float4 bw = s.b2w3[4 * nt + t];
        float c[4] = {bw.x, bw.y, bw.x, bw.y};
        const uint4 *w = reinterpret_cast<const uint4 *>(&s.W2[(8 * nt + g) * kW2Stride + 8 * t]);
        const uint4 w01 = w[0], w23 = w[1];
        mma_bf16(c, a2[0], w01.x, w01.y);
        mma_bf16(c, a2[1], w01.z, w01.w);
        mma_bf16(c, a2[2], w23.x, w23.y);
        mma_bf16(c, a2[3], w23.z, w23.w);
        const f32x2 w3 = f2_pack(bw.z, bw.w);
        q0 = f2_fma(w3, twice_gelu2(f2_pack(c[0], c[1])), q0);
        q1 = f2_fma(w3, twice_gelu2(f2_pack(c[2], c[3])), q1);
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

// g(x) for the 32 samples of a warp, one per lane (all 32 lanes must call).  xw: 32 kXStride
// words of warp-private shared memory, 16-byte aligned.
__device__ __forceinline__ float warp_mlp(const MlpShared &s, uint32_t *xw, const float x[kInputs])
{
    const int lane = threadIdx.x & 31;
    // two 16-byte stores per lane
    uint4 *row = reinterpret_cast<uint4 *>(&xw[lane * kXStride]);
    row[0] = make_uint4(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]), pack_bf16x2(x[4], x[5]), pack_bf16x2(x[6], x[7]));
    row[1] = make_uint4(pack_bf16x2(x[8], x[9]), pack_bf16x2(x[10], x[11]), pack_bf16x2(x[12], x[13]),
                        pack_bf16x2(x[14], x[15]));
    __syncwarp();
    float mine = 0.f;
#pragma unroll 1
    for (int tile = 0; tile < 2; ++tile) {
        float r0, r1;
        mlp_tile(s, xw + tile * 16 * kXStride, r0, r1);
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
