// tc_mlp.cuh -- the control-variate network on the fifth-generation tensor cores (tcgen05):
// g(x) = w3 . GELU(W2 GELU(W1 x + b1) + b2) + b3 for a tile of 128 samples per CTA.
//
// Both products are tcgen05.mma kind::f16 with bfloat16 operands in shared memory and an FP32
// accumulator of 128 x 64 in tensor memory (TMEM): layer 1 is one MMA (K = 16, the 16 inputs),
// layer 2 four (K = 64).  One thread issues the MMAs; their completion is
// signalled through an mbarrier (tcgen05.commit), which the CTA waits on with a bounded spin.
// The epilogues read the accumulator with tcgen05.ld (thread t of the CTA owns row t, i.e. one
// sample), add the bias and apply GELU in FP32 with the hardware tanh; layer 1's result is
// rounded to bfloat16 and written back to shared memory as layer 2's A operand.  The numerics
// are those of the mma.sync form (bfloat16 x, W1, W2, GELU(z1); FP32 accumulation and epilogue),
// including its exact folding of GELU's factor 1/2 into W2 and w3.
//
// Operand layout (no swizzle, K-major): 8 x 8 bfloat16 "core matrices" of 128 contiguous bytes
// (row r at byte 16 r); the two core matrices of one MMA's K = 16 sit LBO = 128 bytes apart and
// consecutive 8-row groups SBO = (K / 8) x 128 bytes apart.  Element (row, k) of an operand with
// K columns is at byte (row / 8) SBO + (k / 8) 128 + (row % 8) 16 + (k % 8) 2.
#pragma once
#include <cstdint>

#include "mlp.cuh"

namespace mlmcgb {

constexpr int kTcRows = 128;       // samples per tile: the MMA's M
constexpr uint32_t kTcCols = 64;   // TMEM columns: one FP32 128 x 64 accumulator, reused by both layers
constexpr uint32_t kTcWaitLimit = 1u << 22;  // mbarrier polls before a tile is declared failed

struct TcShared {
    alignas(1024) uint8_t a1[kTcRows * 16 * 2];      // x: 128 x 16 bfloat16, SBO 256
    alignas(1024) uint8_t a2[kTcRows * 64 * 2];      // 2 GELU(z1): 128 x 64 bfloat16, SBO 1024
    alignas(1024) uint8_t w1[kHidden * 16 * 2];      // W1: 64 x 16 bfloat16, SBO 256
    alignas(1024) uint8_t w2[kHidden * 64 * 2];      // W2 / 2: 64 x 64 bfloat16, SBO 1024
    float b1[kHidden], b2[kHidden], w3[kHidden];     // w3 halved
    float b3;
    alignas(8) uint64_t mbar;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t cm_byte(int row, int k, int sbo)
{
    return (uint32_t)((row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bfloat16 A and B, both K-major,
// N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy stores to shared memory made visible to the tensor cores' reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the phase with the given parity to complete; false if it did not within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    const uint32_t a = smem_u32(mbar);
    for (uint32_t i = 0; i < kTcWaitLimit; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Columns col .. col + 15 of this thread's TMEM lane (32x32b shape: thread t of a warp reads lane
// (lane base of the warp) + t), waited for before return.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                 "%12, %13, %14, %15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// One CTA of 128 threads.  Prologue: the network's weights into the operand layout, the mbarrier
// and 64 TMEM columns (warp 0).  Returns the TMEM base address.
__device__ __forceinline__ uint32_t tc_setup(TcShared &s, const float *__restrict__ params)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    static_assert(kInputs == 16, "layer 1 is one MMA of K = 16");
    for (int i = tid; i < kHidden * 8; i += blockDim.x) {  // W1 pairs (n, k..k+1), k < 16
        const int n = i >> 3, k = 2 * (i & 7);
        *reinterpret_cast<uint32_t *>(s.w1 + cm_byte(n, k, 256)) =
            pack_bf16x2(params[kOffW1 + n * kInputs + k], params[kOffW1 + n * kInputs + k + 1]);
    }
    for (int i = tid; i < kHidden * 32; i += blockDim.x) {  // W2 / 2 pairs (the epilogues form 2 GELU)
        const int n = i >> 5, k = 2 * (i & 31);
        *reinterpret_cast<uint32_t *>(s.w2 + cm_byte(n, k, 1024)) =
            pack_bf16x2(0.5f * params[kOffW2 + n * kHidden + k], 0.5f * params[kOffW2 + n * kHidden + k + 1]);
    }
    for (int i = tid; i < kHidden; i += blockDim.x) {
        s.b1[i] = params[kOffB1 + i];
        s.b2[i] = params[kOffB2 + i];
        s.w3[i] = 0.5f * params[kOffW3 + i];
    }
    if (tid == 0) {
        s.b3 = params[kOffB3];
        mbar_init(&s.mbar, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s.tmem_base)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return s.tmem_base;
}

__device__ __forceinline__ void tc_teardown(TcShared &s, uint32_t tmem)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols) : "memory");
    }
}

// g for the sample of this thread (row threadIdx.x of the tile) from its inputs x[16].  All 128
// threads of the CTA call it together.  `phase` is the mbarrier parity to wait for next; `ok`
// turns false if a wait ran out (the result is then meaningless and the caller reports it).
__device__ __forceinline__ float tc_mlp_tile(TcShared &s, uint32_t tmem, const float x[kInputs], uint32_t &phase,
                                             bool &ok)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    // layer-1 A operand: this thread's row, k = 0..7 and 8..15 (two core matrices)
    *reinterpret_cast<uint4 *>(s.a1 + cm_byte(tid, 0, 256)) =
        make_uint4(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]), pack_bf16x2(x[4], x[5]), pack_bf16x2(x[6], x[7]));
    *reinterpret_cast<uint4 *>(s.a1 + cm_byte(tid, 8, 256)) = make_uint4(
        pack_bf16x2(x[8], x[9]), pack_bf16x2(x[10], x[11]), pack_bf16x2(x[12], x[13]), pack_bf16x2(x[14], x[15]));
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        tc_mma(tmem, tc_smem_desc(s.a1, 128, 256), tc_smem_desc(s.w1, 128, 256), 0u);
        tc_commit(&s.mbar);
    }
    ok = mbar_wait(&s.mbar, phase) && ok;
    phase ^= 1u;
    tc_fence_after();
    // epilogue 1: 2 GELU(z1 + b1) as bfloat16 into the layer-2 A operand (the layer-2 weights are
    // halved), 16 columns at a time, in packed FP32 pairs
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[16];
        tmem_ld16(taddr + 16u * c, z);
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            h[j] = pack_bf16x2_f2(twice_gelu2(f2_add(f2_pack(z[2 * j], z[2 * j + 1]),
                                               f2_pack(s.b1[16 * c + 2 * j], s.b1[16 * c + 2 * j + 1]))));
        *reinterpret_cast<uint4 *>(s.a2 + cm_byte(tid, 16 * c, 1024)) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(s.a2 + cm_byte(tid, 16 * c + 8, 1024)) = make_uint4(h[4], h[5], h[6], h[7]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc_mma(tmem, tc_smem_desc(s.a2 + 256 * kk, 128, 1024), tc_smem_desc(s.w2 + 256 * kk, 128, 1024),
                   kk > 0 ? 1u : 0u);
        tc_commit(&s.mbar);
    }
    ok = mbar_wait(&s.mbar, phase) && ok;
    phase ^= 1u;
    tc_fence_after();
    // epilogue 2: g = b3 + sum_o (w3_o / 2) 2 GELU(z2_o + b2_o), in packed FP32 pairs (even and odd
    // units summed apart, then together)
    f32x2 q = f2_splat(0.f);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[16];
        tmem_ld16(taddr + 16u * c, z);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int o = 16 * c + 2 * j;
            const f32x2 h = twice_gelu2(f2_add(f2_pack(z[2 * j], z[2 * j + 1]), f2_pack(s.b2[o], s.b2[o + 1])));
            q = f2_fma(f2_pack(s.w3[o], s.w3[o + 1]), h, q);
        }
    }
    float qe, qo;
    f2_unpack(q, qe, qo);
    const float g = s.b3 + (qe + qo);
    tc_fence_before();  // the next tile's MMAs overwrite the accumulator after the next barrier
    return g;
}

}  // namespace mlmcgb
