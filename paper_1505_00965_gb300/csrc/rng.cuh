// rng.cuh -- counter-based normal generation in registers (device only).
//
// The random input of Euler--Maruyama (Sec. 2, Eq. em) is a sequence of Brownian increments
// dW ~ N(0, dt).  Every level draws fresh numbers (Sec. 5), and every sample must be
// reproducible from its index alone, so the generator is counter based: Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) maps
// (counter, key) to four 32-bit words with ten rounds of two 32x32->64 multiplies and xors.
// Box--Muller turns a pair of uniforms into a pair of independent N(0, 1) values.
#pragma once
#include <cstdint>

namespace mlmcgb {

// Philox4x32-10 round constants (SC'11): multipliers and the Weyl key increments.
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long pa = (unsigned long long)kPhiloxMulA * c.x;
        const unsigned long long pb = (unsigned long long)kPhiloxMulB * c.z;
        const uint32_t next_x = (uint32_t)(pb >> 32) ^ c.y ^ k0;
        const uint32_t next_z = (uint32_t)(pa >> 32) ^ c.w ^ k1;
        c = make_uint4(next_x, (uint32_t)pb, next_z, (uint32_t)pa);
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return c;
}

// The same function with the key schedule precomputed: rk[2 i], rk[2 i + 1] are the two key
// words of round i (k0 + i W_A, k1 + i W_B).  When rk lives in the kernel's parameter space the
// round keys are constant-bank operands of the xors and the per-round key additions vanish.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long pa = (unsigned long long)kPhiloxMulA * c.x;
        const unsigned long long pb = (unsigned long long)kPhiloxMulB * c.z;
        const uint32_t next_x = (uint32_t)(pb >> 32) ^ c.y ^ rk[2 * round];
        const uint32_t next_z = (uint32_t)(pa >> 32) ^ c.w ^ rk[2 * round + 1];
        c = make_uint4(next_x, (uint32_t)pb, next_z, (uint32_t)pa);
    }
    return c;
}

// Hardware approximations (the MUFU unit): log2, square root, sine and cosine.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One Box--Muller pair from two Philox words, returned as (rho, c, s) with the pair of
// normals z0 = rho * c, z1 = rho * s.  Callers fold rho into their next multiply.
template <typename R> struct BoxMuller;

// FP32 stream: u = 1 - (x mod 2^23) 2^-23 in (0, 1].  The float f = 1 + (x mod 2^23) 2^-23 is
// built by setting the exponent bits, u = 2 - f exactly.  With v = u2 - 1/2 = 3/2 - f2,
// cos(2 pi u2) = -cos(2 pi v) and sin(2 pi u2) = -sin(2 pi v) with 2 pi v in (-pi, pi], the
// range where the hardware sine and cosine are most accurate; the sign goes into rho.  The
// angle 2 pi v = 3 pi - 2 pi f2 is one fused multiply-add (absolute error below 5e-7, the size
// of the hardware sine's own error).
template <> struct BoxMuller<float> {
    __device__ __forceinline__ static void pair(uint32_t xa, uint32_t xb, float &rho, float &c,
                                                float &s, bool = false)
    {
        const float f1 = __uint_as_float((xa & 0x007FFFFFu) | 0x3F800000u);
        const float f2 = __uint_as_float((xb & 0x007FFFFFu) | 0x3F800000u);
        const float u1 = 2.0f - f1;
        // -2 ln u1 = -2 ln(2) log2(u1)
        rho = -sqrt_approx(-1.38629436111989061883f * lg2_approx(u1));
        const float theta = fmaf(-6.28318530717958647692f, f2, 9.42477796076937971538f);
        s = sin_approx(theta);
        c = cos_approx(theta);
    }
};

// The FP32 pair with rho / sqrt(2 ln 2) in place of rho: rho_s = -sqrt(-log2 u1), one multiply
// fewer.  Callers that multiply rho by a scale anyway use rho_s times (scale sqrt(2 ln 2)).
__device__ __forceinline__ void box_muller_lg2(uint32_t xa, uint32_t xb, float &rho_s, float &c, float &s)
{
    const float f1 = __uint_as_float((xa & 0x007FFFFFu) | 0x3F800000u);
    const float f2 = __uint_as_float((xb & 0x007FFFFFu) | 0x3F800000u);
    rho_s = -sqrt_approx(-lg2_approx(2.0f - f1));
    const float theta = fmaf(-6.28318530717958647692f, f2, 9.42477796076937971538f);
    s = sin_approx(theta);
    c = cos_approx(theta);
}
constexpr float kSqrt2Ln2 = 1.17741002251547469101f;  // sqrt(2 ln 2)

// FP64 stream: u = (x + 1) 2^-32 in (0, 1]; CUDA's double-precision log, sqrt and sincospi.
// With u23 set, the FP32 stream's uniforms u = 1 - (x mod 2^23) 2^-23 instead (the samples of
// the FP32 path, computed in FP64).
template <> struct BoxMuller<double> {
    __device__ __forceinline__ static void pair(uint32_t xa, uint32_t xb, double &rho,
                                                double &c, double &s, bool u23 = false)
    {
        const double u1 = u23 ? 1.0 - (double)(xa & 0x007FFFFFu) * 0x1p-23 : ((double)xa + 1.0) * 0x1p-32;
        const double u2 = u23 ? 1.0 - (double)(xb & 0x007FFFFFu) * 0x1p-23 : ((double)xb + 1.0) * 0x1p-32;
        rho = sqrt(-2.0 * log(u1));
        sincospi(2.0 * u2, &s, &c);
    }
};

}  // namespace mlmcgb
