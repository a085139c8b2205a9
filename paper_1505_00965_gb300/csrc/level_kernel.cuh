// level_kernel.cuh -- one level of multilevel Monte Carlo on the GPU (Sec. 5).
//
// For each sample s in [first, first + N) the kernel simulates, in registers, the fine
// Euler--Maruyama path of GBM with step h = T / M^l and the coarse path with step M h driven by
// sums of M consecutive fine increments (Sec. 2 Eq. em; Sec. 5 Eq. Yldef and Fig. 2), evaluates
// the payoff difference Y = P_l - P_{l-1} (Y = P_0 on level 0, Eq. mlmc:Yzero), and accumulates
// sum Y^k, k = 1..4, in FP64.  Warp shuffles and shared memory reduce each block to four
// doubles; the last block to finish adds the block partials in a fixed order, so the result
// does not depend on scheduling.
//
// GBM's Euler--Maruyama step is S_{n+1} = S_n (1 + d_n) with d_n = r h + sigma dW_n, so the step
// is written S <- fma(S, d, S) and the coarse factor is 1 + sum of the M fine d_n (their sum is
// r M h + sigma dW_coarse).  With lanes_per_path > 1 a sample's time steps are split into equal
// chunks, one per lane; every lane runs its chunk from the value 1, and a product scan over the
// lanes gives each chunk's true starting value (the recurrence is linear in S).
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "engine.h"
#include "rng.cuh"

namespace mlmcgb {

// Philox calls (4 fine steps each) per partial of the Asian running sums: a path's sum of its
// values adds in two levels, a partial over each group of 4 kSumGroup = 256 steps folded into the
// total at the group's end.  One accumulator over all M^l values of order one loses, in FP32, a
// relative 1e-5 of the average at 2^16 steps and 1e-3 to 1e-2 at 2^20 to 2^22 steps (each add
// rounds to the total's ulp); two levels keep it near 1e-6 up to 2^24 steps.  The kernels for
// lanes of more than kLongLaneSteps steps (template flag LONG, FP32 arithmetic-Asian kernels
// only) sum in two levels; shorter lanes, FP64 paths (whose adds round 2^29 times finer) and the
// other payoffs keep the single step loop, whose code the grouped one slows by 2-3 %.
constexpr int kSumGroup = 64;
// Samples per span of the one-thread-per-sample loop, walked with 32-bit offsets.
constexpr uint64_t kSpan32 = uint64_t(1) << 31;
template <typename R, int PAY> constexpr bool kBlockedSum = PAY == kAsian && sizeof(R) == 4;

// Running state of one path over the steps a lane simulates.  The step loops below keep these
// values in local scalars and store the struct once at the end: an FP64 build that updated the
// struct's members through a reference inside the loop lost the updates (every step restarted
// from the initial value), while the same arithmetic on local scalars is exact.
template <typename R, int PAY, bool SPLIT> struct PathAcc {
    R S;     // current value (relative to the chunk's start when SPLIT)
    R sum;   // sum of the values after each step (Asian)
    R hi;    // largest value seen, start included (lookback)
    R lo;    // smallest value seen (lookback, SPLIT only: a negative start flips max and min)
    R lsum;  // sum of log of the values after each step (geometric Asian test payoff)

    __device__ __forceinline__ void init(R x0)
    {
        S = x0;
        sum = R(0);
        hi = x0;
        lo = x0;
        lsum = R(0);
    }
    __device__ __forceinline__ static R log_r(R x)
    {
        return log(x);  // test payoff only: the accurate library logarithm
    }
};

// One Euler--Maruyama step of GBM, S <- S (1 + d), and the payoff's running functionals of
// the new value (on local scalars).
template <typename R, int PAY, bool SPLIT>
__device__ __forceinline__ void em_step(R &S, R &sum, R &hi, R &lo, R &lsum, R d)
{
    S = fma(S, d, S);
    if constexpr (PAY == kAsian) sum += S;
    if constexpr (PAY == kLookback) {
        hi = fmax(hi, S);
        if constexpr (SPLIT) lo = fmin(lo, S);
    }
    if constexpr (PAY == kGeoAsian) lsum += log(S);
}

// Separately rounded multiply, add and subtract, which the compiler may not fuse with a
// neighbouring operation.  The sample loops exist in several copies (with and without per-sample
// output, straight-line and looped), and floating-point contraction is decided per copy: the
// payoff, the quantities passed to it and the moment sums use these so that a sample's value
// and a launch's sums do not depend on the copy that computes them.
template <typename R> __device__ __forceinline__ R mul_rn(R a, R b)
{
    if constexpr (sizeof(R) == 4) return __fmul_rn(a, b);
    else return __dmul_rn(a, b);
}
template <typename R> __device__ __forceinline__ R add_rn(R a, R b)
{
    if constexpr (sizeof(R) == 4) return __fadd_rn(a, b);
    else return __dadd_rn(a, b);
}
template <typename R> __device__ __forceinline__ R sub_rn(R a, R b)
{
    if constexpr (sizeof(R) == 4) return __fsub_rn(a, b);
    else return __dsub_rn(a, b);
}
// The geometric Asian's log-sum argument n log S_0 + sum log(S_i / S_0).
template <typename R> __device__ __forceinline__ R lpost_of(R n, R logS0, R lsum)
{
    return add_rn(mul_rn(n, logS0), lsum);
}

// Discounted payoff of a path from its totals: final value Sn, sum of post-step values
// `post` (i = 1..n), maximum over S_0..S_n, sum of log post-step values; n = steps.  K, disc, S0
// and Q are the strike, discount factor, initial value and digital cash in the path's precision.
template <typename R, int PAY>
__device__ __forceinline__ R payoff_from(R Sn, R post, R hi, R lpost, R inv_n, R K, R disc, R S0, R Q)
{
    if constexpr (PAY == kEuropean) {
        return mul_rn(disc, fmax(sub_rn(Sn, K), R(0)));
    } else if constexpr (PAY == kAsian) {
        // (1/n) sum_{i<n} (S_i + S_{i+1}) / 2 = (1/n) (sum_{i=1..n} S_i + (S_0 - S_n) / 2)
        const R A = mul_rn(add_rn(post, mul_rn(R(0.5), sub_rn(S0, Sn))), inv_n);
        return mul_rn(disc, fmax(sub_rn(A, K), R(0)));
    } else if constexpr (PAY == kLookback) {
        return mul_rn(disc, fmax(sub_rn(hi, K), R(0)));
    } else if constexpr (PAY == kDigital) {
        return Sn > K ? mul_rn(disc, Q) : (Sn == K ? mul_rn(mul_rn(R(0.5), disc), Q) : R(0));
    } else if constexpr (PAY == kLinear) {
        return Sn;
    } else {  // kGeoAsian
        const R lg = mul_rn(add_rn(lpost, mul_rn(R(0.5), sub_rn(PathAcc<R, PAY, false>::log_r(S0),
                                                                PathAcc<R, PAY, false>::log_r(Sn)))),
                            inv_n);
        const R G = sizeof(R) == 4 ? R(expf(float(lg))) : R(exp(double(lg)));
        return mul_rn(disc, fmax(sub_rn(G, K), R(0)));
    }
}

template <typename R, int PAY>
__device__ __forceinline__ R payoff_value(R Sn, R post, R hi, R lpost, R inv_n, const LevelParams &p)
{
    return payoff_from<R, PAY>(Sn, post, hi, lpost, inv_n, R(p.K), R(p.disc), R(p.S0), R(p.Q));
}

// FP32 paths, European, arithmetic Asian and lookback calls: the payoff from the path relative to
// S0 (start value 1; primes below) as one or two fused multiply-adds and a max, with constants
// the host forms in FP64 (LevelParams::pay_*, kernel-parameter operands).  Since disc > 0,
// disc max(x, 0) = max(disc x, 0):
//   European  max(disc S0 S_n' - disc K, 0), lookback the same on the maximum;
//   Asian     max(disc S0 / n (sum' - S_n' / 2) + (disc S0 / (2 n) - disc K), 0), sum' over the
//             post-step values: (1/n) sum_{i<n} (S_i + S_{i+1}) / 2 written out as in payoff_from.
// The values equal payoff_from's in exact arithmetic and differ by FP32 rounding only.  Every
// one-thread-per-sample copy of the FP32 level kernels uses this form, so a sample's Y does not
// depend on the copy that computes it.
template <typename R, int PAY> constexpr bool kRelPayoff =
    sizeof(R) == 4 && (PAY == kEuropean || PAY == kAsian || PAY == kLookback);
template <int PAY>
__device__ __forceinline__ float rel_payoff(const LevelParams &p, bool coarse, float S, float sum, float hi)
{
    if constexpr (PAY == kEuropean) return fmaxf(fmaf(p.pay_dS0, S, p.pay_mdK), 0.f);
    else if constexpr (PAY == kLookback) return fmaxf(fmaf(p.pay_dS0, hi, p.pay_mdK), 0.f);
    else return fmaxf(fmaf(coarse ? p.pay_ac : p.pay_af, fmaf(-0.5f, S, sum), coarse ? p.pay_bc : p.pay_bf), 0.f);
}

// Payoff of one whole path relative to S0 (values S, sum, hi, log-sum ls after its n steps, 1/n =
// inv_n; `coarse` picks the coarse path): the relative form above where it exists, else
// payoff_value on the values times S0.
template <typename R, int PAY>
__device__ __forceinline__ R path_payoff(const LevelParams &p, bool coarse, R S, R sum, R hi, R ls, R S0, R logS0,
                                         R inv_n)
{
    if constexpr (kRelPayoff<R, PAY>) {
        return rel_payoff<PAY>(p, coarse, S, sum, hi);
    } else {
        const R n = coarse ? R(p.nf / p.M) : R(p.nf);
        return payoff_value<R, PAY>(S0 * S, S0 * sum, S0 * hi, lpost_of(n, logS0, ls), inv_n, p);
    }
}

// Philox block of counter c under the parameters' key: from the precomputed round keys (RK, the
// level kernels, whose parameters sit in the constant bank) or from the two key words (the
// batched kernel, whose parameters sit in global memory).
template <bool RK>
__device__ __forceinline__ uint4 philox_of(const LevelParams &p, uint4 c)
{
    if constexpr (RK) return philox4x32_10(c, p.rkey);
    else return philox4x32_10(c, p.key0, p.key1);
}

// Fine and coarse paths of one sample on a level with M^l >= 4 (one normal per fine step), over
// the Philox calls [j0, j1) (4 fine steps per call).  Euler--Maruyama: d = r h + sigma dW and the
// coarse factor's d is the sum of the M fine ones.  Milstein (MIL): d = r h + sigma dW
// + sigma^2 (dW^2 - h) / 2 = (r h - c2) + a z + c2 z^2 with a = sigma sqrt(h), c2 = sigma^2 h / 2,
// and the coarse step the same formula on the summed increment with step M h.
template <typename R, int MT, int PAY, bool SPLIT, bool MIL, bool RK = true, bool LONG = false, bool POS = false>
__device__ __forceinline__ void simulate_steps(const LevelParams &p, uint32_t slo, uint32_t shi,
                                               int j0, int j1, PathAcc<R, PAY, SPLIT> &fa,
                                               PathAcc<R, PAY, SPLIT> &ca)
{
    const R a = R(p.a), rh = R(p.rh);
    const R c2 = R(p.c2), rhm = R(p.rh - p.c2);
    R fS = fa.S, fsum = fa.sum, fhi = fa.hi, flo = fa.lo, fls = fa.lsum;
    R cS = ca.S, csum = ca.sum, chi = ca.hi, clo = ca.lo, cls = ca.lsum;
    R dc = R(0);
    int q = 0;
    const int M = MT ? MT : p.M;
    const R rHm = R(M * (p.rh - p.c2));
    const bool u23 = p.u23 != 0;
    const R a_s = R(p.a) * R(kSqrt2Ln2);  // FP32: sigma sqrt(h) sqrt(2 ln 2), for box_muller_lg2
    // one Philox call: four fine steps and the coarse steps they complete
    auto call = [&](int j) {
        const uint4 x = philox_of<RK>(p, make_uint4(p.ctr3, (uint32_t)j, shi, slo));
        R rho, c, s;
        R d[4];
        if constexpr (!MIL && sizeof(R) == 4) {
            box_muller_lg2(x.x, x.y, rho, c, s);
            R ra = rho * a_s;
            d[0] = fma(ra, c, rh);
            d[1] = fma(ra, s, rh);
            box_muller_lg2(x.z, x.w, rho, c, s);
            ra = rho * a_s;
            d[2] = fma(ra, c, rh);
            d[3] = fma(ra, s, rh);
        } else if constexpr (!MIL) {
            BoxMuller<R>::pair(x.x, x.y, rho, c, s, u23);
            R ra = rho * a;
            d[0] = fma(ra, c, rh);
            d[1] = fma(ra, s, rh);
            BoxMuller<R>::pair(x.z, x.w, rho, c, s, u23);
            ra = rho * a;
            d[2] = fma(ra, c, rh);
            d[3] = fma(ra, s, rh);
        } else {
            BoxMuller<R>::pair(x.x, x.y, rho, c, s, u23);
            d[0] = rho * c;  // here d holds the normals z until the steps below
            d[1] = rho * s;
            BoxMuller<R>::pair(x.z, x.w, rho, c, s, u23);
            d[2] = rho * c;
            d[3] = rho * s;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            R dk;
            // with M = 4 a call starts a coarse step: its sum starts from d[0] itself (the same
            // value as 0 + d[0] up to the sign of a zero, which no step can see)
            if constexpr (MIL) {
                dc = (MT == 4 && k == 0) ? d[k] : dc + d[k];  // the coarse increment's sum of normals
                dk = fma(fma(c2, d[k], a), d[k], rhm);
            } else {
                dk = d[k];
                dc = (MT == 4 && k == 0) ? dk : dc + dk;
            }
            em_step<R, PAY, SPLIT && !POS>(fS, fsum, fhi, flo, fls, dk);
            bool coarse_now;
            if constexpr (MT != 0) {
                coarse_now = (k + 1) % MT == 0;
            } else {
                coarse_now = ++q == M;
                if (coarse_now) q = 0;
            }
            if (coarse_now) {
                R dcs;
                if constexpr (MIL) dcs = fma(fma(c2, dc, a), dc, rHm);
                else dcs = dc;
                em_step<R, PAY, SPLIT && !POS>(cS, csum, chi, clo, cls, dcs);
                dc = R(0);
            }
        }
    };
    if constexpr (!(LONG && kBlockedSum<R, PAY>)) {
        for (int j = j0; j < j1; ++j) call(j);
    } else {
        R fsum_t = R(0), csum_t = R(0);  // totals of the finished groups
        for (int g = j0; g < j1; g += kSumGroup) {
            const int ge = min(g + kSumGroup, j1);
            for (int j = g; j < ge; ++j) call(j);
            fsum_t += fsum;
            csum_t += csum;
            fsum = csum = R(0);
        }
        fsum = fsum_t;
        csum = csum_t;
    }
    fa.S = fS; fa.sum = fsum; fa.hi = fhi; fa.lo = flo; fa.lsum = fls;
    ca.S = cS; ca.sum = csum; ca.hi = chi; ca.lo = clo; ca.lsum = cls;
}

// NS samples' fine and coarse paths in lockstep on a level with M^l >= 4, one thread per sample
// (no split): the samples' Philox chains and step chains are independent, so the scheduler can
// interleave them.  Each sample's arithmetic is the same as in simulate_steps.  States start at
// 1 (paths relative to S0).  CALLS, when nonzero, is the number of Philox calls per path known
// at compile time (1 on levels with M^l = 4: straight-line code).  ANTI adds the antithetic fine
// path (aS, asum, ahi, als): the same increments with each coarse step's M in reverse order
// (M = 4: a Philox block is one coarse step, read backwards; M = 2: its two pairs swapped).
template <typename R, int MT, int PAY, bool MIL, int NS, bool RK = true, int CALLS = 0, bool ANTI = false,
          bool LONG = false>
__device__ __forceinline__ void simulate_multi(const LevelParams &p, uint32_t s_hi, const uint32_t s_lo[NS], R fS[NS],
                                               R fsum[NS], R fhi[NS], R fls[NS], R cS[NS], R csum[NS],
                                               R chi[NS], R cls[NS], R aS[NS], R asum[NS], R ahi[NS],
                                               R als[NS])
{
    static_assert(!ANTI || MT == 4 || MT == 0, "antithetic paths for M = 4 (MT = 4) and M = 2 (MT = 0)");
    const R a = R(p.a), rh = R(p.rh);
    const R c2 = R(p.c2), rhm = R(p.rh - p.c2);
    const int M = MT ? MT : p.M;
    const R rHm = R(M * (p.rh - p.c2));
    const bool u23 = p.u23 != 0;
    const R a_s = R(p.a) * R(kSqrt2Ln2);  // FP32: sigma sqrt(h) sqrt(2 ln 2), for box_muller_lg2
    R flo[NS], clo[NS], alo[NS], dc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        fS[i] = cS[i] = R(1);
        fsum[i] = csum[i] = R(0);
        fhi[i] = chi[i] = flo[i] = clo[i] = R(1);
        fls[i] = cls[i] = R(0);
        dc[i] = R(0);
        if constexpr (ANTI) {
            aS[i] = ahi[i] = alo[i] = R(1);
            asum[i] = als[i] = R(0);
        }
    }
    int q = 0;
    const int calls = CALLS ? CALLS : p.nf >> 2;
    // one Philox call per sample: four fine steps and the coarse steps they complete
    auto call = [&](int j) {
        R d[NS][4];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const uint4 x = philox_of<RK>(p, make_uint4(p.ctr3, (uint32_t)j, s_hi, s_lo[i]));
            R rho, c, sn;
            if constexpr (!MIL && sizeof(R) == 4) {
                box_muller_lg2(x.x, x.y, rho, c, sn);
                R ra = rho * a_s;
                d[i][0] = fma(ra, c, rh);
                d[i][1] = fma(ra, sn, rh);
                box_muller_lg2(x.z, x.w, rho, c, sn);
                ra = rho * a_s;
                d[i][2] = fma(ra, c, rh);
                d[i][3] = fma(ra, sn, rh);
            } else {
                BoxMuller<R>::pair(x.x, x.y, rho, c, sn, u23);
                if constexpr (MIL) {
                    d[i][0] = rho * c;
                    d[i][1] = rho * sn;
                } else {
                    const R ra = rho * a;
                    d[i][0] = fma(ra, c, rh);
                    d[i][1] = fma(ra, sn, rh);
                }
                BoxMuller<R>::pair(x.z, x.w, rho, c, sn, u23);
                if constexpr (MIL) {
                    d[i][2] = rho * c;
                    d[i][3] = rho * sn;
                } else {
                    const R ra = rho * a;
                    d[i][2] = fma(ra, c, rh);
                    d[i][3] = fma(ra, sn, rh);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            bool coarse_now;
            if constexpr (MT != 0) {
                coarse_now = (k + 1) % MT == 0;
            } else {
                coarse_now = ++q == M;
                if (coarse_now) q = 0;
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                R dk;
                // M = 4: a call starts a coarse step, whose sum starts from d[i][0] (as in simulate_steps)
                if constexpr (MIL) {
                    dc[i] = (MT == 4 && k == 0) ? d[i][k] : dc[i] + d[i][k];
                    dk = fma(fma(c2, d[i][k], a), d[i][k], rhm);
                } else {
                    dk = d[i][k];
                    dc[i] = (MT == 4 && k == 0) ? dk : dc[i] + dk;
                }
                em_step<R, PAY, false>(fS[i], fsum[i], fhi[i], flo[i], fls[i], dk);
                if constexpr (ANTI) {
                    const int ka = MT == 4 ? 3 - k : (k ^ 1);
                    R da;
                    if constexpr (MIL) da = fma(fma(c2, d[i][ka], a), d[i][ka], rhm);
                    else da = d[i][ka];
                    em_step<R, PAY, false>(aS[i], asum[i], ahi[i], alo[i], als[i], da);
                }
                if (coarse_now) {
                    R dcs;
                    if constexpr (MIL) dcs = fma(fma(c2, dc[i], a), dc[i], rHm);
                    else dcs = dc[i];
                    em_step<R, PAY, false>(cS[i], csum[i], chi[i], clo[i], cls[i], dcs);
                    dc[i] = R(0);
                }
            }
        }
    };
    if constexpr (!(LONG && kBlockedSum<R, PAY>)) {
        if constexpr (CALLS == 0) {
            // two calls per iteration: the arithmetic-Asian kernel otherwise waited on its MUFU
            // results (short-scoreboard stalls 0.21 per issue against 0.04 in the split form) and
            // ran 5 % slower than its split form.  The lookback kernel ran slower unrolled until
            // the counter layout left 16 loop-variant multiplies per block; with it, unrolled
            // runs 4 % faster (1.229 -> 1.280e12 steps/s at level 6 over whole waves)
#pragma unroll 2
            for (int j = 0; j < calls; ++j) call(j);
        } else {
            for (int j = 0; j < calls; ++j) call(j);
        }
    } else {
        R fsum_t[NS], csum_t[NS], asum_t[NS];  // totals of the finished groups
#pragma unroll
        for (int i = 0; i < NS; ++i) fsum_t[i] = csum_t[i] = asum_t[i] = R(0);
        for (int g = 0; g < calls; g += kSumGroup) {
            const int ge = min(g + kSumGroup, calls);
            for (int j = g; j < ge; ++j) call(j);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                fsum_t[i] += fsum[i];
                csum_t[i] += csum[i];
                fsum[i] = csum[i] = R(0);
                if constexpr (ANTI) {
                    asum_t[i] += asum[i];
                    asum[i] = R(0);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            fsum[i] = fsum_t[i];
            csum[i] = csum_t[i];
            if constexpr (ANTI) asum[i] = asum_t[i];
        }
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum four doubles over the block; the result is valid in thread 0.
__device__ __forceinline__ void block_sum4(double v[4])
{
    __shared__ double sm[32][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();  // sm may still be read by an earlier call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sm[warp][k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = warp_sum(lane < nw ? sm[lane][k] : 0.0);
    }
}

// Block partials -> workspace; the last block adds them in block order and writes p.out.
__device__ __forceinline__ void finish_sums(double m[4], const LevelParams &p)
{
    __shared__ bool is_last;
    block_sum4(m);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) p.partials[4 * blockIdx.x + k] = m[k];
        __threadfence();
        const unsigned done = atomicAdd(p.ticket, 1u);
        is_last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += __ldcg(p.partials + 4 * b + k);
    }
    block_sum4(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) p.out[k] = acc[k];
        *p.ticket = 0u;  // leave the workspace ready for the next launch
    }
}

// Add Y, Y^2, Y^3, Y^4 of one sample.  FP64 paths add into the FP64 sums m directly.  FP32
// paths sum a batch of at most 32 samples in FP32 (b1..b4, nb counts the batch) and add each
// batch into m, which keeps FP64 off the per-sample path.
__device__ __forceinline__ void batch_add(float Y, float &b1, float &b2, float &b3, float &b4)
{
    const float y2 = __fmul_rn(Y, Y);
    b1 = __fadd_rn(b1, Y);
    b2 = __fadd_rn(b2, y2);
    b3 = fmaf(y2, Y, b3);
    b4 = fmaf(y2, y2, b4);
}
__device__ __forceinline__ void fold_batch_now(double m[4], float &b1, float &b2, float &b3, float &b4, int &nb)
{
    m[0] += b1; m[1] += b2; m[2] += b3; m[3] += b4;
    b1 = b2 = b3 = b4 = 0.f;
    nb = 0;
}
__device__ __forceinline__ void add_moments(float Y, double m[4], float &b1, float &b2, float &b3,
                                            float &b4, int &nb)
{
    batch_add(Y, b1, b2, b3, b4);
    if (++nb == 32) fold_batch_now(m, b1, b2, b3, b4, nb);
}
// Four samples at once (the batch never exceeds 32).
__device__ __forceinline__ void add_moments4(const float Y[4], double m[4], float &b1, float &b2,
                                             float &b3, float &b4, int &nb)
{
    if (nb > 28) fold_batch_now(m, b1, b2, b3, b4, nb);
#pragma unroll
    for (int k = 0; k < 4; ++k) batch_add(Y[k], b1, b2, b3, b4);
    nb += 4;
}
__device__ __forceinline__ void add_moments(double Y, double m[4], float &, float &, float &,
                                            float &, int &)
{
    const double y2 = __dmul_rn(Y, Y);
    m[0] = __dadd_rn(m[0], Y);
    m[1] = __dadd_rn(m[1], y2);
    m[2] = fma(y2, Y, m[2]);
    m[3] = fma(y2, y2, m[3]);
}
__device__ __forceinline__ void add_moments4(const double Y[4], double m[4], float &b1, float &b2,
                                             float &b3, float &b4, int &nb)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) add_moments(Y[k], m, b1, b2, b3, b4, nb);
}

// Join the chunks of one sample split over P lanes: an exclusive product scan of the chunk
// factors gives each chunk's starting value relative to S0; the path totals are then sums and
// maxima over the lanes.  Every lane of the group receives the totals.
template <typename R, int PAY, bool POS = false>
__device__ __forceinline__ void join_chunks(const PathAcc<R, PAY, true> &A, int lig, int P, R S0,
                                            R steps, R &total, R &post, R &hi, R &lpost)
{
    R incl = A.S;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        if (o < P) {
            const R t = __shfl_up_sync(0xffffffffu, incl, o, P);
            if (lig >= o) incl *= t;
        }
    }
    R excl = __shfl_up_sync(0xffffffffu, incl, 1, P);
    if (lig == 0) excl = R(1);
    total = S0 * __shfl_sync(0xffffffffu, incl, P - 1, P);
    const R start = S0 * excl;
    R ps = start * A.sum;
    R ph = (POS || start >= R(0)) ? start * A.hi : start * A.lo;  // POS: every start is positive
    R pl = R(0);
    if constexpr (PAY == kGeoAsian) pl = steps * PathAcc<R, PAY, true>::log_r(start) + A.lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (o < P) {
            ps += __shfl_xor_sync(0xffffffffu, ps, o, P);
            ph = fmax(ph, __shfl_xor_sync(0xffffffffu, ph, o, P));
            if constexpr (PAY == kGeoAsian) pl += __shfl_xor_sync(0xffffffffu, pl, o, P);
        }
    }
    post = ps;
    hi = ph;
    lpost = pl;
}

// Y of sample s on a level with M^l >= 4, computed by the P lanes of one group (lane lig);
// every lane of the group returns the same Y.
template <typename R, int MT, int PAY, bool SPLIT, bool MIL, bool RK = true, bool LONG = false, bool POS = false>
__device__ __forceinline__ R sample_Y(const LevelParams &p, uint64_t s, int lig, int P)
{
    const uint32_t slo = (uint32_t)s, shi = (uint32_t)(s >> 32);
    const R S0 = R(p.S0);
    const R inv_nf = R(p.inv_nf), inv_nc = R(p.inv_nc);
    // Paths run relative to S0 (start value 1) and are scaled once per sample: the running sums
    // then hold values of order one, which keeps the FP32 sums of many steps accurate.
    PathAcc<R, PAY, SPLIT> fa, ca;
    fa.init(R(1));
    ca.init(R(1));
    if constexpr (!SPLIT) {
        simulate_steps<R, MT, PAY, false, MIL, RK, LONG>(p, slo, shi, 0, p.nf >> 2, fa, ca);
        const R logS0 = PAY == kGeoAsian ? PathAcc<R, PAY, false>::log_r(S0) : R(0);
        const R Pf = path_payoff<R, PAY>(p, false, fa.S, fa.sum, fa.hi, fa.lsum, S0, logS0, inv_nf);
        if (p.fine_only) return Pf;
        const R Pc = path_payoff<R, PAY>(p, true, ca.S, ca.sum, ca.hi, ca.lsum, S0, logS0, inv_nc);
        return Pf - Pc;
    } else {
        const int calls = (p.nf >> 2) / P;
        simulate_steps<R, MT, PAY, true, MIL, RK, LONG, POS>(p, slo, shi, lig * calls, (lig + 1) * calls, fa, ca);
        const R steps_f = R(4 * calls);
        R tf, pf, hf, lf, tc, pc, hc, lc;
        join_chunks<R, PAY, POS>(fa, lig, P, S0, steps_f, tf, pf, hf, lf);
        join_chunks<R, PAY, POS>(ca, lig, P, S0, steps_f / R(p.M), tc, pc, hc, lc);
        const R Pf = payoff_value<R, PAY>(tf, pf, hf, lf, inv_nf, p);
        if (p.fine_only) return Pf;
        const R Pc = payoff_value<R, PAY>(tc, pc, hc, lc, inv_nc, p);
        return Pf - Pc;
    }
}

// NS samples of one span run in lockstep: offsets i0, i0 + T, ... below n (the first always is),
// sample indices (s_hi, lo0 + offset); moments go into m / b1..b4 / nb and Y into y_out[c0 + offset].
template <typename R, int MT, int PAY, bool MIL, int NS, bool RK, int CALLS, bool ANTI, bool LONG>
__device__ __forceinline__ void multi_samples(const LevelParams &p, uint32_t s_hi, uint32_t lo0, uint32_t i0,
                                              uint32_t T32, uint32_t n, uint64_t c0, R S0, R inv_nf, R inv_nc,
                                              R logS0, double m[4], float &b1, float &b2, float &b3,
                                              float &b4, int &nb, double *y_out)
{
    uint32_t s_lo[NS];
    bool valid[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const uint32_t j = i0 + (uint32_t)i * T32;
        valid[i] = i == 0 || j < n;
        s_lo[i] = lo0 + (valid[i] ? j : i0);  // below 2^32: the span stops at the boundary
    }
    R fS[NS], fsum[NS], fhi[NS], fls[NS], cS[NS], csum[NS], chi[NS], cls[NS];
    R aS[NS], asum[NS], ahi[NS], als[NS];
    simulate_multi<R, MT, PAY, MIL, NS, RK, CALLS, ANTI, LONG>(p, s_hi, s_lo, fS, fsum, fhi, fls, cS, csum, chi, cls,
                                                               aS, asum, ahi, als);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        R Pf = path_payoff<R, PAY>(p, false, fS[i], fsum[i], fhi[i], fls[i], S0, logS0, inv_nf);
        if constexpr (ANTI)
            Pf = mul_rn(R(0.5), add_rn(Pf, path_payoff<R, PAY>(p, false, aS[i], asum[i], ahi[i], als[i], S0,
                                                                logS0, inv_nf)));
        R Y = Pf;
        if (!p.fine_only) Y -= path_payoff<R, PAY>(p, true, cS[i], csum[i], chi[i], cls[i], S0, logS0, inv_nc);
        if (valid[i]) {
            if (y_out) y_out[c0 + i0 + (uint32_t)i * T32] = (double)Y;
            add_moments(Y, m, b1, b2, b3, b4, nb);
        }
    }
}

// One thread per sample over the samples [first, first + N) (the arguments as for regular_range
// below): thread t takes the offsets t, t + T, t + 2T, ... of each span, NS of them per iteration.
// With NS = 2 a thread whose last offset has no partner runs it alone, so every thread takes the
// same samples as with NS = 1 and the grid is the same; only the pairing differs.
template <typename R, int MT, int PAY, bool MIL, int NS, bool RK = true, int CALLS = 0, bool ANTI = false,
          bool LONG = false>
__device__ __forceinline__ void multi_range(const LevelParams &p, uint64_t first, uint64_t N, uint64_t t,
                                            uint64_t T, double m[4], float &b1, float &b2, float &b3,
                                            float &b4, int &nb, double *y_out)
{
    static_assert(NS == 1 || NS == 2, "one or two samples per thread");
    const R S0 = R(p.S0), inv_nf = R(p.inv_nf), inv_nc = R(p.inv_nc);
    const R logS0 = PAY == kGeoAsian ? PathAcc<R, PAY, false>::log_r(S0) : R(0);
    // The range in spans of at most 2^31 samples that stay inside one 2^32-aligned block of sample
    // indices, each walked with 32-bit offsets (threads leave the loop independently: nothing in it
    // synchronises the warp).  The sample index's high word is then the same for the whole span,
    // so the Philox products of that counter word are formed once per span, not once per sample.
    // With 64-bit offsets and a warp-uniform exit the loop control took about 25 of the 126
    // instructions of a sample on levels with M^l = 4.
    const uint32_t t32 = (uint32_t)t, T32 = (uint32_t)T;
    for (uint64_t c0 = 0; c0 < N;) {
        const uint64_t start = first + c0;
        const uint64_t room = (uint64_t(1) << 32) - (uint32_t)start;  // samples left below the next 2^32 boundary
        const uint64_t left = N - c0 < kSpan32 ? N - c0 : kSpan32;
        const uint32_t n = (uint32_t)(left < room ? left : room);  // c0 + n <= N
        const uint32_t s_hi = (uint32_t)(start >> 32), lo0 = (uint32_t)start;
        uint32_t i0 = t32;
        if constexpr (NS == 2) {
            // i0 < n <= 2^31 and T32 < 2^31, so i0 + T32 does not wrap
            for (; i0 < n && n - i0 > T32; i0 += 2 * T32)
                multi_samples<R, MT, PAY, MIL, 2, RK, CALLS, ANTI, LONG>(p, s_hi, lo0, i0, T32, n, c0, S0, inv_nf,
                                                                         inv_nc, logS0, m, b1, b2, b3, b4, nb, y_out);
            if (i0 < n)
                multi_samples<R, MT, PAY, MIL, 1, RK, CALLS, ANTI, LONG>(p, s_hi, lo0, i0, T32, n, c0, S0, inv_nf,
                                                                         inv_nc, logS0, m, b1, b2, b3, b4, nb, y_out);
        } else {
            for (; i0 < n; i0 += T32)
                multi_samples<R, MT, PAY, MIL, 1, RK, CALLS, ANTI, LONG>(p, s_hi, lo0, i0, T32, n, c0, S0, inv_nf,
                                                                         inv_nc, logS0, m, b1, b2, b3, b4, nb, y_out);
        }
        c0 += n;
    }
}

// Samples [first, first + N) of a level with M^l >= 4, shared by T threads of which this is
// thread t (T a multiple of 32).  Whole paths: one thread per sample (multi_range).  Split paths:
// groups of P = p.lanes lanes take one sample each, and since the lanes of a group join by
// shuffles, t and T count whole warps and the loop exits are warp uniform.  Moments go into
// m / b1..b4 / nb, and Y of sample first + i into y_out[i] when y_out is not NULL.
template <typename R, int MT, int PAY, bool SPLIT, bool MIL, bool RK = true, bool ANTI = false,
          bool LONG = false, bool POS = false>
__device__ __forceinline__ void regular_range(const LevelParams &p, uint64_t first, uint64_t N,
                                              uint64_t t, uint64_t T, double m[4], float &b1,
                                              float &b2, float &b3, float &b4, int &nb,
                                              double *y_out)
{
    if constexpr (!SPLIT) {
        // one sample per thread and iteration; a sample of a level with M^l = 4 is a single
        // Philox block and runs as straight-line code, in two copies (with and without
        // per-sample output) so that the output test leaves its loop
        if (p.nf == 4) {
            if (y_out)
                multi_range<R, MT, PAY, MIL, 1, RK, 1, ANTI, LONG>(p, first, N, t, T, m, b1, b2, b3, b4, nb, y_out);
            else
                multi_range<R, MT, PAY, MIL, 1, RK, 1, ANTI, LONG>(p, first, N, t, T, m, b1, b2, b3, b4, nb, nullptr);
        } else
            multi_range<R, MT, PAY, MIL, 1, RK, 0, ANTI, LONG>(p, first, N, t, T, m, b1, b2, b3, b4, nb, y_out);
    } else {
        static_assert(!ANTI, "antithetic paths run one thread per sample");
        const int P = p.lanes;
        const uint64_t groups = T / P;
        const uint64_t g = t / P;
        const uint64_t g_warp = (t & ~uint64_t(31)) / P;  // first group of this warp
        const int lig = (int)(t % P);
        for (uint64_t base = 0; base + g_warp < N; base += groups) {
            const uint64_t idx = base + g;
            const bool valid = idx < N;
            const uint64_t s = first + (valid ? idx : N - 1);
            const R Y = sample_Y<R, MT, PAY, true, MIL, RK, LONG, POS>(p, s, lig, P);
            if (valid && lig == 0) {
                if (y_out) y_out[idx] = (double)Y;
                add_moments(Y, m, b1, b2, b3, b4, nb);
            }
        }
    }
}

// The four normals z of Philox block q = (q_hi, q_lo) of a level with M^l < 4 and their step
// increments d.
template <typename R, bool MIL, bool RK = true>
__device__ __forceinline__ void block_increments(const LevelParams &p, uint32_t q_hi, uint32_t q_lo, R z[4], R d[4])
{
    const R a = R(p.a), rh = R(p.rh), c2 = R(p.c2), rhm = R(p.rh - p.c2);
    const bool u23 = p.u23 != 0;
    const uint4 x = philox_of<RK>(p, make_uint4(p.ctr3, 0u, q_hi, q_lo));
    R rho, c, s;
    if constexpr (!MIL && sizeof(R) == 4) {
        // FP32 Euler--Maruyama needs the increments only (z is left unset)
        const R a_s = a * R(kSqrt2Ln2);
        box_muller_lg2(x.x, x.y, rho, c, s);
        R ra = rho * a_s;
        d[0] = fma(ra, c, rh);
        d[1] = fma(ra, s, rh);
        box_muller_lg2(x.z, x.w, rho, c, s);
        ra = rho * a_s;
        d[2] = fma(ra, c, rh);
        d[3] = fma(ra, s, rh);
        return;
    }
    BoxMuller<R>::pair(x.x, x.y, rho, c, s, u23);
    z[0] = rho * c;
    z[1] = rho * s;
    BoxMuller<R>::pair(x.z, x.w, rho, c, s, u23);
    z[2] = rho * c;
    z[3] = rho * s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if constexpr (MIL) d[k] = fma(fma(c2, z[k], a), z[k], rhm);
        else d[k] = fma(a, z[k], rh);
    }
}

// Level 0 of the FP32 path, one Euler step S_1 = S_0 (1 + d), for the payoffs whose value is
// affine in d up to a max: the discounted payoff in two or three operations, its constants
// formed in FP64 (disc S_0, disc S_0 / 2, disc (S_0 - K)).  The same value as payoff_value on the
// one-step path in exact arithmetic: European disc (S_1 - K)^+; arithmetic Asian (trapezoid,
// n = 1) A = (S_0 + S_1) / 2 = S_0 (1 + d / 2); lookback max(S_0, S_1) = S_0 (1 + max(d, 0)).
template <int PAY> constexpr bool kLevel0Affine = PAY == kEuropean || PAY == kAsian || PAY == kLookback;
struct Level0Consts {
    float dS0, half_dS0, dS0mK, dS0mK_pos;  // dS0mK_pos = max(dS0mK, 0)
};
__device__ __forceinline__ Level0Consts level0_consts(const LevelParams &p)
{
    const float dS0mK = (float)(p.disc * (p.S0 - p.K));
    return {(float)(p.disc * p.S0), (float)(0.5 * p.disc * p.S0), dS0mK, fmaxf(dS0mK, 0.f)};
}
// Lookback: max(fma(max(d, 0), dS0, dS0mK), 0) = max(fma(d, dS0, dS0mK), max(dS0mK, 0)) exactly,
// since dS0 > 0: for d > 0 the fma rounds to at least dS0mK, and for d <= 0 it rounds to at most
// dS0mK (equal at d = -0), so both forms give the same float.  One multiply-add and one max.
template <int PAY>
__device__ __forceinline__ float level0_payoff(float d, const Level0Consts &c)
{
    if constexpr (PAY == kEuropean) return fmaxf(fmaf(d, c.dS0, c.dS0mK), 0.f);
    else if constexpr (PAY == kAsian) return fmaxf(fmaf(d, c.half_dS0, c.dS0mK), 0.f);
    else return fmaxf(fmaf(d, c.dS0, c.dS0mK), c.dS0mK_pos);
}

// The samples of Philox block q (slots r = 0 .. G - 1, sample q G + r) that lie in
// [first, end), from the block's normals z and increments d.
template <typename R, int PAY, bool MIL>
__device__ __forceinline__ void small_block(const LevelParams &p, uint64_t q, uint64_t first, uint64_t end,
                                            const R z[4], const R d[4], double m[4], float &b1, float &b2,
                                            float &b3, float &b4, int &nb, double *y_out)
{
    const int nf = p.nf;
    const uint32_t G = 4u / (uint32_t)nf;
    const R a = R(p.a), S0 = R(p.S0), c2 = R(p.c2), rhm = R(p.rh - p.c2);
    const R inv_nf = R(p.inv_nf), inv_nc = R(p.inv_nc);
    const R logS0 = PAY == kGeoAsian ? log(S0) : R(0);
    if (nf == 1 && q * 4 >= first && end - q * 4 >= 4) {
        // four whole level-0 samples: no per-sample range checks, moments added together (the
        // test avoids q * 4 + 4, which wraps to 0 for the last block below 2^64)
        R Y[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if constexpr (sizeof(R) == 4 && kLevel0Affine<PAY> && !MIL) {
                Y[r] = level0_payoff<PAY>(d[r], level0_consts(p));
            } else {
                R fS = R(1), fsum = R(0), fhi = R(1), flo = R(1), fls = R(0);
                em_step<R, PAY, false>(fS, fsum, fhi, flo, fls, d[r]);
                Y[r] = payoff_value<R, PAY>(S0 * fS, S0 * fsum, S0 * fhi, logS0 + fls, inv_nf, p);
            }
            if (y_out) y_out[q * 4 + r - first] = (double)Y[r];
        }
        add_moments4(Y, m, b1, b2, b3, b4, nb);
        return;
    }
#pragma unroll
    for (uint32_t r = 0; r < 4; ++r) {
        if (r >= G) break;
        const uint64_t sample = q * G + r;
        if (sample < first || sample >= end) continue;
        R fS = R(1), fsum = R(0), fhi = R(1), flo = R(1), fls = R(0);
        R cS = R(1), csum = R(0), chi = R(1), clo = R(1), cls = R(0);
        R Y;
        if (nf == 1) {
            if constexpr (sizeof(R) == 4 && kLevel0Affine<PAY> && !MIL) {
                Y = level0_payoff<PAY>(d[r], level0_consts(p));
            } else {
                em_step<R, PAY, false>(fS, fsum, fhi, flo, fls, d[r]);
                Y = payoff_value<R, PAY>(S0 * fS, S0 * fsum, S0 * fhi, logS0 + fls, inv_nf, p);
            }
        } else {  // nf == 2, level 1 with M = 2: two fine steps, one coarse step
            const R d0 = d[2 * (r & 1)], d1 = d[2 * (r & 1) + 1];
            em_step<R, PAY, false>(fS, fsum, fhi, flo, fls, d0);
            em_step<R, PAY, false>(fS, fsum, fhi, flo, fls, d1);
            R dcs;
            if constexpr (MIL) {
                const R zc = z[2 * (r & 1)] + z[2 * (r & 1) + 1];
                dcs = fma(fma(c2, zc, a), zc, R(2) * rhm);
            } else {
                dcs = d0 + d1;
            }
            em_step<R, PAY, false>(cS, csum, chi, clo, cls, dcs);
            R Pf = payoff_value<R, PAY>(S0 * fS, S0 * fsum, S0 * fhi, lpost_of(R(2), logS0, fls), inv_nf, p);
            if (p.antithetic) {
                // the antithetic fine path: the coarse step's two increments swapped
                R aS = R(1), asum = R(0), ahi = R(1), alo = R(1), als = R(0);
                em_step<R, PAY, false>(aS, asum, ahi, alo, als, d1);
                em_step<R, PAY, false>(aS, asum, ahi, alo, als, d0);
                Pf = mul_rn(R(0.5), add_rn(Pf, payoff_value<R, PAY>(S0 * aS, S0 * asum, S0 * ahi, lpost_of(R(2), logS0, als),
                                                         inv_nf, p)));
            }
            if (p.fine_only) {
                Y = Pf;
            } else {
                const R Pc = payoff_value<R, PAY>(S0 * cS, S0 * csum, S0 * chi, logS0 + cls, inv_nc, p);
                Y = Pf - Pc;
            }
        }
        if (y_out) y_out[sample - first] = (double)Y;
        add_moments(Y, m, b1, b2, b3, b4, nb);
    }
}

// Samples [first, first + N) of a level with M^l < 4.  G = 4 / M^l consecutive samples share
// one Philox block: thread t takes blocks q = first / G + t, + T, ... and the G samples
// q G .. q G + G - 1 that fall in the range; sample slot r takes normals r M^l .. of the block.
template <typename R, int PAY, bool MIL, bool RK = true>
__device__ __forceinline__ void small_range(const LevelParams &p, uint64_t first, uint64_t N,
                                            uint64_t t, uint64_t T, double m[4], float &b1,
                                            float &b2, float &b3, float &b4, int &nb,
                                            double *y_out)
{
    const uint32_t G = 4u / (uint32_t)p.nf;
    const uint64_t end = first + N;
    const uint64_t q0 = first / G;
    const uint64_t nq = (end - 1) / G - q0 + 1;
    if (p.nf != 1) {
        for (uint64_t u = t; u < nq; u += T) {
            R z[4], d[4];
            const uint64_t q = q0 + u;
            block_increments<R, MIL, RK>(p, (uint32_t)(q >> 32), (uint32_t)q, z, d);
            small_block<R, PAY, MIL>(p, q0 + u, first, end, z, d, m, b1, b2, b3, b4, nb, y_out);
        }
        return;
    }
    // level 0: the blocks [qa, qb) hold four samples of the range each and run without range
    // checks; the first and last block of the range, when only partly inside, follow (qa rounds
    // first / 4 up without forming first + 3, which wraps for ranges at the top of 64 bits)
    const uint64_t qa = first / 4 + ((first & 3) != 0), qb = end / 4;
    const R S0 = R(p.S0), inv_nf = R(p.inv_nf);
    const R logS0 = PAY == kGeoAsian ? log(S0) : R(0);
    const Level0Consts c0 = level0_consts(p);
    // two copies of the loop, with and without per-sample output, keep the output test out of it;
    // the blocks go in spans inside one 2^32-aligned run of block indices, so the counter's high
    // word and its Philox products stay fixed over a span.  Thread t takes blocks t, t + T, ... of
    // a span; on the FP32 one-step payoffs two at a time (two independent Philox chains for the
    // scheduler: 1.3-1.9 % faster at 4e8 samples), and an unpaired last block alone.
    constexpr bool kPairBlocks = sizeof(R) == 4 && kLevel0Affine<PAY> && !MIL;
    auto whole_blocks = [&](auto with_output) {
        for (uint64_t qs = qa; qs < qb;) {
            const uint64_t room = (uint64_t(1) << 32) - (uint32_t)qs;
            const uint64_t len = qb - qs < room ? qb - qs : room;
            const uint32_t q_hi = (uint32_t)(qs >> 32), lo0 = (uint32_t)qs;
            // the four samples of block lo0 + u (below 2^32: the span stops at the boundary)
            auto block_Y = [&](uint64_t u, R Y[4]) {
                R z[4], d[4];
                block_increments<R, MIL, RK>(p, q_hi, lo0 + (uint32_t)u, z, d);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if constexpr (sizeof(R) == 4 && kLevel0Affine<PAY> && !MIL) {
                        Y[r] = level0_payoff<PAY>(d[r], c0);
                    } else {
                        R fS = R(1), fsum = R(0), fhi = R(1), flo = R(1), fls = R(0);
                        em_step<R, PAY, false>(fS, fsum, fhi, flo, fls, d[r]);
                        Y[r] = payoff_value<R, PAY>(S0 * fS, S0 * fsum, S0 * fhi, logS0 + fls, inv_nf, p);
                    }
                }
            };
            auto emit = [&](uint64_t u, const R Y[4]) {
                if constexpr (decltype(with_output)::value) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) y_out[(qs + u) * 4 + r - first] = (double)Y[r];
                }
                add_moments4(Y, m, b1, b2, b3, b4, nb);
            };
            uint64_t u = t;
            if constexpr (kPairBlocks) {
                for (; u + T < len; u += 2 * T) {  // len <= 2^32 and T < 2^31: no wrap
                    R Ya[4], Yb[4];
                    block_Y(u, Ya);
                    block_Y(u + T, Yb);
                    emit(u, Ya);
                    emit(u + T, Yb);
                }
            }
            for (; u < len; u += T) {
                R Y[4];
                block_Y(u, Y);
                emit(u, Y);
            }
            qs += len;
        }
    };
    if (y_out) whole_blocks(std::true_type{});
    else whole_blocks(std::false_type{});
    const uint64_t qlast = (end - 1) / 4;
    const bool first_partial = q0 < qa || q0 >= qb;
    const bool last_partial = qlast != q0 && qlast >= qb;
    if ((t == 0 && first_partial) || (t == 1 && last_partial)) {
        const uint64_t q = t == 0 ? q0 : qlast;
        R z[4], d[4];
        block_increments<R, MIL, RK>(p, (uint32_t)(q >> 32), (uint32_t)q, z, d);
        small_block<R, PAY, MIL>(p, q, first, end, z, d, m, b1, b2, b3, b4, nb, y_out);
    }
}

template <typename R>
__device__ __forceinline__ void fold_batch(double m[4], float b1, float b2, float b3, float b4)
{
    if constexpr (sizeof(R) == 4) {
        m[0] += b1; m[1] += b2; m[2] += b3; m[3] += b4;
    }
}

// One level, one thread (or P lanes) per sample, grid-stride over the samples; ANTI: the
// antithetic estimator Y = (P_f + P_f^a) / 2 - P_c (one thread per sample); LONG: lanes of more
// than kLongLaneSteps steps (two-level Asian sums); POS: split paths whose step factors 1 + d are
// all positive (the host checks the bound of the normals), so that no chunk starts below zero
// and the lookback lanes keep no running minimum.
template <typename R, int MT, int PAY, bool SPLIT, bool MIL, bool ANTI = false, bool LONG = false, bool POS = false>
__global__ void __launch_bounds__(1024) level_kernel(const LevelParams p)
{
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f;  // FP32-path batch sums
    int nb = 0;
    regular_range<R, MT, PAY, SPLIT, MIL, true, ANTI, LONG, POS>(p, p.first, p.N, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                     (uint64_t)gridDim.x * blockDim.x, m, b1, b2, b3, b4, nb, p.y_out);
    fold_batch<R>(m, b1, b2, b3, b4);
    finish_sums(m, p);
}

// Two samples per thread and iteration, one thread per sample (no split, no antithetic path): the
// two samples' Philox and step chains are independent, so each scheduler has twice the
// instruction-level parallelism per warp, at more registers (64 against 54).  A kernel of its own
// (not a runtime branch of level_kernel) so that the one-sample kernels keep their register count;
// at most 512 threads per block, which lets it hold up to 128 registers.
template <typename R, int MT, int PAY, bool LONG = false>
__global__ void __launch_bounds__(512) level_ns2_kernel(const LevelParams p)
{
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f;
    int nb = 0;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, T = (uint64_t)gridDim.x * blockDim.x;
    if (p.nf == 4) {
        if (p.y_out)
            multi_range<R, MT, PAY, false, 2, true, 1, false, LONG>(p, p.first, p.N, t, T, m, b1, b2, b3, b4, nb, p.y_out);
        else
            multi_range<R, MT, PAY, false, 2, true, 1, false, LONG>(p, p.first, p.N, t, T, m, b1, b2, b3, b4, nb, nullptr);
    } else {
        multi_range<R, MT, PAY, false, 2, true, 0, false, LONG>(p, p.first, p.N, t, T, m, b1, b2, b3, b4, nb, p.y_out);
    }
    fold_batch<R>(m, b1, b2, b3, b4);
    finish_sums(m, p);
}

// Levels with M^l < 4 (level 0, and level 1 when M = 2).
template <typename R, int PAY, bool MIL>
__global__ void __launch_bounds__(1024) level_small_kernel(const LevelParams p)
{
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f;
    int nb = 0;
    small_range<R, PAY, MIL>(p, p.first, p.N, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                        (uint64_t)gridDim.x * blockDim.x, m, b1, b2, b3, b4, nb, p.y_out);
    fold_batch<R>(m, b1, b2, b3, b4);
    finish_sums(m, p);
}

// ------------------------------------------------------------------ batched rounds

// All samples of one chunk, by the threads of one block, on the code path of the chunk's task.
// Y of sample first + i goes to y[i] when the task has per-sample output (p.y_out, indexed from
// the task's first sample; NULL in the adaptive driver's rounds).
template <typename R, int MT>
__device__ __forceinline__ void batch_chunk(const LevelParams &p, uint64_t first, uint64_t count,
                                            double m[4], float &b1, float &b2, float &b3, float &b4,
                                            int &nb)
{
    const uint64_t t = threadIdx.x, T = blockDim.x;
    double *y = p.y_out ? p.y_out + (first - p.first) : nullptr;
#define MLMC_BATCH_CASES(CALL)                                                                  \
    switch (p.payoff) {                                                                         \
    case kEuropean: CALL(kEuropean); break;                                                     \
    case kAsian: CALL(kAsian); break;                                                           \
    case kLookback: CALL(kLookback); break;                                                     \
    case kDigital: CALL(kDigital); break;                                                       \
    case kLinear: CALL(kLinear); break;                                                         \
    case kGeoAsian: CALL(kGeoAsian); break;                                                     \
    default: break;                                                                             \
    }
#define MLMC_SMALL(PAY) small_range<R, PAY, false, false>(p, first, count, t, T, m, b1, b2, b3, b4, nb, y)
#define MLMC_SPLIT(PAY) regular_range<R, MT, PAY, true, false, false>(p, first, count, t, T, m, b1, b2, b3, b4, nb, y)
#define MLMC_PLAIN(PAY) regular_range<R, MT, PAY, false, false, false>(p, first, count, t, T, m, b1, b2, b3, b4, nb, y)
    if (p.small) {
        MLMC_BATCH_CASES(MLMC_SMALL)
    } else if (p.lanes > 1) {
        MLMC_BATCH_CASES(MLMC_SPLIT)
    } else {
        MLMC_BATCH_CASES(MLMC_PLAIN)
    }
#undef MLMC_SMALL
#undef MLMC_SPLIT
#undef MLMC_PLAIN
#undef MLMC_BATCH_CASES
}

// Persistent kernel of one batched round: each block claims chunks from `counter` until none
// are left and writes the chunk's four power sums to chunk_sums[chunk].  A chunk is always
// processed by one whole block with the same thread-to-sample mapping, so its sums do not
// depend on which block claimed it.
template <typename R, int MT>
__global__ void __launch_bounds__(256) batch_kernel(const LevelParams *__restrict__ tasks,
                                                    const BatchChunk *__restrict__ chunks,
                                                    const BatchHeader *__restrict__ header,
                                                    unsigned *counter, double *chunk_sums)
{
    __shared__ unsigned s_chunk;
    const unsigned n_chunks = header->n_chunks;
    for (;;) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(counter, 1u);
        __syncthreads();
        const unsigned c = s_chunk;
        __syncthreads();
        if (c >= n_chunks) break;
        const BatchChunk ch = chunks[c];
        double m[4] = {0.0, 0.0, 0.0, 0.0};
        float b1 = 0.f, b2 = 0.f, b3 = 0.f, b4 = 0.f;
        int nb = 0;
        batch_chunk<R, MT>(tasks[ch.task], ch.first, ch.count, m, b1, b2, b3, b4, nb);
        fold_batch<R>(m, b1, b2, b3, b4);
        block_sum4(m);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) chunk_sums[4 * (size_t)c + k] = m[k];
        }
    }
}

}  // namespace mlmcgb

namespace mlmcgb {

// The arithmetic-Asian kernel for lanes of `long_lanes` (more than kLongLaneSteps steps) or not;
// the two are the same kernel where the sums keep one level (FP64 paths).
template <typename R, int MT, bool SPLIT, bool MIL, bool ANTI> const void *asian_kernel(bool long_lanes)
{
    if constexpr (kBlockedSum<R, kAsian>) {
        if (long_lanes) return (const void *)level_kernel<R, MT, kAsian, SPLIT, MIL, ANTI, true>;
    }
    return (const void *)level_kernel<R, MT, kAsian, SPLIT, MIL, ANTI>;
}

// Kernel for (payoff, M specialisation, split, scheme, lane length) at precision R; nullptr for
// an unknown payoff.
template <typename R, int MT, bool SPLIT, bool MIL>
const void *select_by_payoff(int payoff, bool long_lanes, bool positive = false)
{
    if constexpr (SPLIT) {
        if (payoff == kLookback && positive) return (const void *)level_kernel<R, MT, kLookback, true, MIL, false, false, true>;
    }
    switch (payoff) {
    case kEuropean: return (const void *)level_kernel<R, MT, kEuropean, SPLIT, MIL>;
    case kAsian: return asian_kernel<R, MT, SPLIT, MIL, false>(long_lanes);
    case kLookback: return (const void *)level_kernel<R, MT, kLookback, SPLIT, MIL>;
    case kDigital: return (const void *)level_kernel<R, MT, kDigital, SPLIT, MIL>;
    case kLinear: return (const void *)level_kernel<R, MT, kLinear, SPLIT, MIL>;
    case kGeoAsian: return (const void *)level_kernel<R, MT, kGeoAsian, SPLIT, MIL>;
    default: return nullptr;
    }
}

template <typename R, bool MIL> const void *select_small_kernel(int payoff)
{
    switch (payoff) {
    case kEuropean: return (const void *)level_small_kernel<R, kEuropean, MIL>;
    case kAsian: return (const void *)level_small_kernel<R, kAsian, MIL>;
    case kLookback: return (const void *)level_small_kernel<R, kLookback, MIL>;
    case kDigital: return (const void *)level_small_kernel<R, kDigital, MIL>;
    case kLinear: return (const void *)level_small_kernel<R, kLinear, MIL>;
    case kGeoAsian: return (const void *)level_small_kernel<R, kGeoAsian, MIL>;
    default: return nullptr;
    }
}

// mt = -1 selects the kernel of levels with M^l < 4; MIL the Milstein kernels.
template <typename R, bool MIL>
const void *select_scheme(int payoff, int mt, bool split, bool long_lanes, bool positive = false)
{
    if (mt < 0) return select_small_kernel<R, MIL>(payoff);
    if (mt == 4)
        return split ? select_by_payoff<R, 4, true, MIL>(payoff, long_lanes, positive)
                     : select_by_payoff<R, 4, false, MIL>(payoff, long_lanes);
    return split ? select_by_payoff<R, 0, true, MIL>(payoff, long_lanes, positive)
                 : select_by_payoff<R, 0, false, MIL>(payoff, long_lanes);
}


// Antithetic kernels: mt = 4 (M = 4) or 0 (M = 2), one thread per sample; nullptr otherwise.
template <typename R, int MT, bool MIL> const void *select_anti_by_payoff(int payoff, bool long_lanes)
{
    switch (payoff) {
    case kEuropean: return (const void *)level_kernel<R, MT, kEuropean, false, MIL, true>;
    case kAsian: return asian_kernel<R, MT, false, MIL, true>(long_lanes);
    case kLookback: return (const void *)level_kernel<R, MT, kLookback, false, MIL, true>;
    case kDigital: return (const void *)level_kernel<R, MT, kDigital, false, MIL, true>;
    case kLinear: return (const void *)level_kernel<R, MT, kLinear, false, MIL, true>;
    case kGeoAsian: return (const void *)level_kernel<R, MT, kGeoAsian, false, MIL, true>;
    default: return nullptr;
    }
}
template <typename R> const void *select_anti_kernel(int payoff, int mt, int scheme, bool long_lanes)
{
    if (mt == 4)
        return scheme == 1 ? select_anti_by_payoff<R, 4, true>(payoff, long_lanes)
                           : select_anti_by_payoff<R, 4, false>(payoff, long_lanes);
    if (mt == 0)
        return scheme == 1 ? select_anti_by_payoff<R, 0, true>(payoff, long_lanes)
                           : select_anti_by_payoff<R, 0, false>(payoff, long_lanes);
    return nullptr;
}

// Two-samples-per-thread kernels (Euler--Maruyama, one thread per sample, mt = 4 or 0).
template <typename R, int MT> const void *select_ns2_by_payoff(int payoff, bool long_lanes)
{
    switch (payoff) {
    case kEuropean: return (const void *)level_ns2_kernel<R, MT, kEuropean>;
    case kAsian:
        if constexpr (kBlockedSum<R, kAsian>) {
            if (long_lanes) return (const void *)level_ns2_kernel<R, MT, kAsian, true>;
        }
        return (const void *)level_ns2_kernel<R, MT, kAsian>;
    case kLookback: return (const void *)level_ns2_kernel<R, MT, kLookback>;
    case kDigital: return (const void *)level_ns2_kernel<R, MT, kDigital>;
    case kLinear: return (const void *)level_ns2_kernel<R, MT, kLinear>;
    case kGeoAsian: return (const void *)level_ns2_kernel<R, MT, kGeoAsian>;
    default: return nullptr;
    }
}
template <typename R> const void *select_ns2_kernel(int payoff, int mt, bool long_lanes)
{
    if (mt == 4) return select_ns2_by_payoff<R, 4>(payoff, long_lanes);
    if (mt == 0) return select_ns2_by_payoff<R, 0>(payoff, long_lanes);
    return nullptr;
}

template <typename R> const void *select_batch_kernel(int mt)
{
    return mt == 4 ? (const void *)batch_kernel<R, 4> : (const void *)batch_kernel<R, 0>;
}

}  // namespace mlmcgb
