// engine.h -- internal interface between the C ABI and the level kernels.
#pragma once
#include <cstddef>
#include <cstdint>

namespace mlmcgb {

// Payoff codes, equal to the public mlmc_payoff_kind values.
enum : int { kEuropean = 0, kAsian = 1, kLookback = 2, kDigital = 3, kLinear = 100, kGeoAsian = 101 };

// Everything one level launch needs, passed by value as the kernel argument.
struct LevelParams {
    double S0;        // initial value
    double disc;      // exp(-r T)
    double K, Q;      // strike, digital cash
    double a;         // sigma * sqrt(h), h = T / M^l
    double rh;        // r * fine step
    double inv_nf;    // 1 / M^l
    double inv_nc;    // 1 / M^(l-1)
    double sqrt_h;    // sqrt(h): Brownian increment scale of one fine step
    double sqrt_tg;   // sqrt(T / 16): scale of the control variate's grid increments
    double h;         // fine step T / M^l
    // FP32 payoff constants of the call options on paths relative to S0 (rel_payoff): disc S0,
    // -disc K, and for the fine (f) and coarse (c) path disc S0 / n, disc S0 / (2 n) - disc K
    float pay_dS0, pay_mdK, pay_af, pay_bf, pay_ac, pay_bc;
    uint64_t first;   // first sample index
    uint64_t N;       // number of samples
    uint32_t key0, key1;  // Philox key (seed low, seed high)
    uint32_t ctr3;        // Philox counter word 3: (tag << 16) | level
    uint32_t rkey[20];    // Philox round keys: key0 + i W_A, key1 + i W_B for rounds i = 0..9
    int level, M;
    int nf;           // fine steps M^l
    int lanes;        // lanes per sample (1 = one thread per sample)
    int small;        // 1 when M^l < 4: 4 / M^l samples share one Philox block
    int payoff;       // payoff code (the batched kernel selects its code path from it)
    double c2;        // sigma^2 h / 2: the Milstein term's scale on the fine grid
    int scheme;       // 0 Euler--Maruyama, 1 Milstein
    int fine_only;    // 1: Y = P_l alone (single-level estimator)
    int u23;          // FP64 arithmetic on the FP32 stream's 23-bit uniforms
    int antithetic;   // antithetic estimator (read by the kernel of levels with M^l < 4)
    double *partials; // [gridDim.x][4] block partial sums (workspace)
    double *out;      // [4] level sums (device)
    unsigned *ticket; // completion counter (workspace), zero between launches
    double *y_out;    // optional per-sample Y, NULL = off
};

// Workspace layout: the completion ticket in the first 256 bytes, then the FP64 partial sums
// of `blocks` blocks.  The ticket sits at a fixed offset so that launches of any grid size can
// share one workspace: it is zero between launches, while the partials need no initial value.
constexpr size_t kTicketBytes = 256;
inline size_t workspace_bytes_for_blocks(int blocks)
{
    return kTicketBytes + (size_t)blocks * 4 * sizeof(double);
}

// Kernel selection.  `mt` is 4 for the M = 4 specialisation, 0 for the generic-M kernel and
// -1 for the kernel of levels with M^l < 4.  `long_lanes`: a lane runs more than kLongLaneSteps
// fine steps of its path (M^l / lanes), for which the FP32 arithmetic-Asian kernels add the
// running sum in two levels (partials of 256 steps).  `positive`: every fine and coarse step
// factor 1 + d is positive for any normal the stream can produce, so the split lookback kernels
// keep no running minimum (no chunk of a path starts below zero).
constexpr long kLongLaneSteps = 4096;
const void *level_kernel_fp32(int payoff, int mt, bool split, int scheme, bool long_lanes, bool positive = false);
// Milstein kernels (level_fp32_mil.cu, level_fp64_mil.cu), selected by the two above.
const void *level_kernel_fp32_milstein(int payoff, int mt, bool split, bool long_lanes, bool positive);
const void *level_kernel_fp64_milstein(int payoff, int mt, bool split, bool long_lanes, bool positive);
// Antithetic level kernels (level_anti_fp32.cu, level_anti_fp64.cu): mt = 4 (M = 4) or 0 (M = 2).
const void *level_anti_kernel_fp32(int payoff, int mt, int scheme, bool long_lanes);
const void *level_anti_kernel_fp64(int payoff, int mt, int scheme, bool long_lanes);
// Two samples per thread (level_fp32_ns2.cu): FP32 paths, Euler--Maruyama, one thread per sample,
// mt = 4 or 0; at most 512 threads per block.
const void *level_ns2_kernel_fp32(int payoff, int mt, bool long_lanes);
constexpr int kNs2MaxThreads = 512;
// The planners' default of two samples per thread: FP32 Euler--Maruyama whole paths with M = 4
// and at least 16 fine steps.  The two-sample kernel takes the same samples per thread on the
// same grid (a thread's unpaired last sample runs alone).  Timed against one sample per thread on
// the lookback and arithmetic Asian calls at levels 2-7 and 0.3-6.4 waves of resident threads, it
// was 0.6 % slower in one case of 84 and faster in the rest: about 3 % on the lookback and 3-8 %
// on the Asian, 4.5 % over the whole set.  On the straight-line sample of M^l = 4 two samples per
// thread were slower.
constexpr long kNs2MinSteps = 16;
// The lanes-per-path model of both planners (plan_level and the device rounds): the cost of a
// partial last wave after whole ones, min(1, kLanesTailSlope f + kLanesTailBase) of a wave at
// fill f, and a split step's cost relative to a whole-path one.
constexpr double kLanesTailSlope = 1.25, kLanesTailBase = 0.1, kLanesSplitStep = 1.08;
// The control variate's level-estimator kernel (cv_level.cu) for a payoff on level `level` with
// refinement M: compiled for M^l = 1, 4, 16 at M = 4, else for a run-time M^l; NULL for an unknown
// payoff.
const void *cv_level_kernel_fp32(int payoff, int level, int M);
// Level kernel of the QUINTIC_ODE model (ode.cu): precision, scheme (EM or tamed EM).
const void *ode_level_kernel(int precision, int scheme);
const void *level_kernel_fp64(int payoff, int mt, bool split, int scheme, bool long_lanes, bool positive = false);

// Batched rounds: one chunk of samples of one task (a level of one problem).
struct BatchChunk {
    uint64_t first;   // first sample of the chunk
    uint32_t task;    // index into the task array
    uint32_t count;   // samples in the chunk
};
// Chunks [begin, end) belong to one task; the header counts tasks and chunks of the round.
struct BatchRange {
    uint32_t begin, end;
};
struct BatchHeader {
    uint32_t n_tasks, n_chunks;
};
// Persistent batch kernel and its fixed-order reduction, per precision and M specialisation
// (mt = 4 or 0).
const void *batch_kernel_fp32(int mt);
const void *batch_kernel_fp64(int mt);
const void *batch_reduce_kernel();

}  // namespace mlmcgb
