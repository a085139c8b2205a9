// api.cu -- the C ABI declared in include/mlmc.h: argument checks, launch planning, the
// workspace, and the adaptive multilevel driver (host side, FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "driver.h"
#include "engine.h"
#include "host.h"
#include "mlmc.h"
#include "rng.cuh"

using namespace mlmcgb;

namespace {

thread_local std::string g_error;

// Least cost of a launch with fewer items than one wave, in waves (see plan_level)
constexpr double kLoneWaveCost = 0.25;
// Samples per thread of one-thread-per-sample FP32 launches when neither the caller nor the
// autotuner chose.
constexpr int kDefaultSamplesPerThread = 1;

}  // namespace

namespace mlmcgb {

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}


long ipow(long b, int e)
{
    long p = 1;
    while (e-- > 0) p *= b;
    return p;
}

bool valid_payoff_kind(int k)
{
    return k == kEuropean || k == kAsian || k == kLookback || k == kDigital || k == kLinear ||
           k == kGeoAsian;
}

int check_problem(const mlmc_model *model, const mlmc_payoff *payoff)
{
    if (!model || !payoff) return fail(MLMC_EINVAL, "model and payoff must not be NULL");
    if (model->kind == MLMC_MODEL_QUINTIC_ODE) {
        if (model->scheme != MLMC_EULER_MARUYAMA && model->scheme != MLMC_TAMED_EM)
            return fail(MLMC_EINVAL, "the quintic ODE takes Euler--Maruyama or tamed Euler--Maruyama (scheme %d)",
                        model->scheme);
        if (!(model->T > 0) || !std::isfinite(model->T) || !std::isfinite(model->S0) ||
            !std::isfinite(model->r) || !std::isfinite(model->sigma))
            return fail(MLMC_EINVAL, "the quintic ODE needs a finite T > 0 (and finite unused fields)");
        if (payoff->kind != MLMC_SECOND_MOMENT)
            return fail(MLMC_EINVAL, "the quintic ODE takes the second-moment payoff (kind %d)", payoff->kind);
        if (payoff->estimator != MLMC_COUPLED && payoff->estimator != MLMC_SINGLE_LEVEL)
            return fail(MLMC_EINVAL, "unsupported estimator %d", payoff->estimator);
        return MLMC_OK;
    }
    if (model->kind != MLMC_MODEL_GBM) return fail(MLMC_EINVAL, "unsupported model kind %d", model->kind);
    if (model->scheme != MLMC_EULER_MARUYAMA && model->scheme != MLMC_MILSTEIN)
        return fail(MLMC_EINVAL, "GBM takes Euler--Maruyama or Milstein (scheme %d)", model->scheme);
    if (!(model->S0 > 0) || !std::isfinite(model->S0) || !(model->sigma > 0) ||
        !std::isfinite(model->sigma) || !(model->T > 0) || !std::isfinite(model->T) ||
        !std::isfinite(model->r))
        return fail(MLMC_EINVAL, "GBM needs finite S0 > 0, sigma > 0, T > 0 and r");
    if (!valid_payoff_kind(payoff->kind)) return fail(MLMC_EINVAL, "unsupported payoff kind %d", payoff->kind);
    if (payoff->estimator != MLMC_COUPLED && payoff->estimator != MLMC_SINGLE_LEVEL &&
        payoff->estimator != MLMC_ANTITHETIC)
        return fail(MLMC_EINVAL, "unsupported estimator %d", payoff->estimator);
    if (!std::isfinite(payoff->K) || !std::isfinite(payoff->cash))
        return fail(MLMC_EINVAL, "payoff K and cash must be finite");
    return MLMC_OK;
}

int check_level(int level, int M)
{
    if (M != 2 && M != 4 && M != 8) return fail(MLMC_EINVAL, "M must be 2, 4 or 8 (got %d)", M);
    if (level < 0 || level >= MLMC_MAX_LEVELS || ipow(M, level) > (1L << 24))
        return fail(MLMC_EINVAL, "level %d out of range for M = %d (need M^level <= 2^24)", level, M);
    return MLMC_OK;
}

int device_sms(int *sms)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    return MLMC_OK;
}

// Largest grid the workspace must hold for a given block size: resident blocks of the kernel.
int max_resident_blocks(const void *kernel, int threads, int *out)
{
    int sms = 0, per_sm = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0));
    if (per_sm < 1) return fail(MLMC_EINVAL, "level kernel cannot run with %d threads per block", threads);
    *out = per_sm * sms;
    return MLMC_OK;
}

// Launch shape for one level: explicit fields of `launch` win, zeros are filled in.
int plan_level(int level, int M, uint64_t N, int precision, int payoff, int scheme, const mlmc_launch *launch,
               Plan *plan)
{
    if (precision != MLMC_FP64 && precision != MLMC_FP32_PATH && precision != MLMC_FP64_STREAM32)
        return fail(MLMC_EINVAL, "precision must be MLMC_FP64, MLMC_FP32_PATH or MLMC_FP64_STREAM32");
    const int ns_req = launch ? launch->samples_per_thread : 0;
    if (ns_req < 0 || ns_req > 2) return fail(MLMC_EINVAL, "samples_per_thread must be 0 (automatic), 1 or 2");
    const long nf = ipow(M, level);
    const int unit = std::max(M, 4);  // a lane's chunk holds whole Philox blocks and coarse steps
    // a shape chosen by the autotuner fills the fields the caller left at zero
    TunedShape tuned;
    const bool have_tuned = scheme == MLMC_EULER_MARUYAMA && tuned_lookup(precision, payoff, M, level, N, &tuned);
    int threads = launch && launch->threads_per_block ? launch->threads_per_block
                                                      : (have_tuned ? tuned.threads : 256);
    if (threads < 32 || threads > 1024 || threads % 32)
        return fail(MLMC_EINVAL, "threads_per_block must be a multiple of 32 in [32, 1024]");
    int lanes = launch && launch->lanes_per_path ? launch->lanes_per_path : 0;
    if (!lanes && have_tuned && (tuned.lanes == 1 || (nf >= 8 && nf % tuned.lanes == 0 &&
                                                      (nf / tuned.lanes) % unit == 0)))
        lanes = tuned.lanes;
    if (lanes) {
        if (lanes < 1 || lanes > 32 || (lanes & (lanes - 1)))
            return fail(MLMC_EINVAL, "lanes_per_path must be a power of two in [1, 32]");
        if (lanes > 1 && (nf < 8 || (nf / lanes) % unit != 0 || nf % lanes != 0))
            return fail(MLMC_EINVAL, "lanes_per_path %d does not divide M^l = %ld into chunks of a "
                        "multiple of %d steps", lanes, nf, unit);
    } else {
        // The power of two P (chunks of whole Philox blocks and coarse steps, at least 256 steps
        // each) with the least modelled launch time.  T resident threads run the N P lane-items
        // in waves; after w >= 1 whole waves, a partial last wave filled to a fraction f costs
        // min(1, 1.25 f + 0.1) of a full one (its warps run faster on the emptier SMs), and a
        // launch of fewer items than a wave min(1, 3 f).  A lane costs its M^l / P steps plus
        // about 12 steps of chunk join, payoff and moments, and a split step about 8 % more than
        // a whole-path one (two samples per thread).  A larger P must win by more than 1 %.
        // (Fitted to launch timings of the lookback, levels 5..8 at 0.2..3.7 waves: 1.3-1.6 %
        // less time per level than the earlier fit.)  Fewer items than one wave still cost at least a
        // quarter of a wave: a warp alone on its scheduler takes about 64 cycles per step,
        // against about 266 for each warp of a full SM (measured on levels 6..12 at 1 to 2^15
        // samples), so short launches go to the most lanes.
        lanes = 1;
        if (nf >= 8) {
            const int mt1 = M == 4 ? 4 : 0;
            const void *k1 = precision == MLMC_FP32_PATH ? level_kernel_fp32(payoff, mt1, false, scheme, false)
                                                         : level_kernel_fp64(payoff, mt1, false, scheme, false);
            const void *kp = precision == MLMC_FP32_PATH ? level_kernel_fp32(payoff, mt1, true, scheme, false)
                                                         : level_kernel_fp64(payoff, mt1, true, scheme, false);
            if (!k1 || !kp) return fail(MLMC_EINVAL, "no kernel for payoff %d", payoff);
            int res1 = 0, resp = 0;
            int rc = max_resident_blocks(k1, threads, &res1);
            if (rc) return rc;
            rc = max_resident_blocks(kp, threads, &resp);
            if (rc) return rc;
            double best = 0.0;
            for (int P = 1; P <= 32; P *= 2) {
                if (P > 1 && (nf % P != 0 || (nf / P) % unit != 0 || nf / P < 256)) break;
                const double T = (double)(P == 1 ? res1 : resp) * threads;
                const double w = (double)std::max<uint64_t>(N, 1) * P / T;
                const double full = std::floor(w);
                const double waves = w < 1.0 ? std::max(std::min(1.0, 3.0 * w), kLoneWaveCost)
                                             : full + std::min(1.0, kLanesTailSlope * (w - full) + kLanesTailBase);
                const double per_step = P > 1 ? kLanesSplitStep : 1.0;
                const double cost = waves * ((double)nf / P + 12.0) * per_step;
                if (P == 1 || cost < 0.99 * best) {
                    best = cost;
                    lanes = P;
                }
            }
        }
    }
    const bool split = lanes > 1;
    const bool small = nf < 4;
    const int mt = small ? -1 : (M == 4 ? 4 : 0);
    const bool long_lanes = nf / lanes > kLongLaneSteps;
    // samples per thread: the two-sample kernel exists for FP32 Euler--Maruyama whole paths
    const bool ns2_ok = !split && !small && precision == MLMC_FP32_PATH && scheme == MLMC_EULER_MARUYAMA &&
                        threads <= kNs2MaxThreads;
    const int auto_ns = ns2_ok && M == 4 && nf >= kNs2MinSteps ? 2 : kDefaultSamplesPerThread;
    int ns = ns_req ? ns_req : (have_tuned && tuned.ns ? tuned.ns : auto_ns);
    if (ns == 2 && !ns2_ok) {
        if (ns_req == 2)
            return fail(MLMC_EINVAL, "samples_per_thread 2 needs FP32 Euler--Maruyama paths with M^l >= 4, "
                        "lanes_per_path 1 and at most %d threads per block", kNs2MaxThreads);
        ns = 1;
    }
    plan->kernel = ns == 2 ? level_ns2_kernel_fp32(payoff, mt, long_lanes)
                 : precision == MLMC_FP32_PATH ? level_kernel_fp32(payoff, mt, split, scheme, long_lanes)
                                               : level_kernel_fp64(payoff, mt, split, scheme, long_lanes);
    if (!plan->kernel) return fail(MLMC_EINVAL, "no kernel for payoff %d", payoff);
    int max_blocks = 0;
    int rc = max_resident_blocks(plan->kernel, threads, &max_blocks);
    if (rc) return rc;
    int blocks = launch && launch->blocks ? launch->blocks : 0;
    if (blocks < 0) return fail(MLMC_EINVAL, "blocks must be >= 0");
    // the sample loops stride by the grid's thread count in 32-bit offsets below 2^31
    if ((uint64_t)blocks * (uint64_t)threads >= (uint64_t(1) << 31))
        return fail(MLMC_EINVAL, "blocks x threads_per_block must be below 2^31");
    if (!blocks) {
        // work items: samples x lanes, or Philox blocks of 4 / M^l samples on small levels (the
        // two-sample kernel runs on the one-sample kernel's grid)
        const double items = small ? std::ceil((double)std::max<uint64_t>(N, 1) * nf / 4.0) + 1.0
                                   : (double)std::max<uint64_t>(N, 1) * lanes;
        const double need = std::ceil(items / threads);
        const int oversub = have_tuned ? std::max(1, tuned.oversub) : 1;
        blocks = (int)std::min<double>(need, (double)max_blocks * oversub);
    }
    blocks = std::max(blocks, 1);
    plan->threads = threads;
    plan->lanes = lanes;
    plan->blocks = blocks;
    plan->ns = ns;
    return MLMC_OK;
}

// Launch shape of the QUINTIC_ODE kernel: one thread per Philox block of four samples, no
// lanes split; explicit fields of `launch` (threads, blocks) win.
static int plan_ode(int level, int M, uint64_t N, int precision, int scheme, const mlmc_launch *launch, Plan *plan)
{
    if (precision != MLMC_FP64 && precision != MLMC_FP32_PATH && precision != MLMC_FP64_STREAM32)
        return fail(MLMC_EINVAL, "precision must be MLMC_FP64, MLMC_FP32_PATH or MLMC_FP64_STREAM32");
    if (launch && launch->samples_per_thread > 1)
        return fail(MLMC_EINVAL, "the quintic ODE kernel takes one sample per thread");
    if (launch && launch->lanes_per_path > 1)
        return fail(MLMC_EINVAL, "the quintic ODE runs one thread per sample (lanes_per_path %d)",
                    launch->lanes_per_path);
    (void)level;
    (void)M;
    const int threads = launch && launch->threads_per_block ? launch->threads_per_block : 256;
    if (threads < 32 || threads > 256 || threads % 32)
        return fail(MLMC_EINVAL, "threads_per_block must be a multiple of 32 in [32, 256] for the quintic ODE");
    plan->kernel = ode_level_kernel(precision, scheme);
    if (!plan->kernel) return fail(MLMC_EINVAL, "no quintic ODE kernel for scheme %d", scheme);
    int max_blocks = 0;
    int rc = max_resident_blocks(plan->kernel, threads, &max_blocks);
    if (rc) return rc;
    int blocks = launch && launch->blocks ? launch->blocks : 0;
    if (blocks < 0) return fail(MLMC_EINVAL, "blocks must be >= 0");
    // the sample loops stride by the grid's thread count in 32-bit offsets below 2^31
    if ((uint64_t)blocks * (uint64_t)threads >= (uint64_t(1) << 31))
        return fail(MLMC_EINVAL, "blocks x threads_per_block must be below 2^31");
    if (!blocks) {
        const double items = std::ceil((double)std::max<uint64_t>(N, 1) / 4.0) + 1.0;
        blocks = (int)std::min<double>(std::ceil(items / threads), (double)max_blocks);
    }
    plan->threads = threads;
    plan->lanes = 1;
    plan->blocks = std::max(blocks, 1);
    return MLMC_OK;
}

// Whether every fine and coarse step factor 1 + d of a GBM path on this level is positive for any
// normal the stream can produce.  The uniforms are at least 2^-32 (FP64 stream) or 2^-23 (FP32),
// so |z| <= sqrt(-2 ln 2^-32) < 6.7; the bound used is 7.  Euler--Maruyama: the fine factor is at
// least 1 + r h - sigma sqrt(h) 7, the coarse one (M fine increments summed) at least
// 1 + r M h - sigma M sqrt(h) 7.  Milstein: the factor is a quadratic in w = sigma sqrt(h) z whose
// least value over all w is 1/2 + r h - sigma^2 h / 2, and the same with M h for the coarse step.
bool positive_step_factors(const mlmc_model *m, int level, int M)
{
    constexpr double kNormalBound = 7.0, kMargin = 1e-2;
    const double h = m->T / (double)ipow(M, level), H = M * h;
    if (m->scheme == MLMC_MILSTEIN)
        return 0.5 + m->r * h - 0.5 * m->sigma * m->sigma * h > kMargin &&
               0.5 + m->r * H - 0.5 * m->sigma * m->sigma * H > kMargin;
    return 1.0 + m->r * h - m->sigma * std::sqrt(h) * kNormalBound > kMargin &&
           1.0 + m->r * H - m->sigma * M * std::sqrt(h) * kNormalBound > kMargin;
}

int plan_problem(int level, int M, uint64_t N, int precision, const mlmc_model *model, const mlmc_payoff *payoff,
                 const mlmc_launch *launch, Plan *plan)
{
    if (model->kind == MLMC_MODEL_QUINTIC_ODE) return plan_ode(level, M, N, precision, model->scheme, launch, plan);
    if (payoff->estimator != MLMC_ANTITHETIC) {
        const int rc = plan_level(level, M, N, precision, payoff->kind, model->scheme, launch, plan);
        if (rc) return rc;
        // split lookback paths whose chunks all start above zero keep no running minimum
        if (plan->lanes > 1 && payoff->kind == kLookback && positive_step_factors(model, level, M)) {
            const int mt = M == 4 ? 4 : 0;
            const void *k = precision == MLMC_FP32_PATH
                                ? level_kernel_fp32(payoff->kind, mt, true, model->scheme, false, true)
                                : level_kernel_fp64(payoff->kind, mt, true, model->scheme, false, true);
            if (k) plan->kernel = k;
        }
        return MLMC_OK;
    }
    // antithetic: one thread per sample; the kernel of levels with M^l < 4 reads the flag
    if (M != 2 && M != 4) return fail(MLMC_ENOTIMPL, "the antithetic estimator is built for M = 2 and 4 (M = %d)", M);
    if (launch && launch->lanes_per_path > 1)
        return fail(MLMC_EINVAL, "the antithetic estimator runs one thread per sample (lanes_per_path %d)",
                    launch->lanes_per_path);
    if (launch && launch->samples_per_thread > 1)
        return fail(MLMC_EINVAL, "the antithetic kernels take one sample per thread");
    mlmc_launch one = launch ? *launch : mlmc_launch{0, 0, 0, 0};
    one.lanes_per_path = 1;
    one.samples_per_thread = 1;
    int rc = plan_level(level, M, N, precision, payoff->kind, model->scheme, &one, plan);
    if (rc || ipow(M, level) < 4) return rc;
    const int mt = M == 4 ? 4 : 0;
    const bool long_lanes = ipow(M, level) > kLongLaneSteps;
    plan->kernel = precision == MLMC_FP32_PATH ? level_anti_kernel_fp32(payoff->kind, mt, model->scheme, long_lanes)
                                               : level_anti_kernel_fp64(payoff->kind, mt, model->scheme, long_lanes);
    if (!plan->kernel) return fail(MLMC_EINVAL, "no antithetic kernel for payoff %d", payoff->kind);
    int resident = 0;
    rc = max_resident_blocks(plan->kernel, plan->threads, &resident);
    if (rc) return rc;
    if (!(launch && launch->blocks)) plan->blocks = std::max(1, std::min(plan->blocks, resident));
    return MLMC_OK;
}

double problem_cost(int level, int M, const mlmc_payoff *payoff)
{
    if (level > 0 && payoff->estimator == MLMC_ANTITHETIC)
        return (double)(2 * ipow(M, level) + ipow(M, level - 1));
    if (payoff->estimator == MLMC_SINGLE_LEVEL) return (double)ipow(M, level);
    return level_cost(level, M);
}

void fill_params(LevelParams &p, int level, int M, uint64_t N, uint64_t first,
                 const mlmc_model *m, const mlmc_payoff *pay, uint64_t seed, int tag, int lanes, int precision)
{
    const long nf = ipow(M, level);
    p.S0 = m->S0;
    p.disc = std::exp(-m->r * m->T);
    p.K = pay->K;
    p.Q = pay->cash;
    const double h = m->T / (double)nf;
    p.small = nf < 4 ? 1 : 0;
    p.a = m->sigma * std::sqrt(h);
    p.sqrt_h = std::sqrt(h);
    p.sqrt_tg = std::sqrt(m->T / 16.0);
    p.rh = m->r * h;
    p.h = h;
    p.inv_nf = 1.0 / (double)nf;
    p.inv_nc = level > 0 ? (double)M / (double)nf : 0.0;
    const double dS0 = p.disc * p.S0, dK = p.disc * p.K;
    p.pay_dS0 = (float)dS0;
    p.pay_mdK = (float)(-dK);
    p.pay_af = (float)(dS0 * p.inv_nf);
    p.pay_bf = (float)(0.5 * dS0 * p.inv_nf - dK);
    p.pay_ac = (float)(dS0 * p.inv_nc);
    p.pay_bc = (float)(0.5 * dS0 * p.inv_nc - dK);
    p.first = first;
    p.N = N;
    p.key0 = (uint32_t)seed;
    p.key1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        p.rkey[2 * i] = p.key0 + (uint32_t)i * kPhiloxWeylA;
        p.rkey[2 * i + 1] = p.key1 + (uint32_t)i * kPhiloxWeylB;
    }
    p.ctr3 = ((uint32_t)tag << 16) | (uint32_t)level;
    p.level = level;
    p.M = M;
    p.nf = (int)nf;
    p.lanes = lanes;
    p.payoff = pay->kind;
    p.c2 = 0.5 * m->sigma * m->sigma * h;
    p.scheme = m->scheme;
    p.fine_only = pay->estimator == MLMC_SINGLE_LEVEL ? 1 : 0;
    p.u23 = precision == MLMC_FP64_STREAM32 ? 1 : 0;
    p.antithetic = pay->estimator == MLMC_ANTITHETIC ? 1 : 0;
    p.partials = nullptr;
    p.out = nullptr;
    p.ticket = nullptr;
    p.y_out = nullptr;
}

double level_cost(int level, int M)
{
    return level == 0 ? 1.0 : (double)(ipow(M, level) + ipow(M, level - 1));
}

int check_tag(int tag)
{
    if (tag < 0 || tag > 0xFFFF) return fail(MLMC_EINVAL, "tag must be in [0, 65535]");
    return MLMC_OK;
}

int launch_level(const Plan &plan, LevelParams &p, void *ws, cudaStream_t st)
{
    p.ticket = (unsigned *)ws;
    p.partials = (double *)((char *)ws + kTicketBytes);
    void *args[] = {&p};
    CUDA_TRY(cudaLaunchKernel(plan.kernel, dim3(plan.blocks), dim3(plan.threads), args, 0, st));
    return MLMC_OK;
}

}  // namespace mlmcgb

namespace mlmcgb {

// Cached device address of the allocation-free entry point's scratch, per device (looked up on
// first use; cleared by mlmc_shutdown, since a device reset moves the array).
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[kMaxDevices] = {};
static void noalloc_forget(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    g_noalloc_ptr[dev] = nullptr;
}

// Device buffers of the adaptive drivers (workspace, level sums, pinned host copy, timing
// events), kept between calls in a per-device pool: allocating and pinning them on every call
// cost more than the kernels of a small estimate.  A call takes a set from the pool (or makes
// one) and returns it when it ends; a call that met a CUDA error frees its set instead.
static std::mutex g_pool_mutex;
static std::vector<DriverScratch *> g_pool;

void free_scratch(DriverScratch *s)
{
    if (!s) return;
    if (s->ws) cudaFree(s->ws);
    if (s->d_sums) cudaFree(s->d_sums);
    if (s->h_sums) cudaFreeHost(s->h_sums);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->fork) cudaEventDestroy(s->fork);
    for (int k = 0; k < kDriverStreams - 1; ++k) {
        if (s->aux[k]) {
            cudaStreamSynchronize(s->aux[k]);
            cudaStreamDestroy(s->aux[k]);
        }
        if (s->join[k]) cudaEventDestroy(s->join[k]);
    }
    delete s;
}

int acquire_scratch(size_t ws_bytes, DriverScratch **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        for (size_t i = 0; i < g_pool.size(); ++i) {
            if (g_pool[i]->device == dev && g_pool[i]->ws_bytes >= ws_bytes) {
                *out = g_pool[i];
                g_pool.erase(g_pool.begin() + (long)i);
                return MLMC_OK;
            }
        }
    }
    DriverScratch *s = new DriverScratch;
    s->device = dev;
    s->ws_bytes = ws_bytes;
    cudaError_t e = cudaMalloc(&s->ws, ws_bytes);
    if (e == cudaSuccess) e = cudaMemset(s->ws, 0, ws_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_sums, kDriverSumsPerLevel * MLMC_MAX_LEVELS * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_sums, kDriverSumsPerLevel * MLMC_MAX_LEVELS * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
    for (int k = 0; k < kDriverStreams - 1 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&s->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_scratch(s);
        return fail(MLMC_ECUDA, "driver setup failed: %s", cudaGetErrorString(e));
    }
    *out = s;
    return MLMC_OK;
}

void release_scratch(DriverScratch *s)
{
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    g_pool.push_back(s);
}

}  // namespace mlmcgb

extern "C" {

const char *mlmc_last_error(void) { return g_error.c_str(); }

const char *mlmc_version(void) { return "mlmc-gb300 0.1 (sm_103a)"; }

int mlmc_device_sm_count(void)
{
    int sms = 0;
    if (device_sms(&sms)) return -1;
    return sms;
}

int mlmc_shutdown(void)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    noalloc_forget(dev);
    graph_driver_release(dev);
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    for (size_t i = 0; i < g_pool.size();) {
        if (g_pool[i]->device == dev) {
            free_scratch(g_pool[i]);
            g_pool.erase(g_pool.begin() + (long)i);
        } else {
            ++i;
        }
    }
    return MLMC_OK;
}

size_t mlmc_level_workspace_bytes(int level, int M, uint64_t N, int precision,
                                  const mlmc_launch *launch)
{
    if (check_level(level, M)) return 0;
    Plan plan;
    if (plan_level(level, M, N, precision, kEuropean, MLMC_EULER_MARUYAMA, launch, &plan)) return 0;
    // The grid the planner picks depends on the payoff's kernel; size for the largest grid any
    // of them can get: an explicit block count, or 32 resident blocks on every SM.
    int sms = 0;
    if (device_sms(&sms)) return 0;
    const int bound = launch && launch->blocks ? launch->blocks : sms * 32;
    return workspace_bytes_for_blocks(bound);
}

int mlmc_level_sums_async(int level, int M, uint64_t N, uint64_t first, const mlmc_model *model,
                          const mlmc_payoff *payoff, uint64_t seed, int precision, int tag,
                          const mlmc_launch *launch, double *d_sums, void *d_workspace,
                          size_t workspace_bytes, double *d_y, void *stream)
{
    int rc = check_level(level, M);
    if (!rc) rc = check_problem(model, payoff);
    if (!rc) rc = check_tag(tag);
    if (rc) return rc;
    if (!d_sums) return fail(MLMC_EINVAL, "d_sums must not be NULL");
    if (first + N < first) return fail(MLMC_EINVAL, "first + N overflows 64 bits");
    cudaStream_t st = (cudaStream_t)stream;
    Plan plan;
    rc = plan_problem(level, M, N, precision, model, payoff, launch, &plan);
    if (rc) return rc;
    if (N == 0) {
        CUDA_TRY(cudaMemsetAsync(d_sums, 0, 4 * sizeof(double), st));
        return MLMC_OK;
    }
    if (!d_workspace || ((uintptr_t)d_workspace & 255))
        return fail(MLMC_EINVAL, "workspace must be a 256-byte aligned device pointer");
    if (workspace_bytes < workspace_bytes_for_blocks(plan.blocks))
        return fail(MLMC_EINVAL, "workspace of %zu bytes is smaller than the %zu this launch needs",
                    workspace_bytes, workspace_bytes_for_blocks(plan.blocks));
    LevelParams p;
    fill_params(p, level, M, N, first, model, payoff, seed, tag, plan.lanes, precision);
    p.out = d_sums;
    p.y_out = d_y;
    return launch_level(plan, p, d_workspace, st);
}

// ------------------------------------------------------------------ allocation-free variant
//
// Scratch of the allocation-free entry point: block partials for at most kNoAllocMaxBlocks
// blocks and the completion ticket, in a file-scope device array.  Every GPU that loads this
// library holds it until the process exits.
}  // extern "C"

namespace {
constexpr int kNoAllocMaxBlocks = 2048;
constexpr size_t kNoAllocScratchBytes = kTicketBytes + (size_t)kNoAllocMaxBlocks * 4 * sizeof(double);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];


// Device address of g_noalloc_scratch on the current device.  In host code the array's name
// only stands in for the symbol, so the address is looked up once per device, with that device
// current, and cached.
int noalloc_scratch(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MLMC_EINVAL, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(MLMC_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return MLMC_OK;
}
}  // namespace

extern "C" {

int mlmc_level_sums_noalloc(int level, int M, uint64_t N, uint64_t first, const mlmc_model *model,
                            const mlmc_payoff *payoff, uint64_t seed, int precision, int tag,
                            const mlmc_launch *launch, double *d_sums, double *d_y, void *stream)
{
    int rc = check_level(level, M);
    if (!rc) rc = check_problem(model, payoff);
    if (!rc) rc = check_tag(tag);
    if (rc) return rc;
    if (!d_sums) return fail(MLMC_EINVAL, "d_sums must not be NULL");
    if (first + N < first) return fail(MLMC_EINVAL, "first + N overflows 64 bits");
    if (launch && launch->blocks > kNoAllocMaxBlocks)
        return fail(MLMC_EINVAL, "%d blocks need %zu bytes of scratch; the static scratch holds %d blocks "
                    "(%zu bytes)", launch->blocks, workspace_bytes_for_blocks(launch->blocks),
                    kNoAllocMaxBlocks, kNoAllocScratchBytes);
    cudaStream_t st = (cudaStream_t)stream;
    Plan plan;
    rc = plan_problem(level, M, N, precision, model, payoff, launch, &plan);
    if (rc) return rc;
    if (N == 0) {
        CUDA_TRY(cudaMemsetAsync(d_sums, 0, 4 * sizeof(double), st));
        return MLMC_OK;
    }
    plan.blocks = std::min(plan.blocks, kNoAllocMaxBlocks);
    void *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    LevelParams p;
    fill_params(p, level, M, N, first, model, payoff, seed, tag, plan.lanes, precision);
    p.out = d_sums;
    p.y_out = d_y;
    // The ticket keeps whatever the last call left; clear it on the stream before the launch.
    CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(unsigned), st));
    return launch_level(plan, p, scratch, st);
}

int mlmc_level_sums_ex(int level, int M, uint64_t N, uint64_t first, const mlmc_model *model,
                       const mlmc_payoff *payoff, uint64_t seed, int precision, int tag,
                       const mlmc_launch *launch, void *stream, double sums[4], double *cost)
{
    int rc = check_level(level, M);
    if (!rc) rc = check_problem(model, payoff);
    if (!rc) rc = check_tag(tag);
    if (rc) return rc;
    if (!sums || !cost) return fail(MLMC_EINVAL, "sums and cost must not be NULL");
    if (first + N < first) return fail(MLMC_EINVAL, "first + N overflows 64 bits");
    cudaStream_t st = (cudaStream_t)stream;
    Plan plan;
    rc = plan_problem(level, M, N, precision, model, payoff, launch, &plan);
    if (rc) return rc;
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    if (N > 0) {
        const size_t ws_bytes = workspace_bytes_for_blocks(plan.blocks) + 64;
        void *ws = nullptr;
        CUDA_TRY(cudaMallocAsync(&ws, ws_bytes, st));
        cudaError_t e = cudaMemsetAsync(ws, 0, ws_bytes, st);
        LevelParams p;
        fill_params(p, level, M, N, first, model, payoff, seed, tag, plan.lanes, precision);
        p.out = (double *)((char *)ws + workspace_bytes_for_blocks(plan.blocks));
        if (e == cudaSuccess) rc = launch_level(plan, p, ws, st);
        else rc = fail(MLMC_ECUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
        if (!rc) {
            e = cudaMemcpyAsync(out, p.out, sizeof(out), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) rc = fail(MLMC_ECUDA, "cudaMemcpyAsync failed: %s", cudaGetErrorString(e));
        }
        cudaFreeAsync(ws, st);
        e = cudaStreamSynchronize(st);
        if (!rc && e != cudaSuccess) rc = fail(MLMC_ECUDA, "level kernel failed: %s", cudaGetErrorString(e));
        if (rc) return rc;
    }
    std::memcpy(sums, out, sizeof(out));
    *cost = (double)N * problem_cost(level, M, payoff);
    return MLMC_OK;
}

int mlmc_level_sums(int level, int M, uint64_t N, const mlmc_model *model,
                    const mlmc_payoff *payoff, uint64_t seed, double sums[4], double *cost)
{
    return mlmc_level_sums_ex(level, M, N, 0, model, payoff, seed, MLMC_FP32_PATH, MLMC_TAG_PATHS,
                              nullptr, nullptr, sums, cost);
}

}  // extern "C"

// ------------------------------------------------------------------ adaptive driver (Sec. 5)

namespace mlmcgb {

int check_estimate_args(double eps, int M, int Lmin, int Lmax, uint64_t N0, int precision)
{
    if (!(eps > 0) || !std::isfinite(eps)) return fail(MLMC_EINVAL, "eps must be positive and finite");
    if (M != 2 && M != 4 && M != 8) return fail(MLMC_EINVAL, "M must be 2, 4 or 8");
    if (Lmin < 1 || Lmax < Lmin || Lmax >= MLMC_MAX_LEVELS || ipow(M, Lmax) > (1L << 24))
        return fail(MLMC_EINVAL, "need 1 <= Lmin <= Lmax < %d and M^Lmax <= 2^24", MLMC_MAX_LEVELS);
    if (N0 < 2) return fail(MLMC_EINVAL, "N0 must be at least 2");
    if (precision != MLMC_FP64 && precision != MLMC_FP32_PATH && precision != MLMC_FP64_STREAM32)
        return fail(MLMC_EINVAL, "precision must be MLMC_FP64, MLMC_FP32_PATH or MLMC_FP64_STREAM32");
    return MLMC_OK;
}

}  // namespace mlmcgb

extern "C" int mlmc_estimate(double eps, int M, int Lmin, int Lmax, uint64_t N0,
                             const mlmc_model *model, const mlmc_payoff *payoff, uint64_t seed,
                             int precision, void *stream, mlmc_result *out)
{
    const auto t_start = std::chrono::steady_clock::now();
    int rc = check_problem(model, payoff);
    if (rc) return rc;
    if (!out) return fail(MLMC_EINVAL, "out must not be NULL");
    rc = check_estimate_args(eps, M, Lmin, Lmax, N0, precision);
    if (rc) return rc;
    if (payoff->estimator != MLMC_COUPLED && payoff->estimator != MLMC_ANTITHETIC)
        return fail(MLMC_EINVAL, "the adaptive driver needs the coupled or antithetic estimator");
    cudaStream_t st = (cudaStream_t)stream;

    // rounds on the device (one graph launch) unless the host is asked for or must run them
    const int mode = graph_driver_mode();
    if (mode != MLMC_DRIVER_HOST) {
        if (!graph_driver_covers(model, payoff)) {
            if (mode == MLMC_DRIVER_DEVICE)
                return fail(MLMC_ENOTIMPL, "device-side rounds cover GBM with the coupled or antithetic estimator");
        } else {
            rc = estimate_on_device(eps, M, Lmin, Lmax, N0, model, payoff, seed, precision, st, out, t_start);
            if (rc != MLMC_ENOTIMPL || mode == MLMC_DRIVER_DEVICE) return rc;
        }
    }

    // A round's level launches go round-robin over `st` and the set's own streams, deepest level
    // first: the blocks of the next launch fill the SMs that one launch's last partial wave
    // leaves idle, and a round of a few small launches runs them side by side.  Stream k owns
    // workspace slot k (launches on one stream are ordered); the streams fork from `st` after
    // the round's first event and join it before the sums are copied back, so `st` orders the
    // whole call as before.  Each launch reduces its own sums in a fixed order, so the results
    // do not depend on how the launches overlap.
    int sms = 0;
    rc = device_sms(&sms);
    if (rc) return rc;
    const int ws_blocks = sms * 32;
    const size_t ws_slot = (workspace_bytes_for_blocks(ws_blocks) + 255) / 256 * 256;
    DriverScratch *sc = nullptr;
    rc = acquire_scratch(ws_slot * kDriverStreams, &sc);
    if (rc) return rc;
    double *d_sums = sc->d_sums, *h_sums = sc->h_sums;
    cudaEvent_t ev0 = sc->ev0, ev1 = sc->ev1;
    RoundStreams rs(sc, st, ws_slot);
    auto cleanup = [&]() { release_scratch(sc); };
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        free_scratch(sc);
        return fail(MLMC_ECUDA, "%s failed: %s", what, cudaGetErrorString(e));
    };
    // the completion tickets are zero after every finished launch; clear them in case an earlier
    // call on this set stopped between a launch and its completion
    cudaError_t e = rs.clear_tickets(kTicketBytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

    AdaptiveMLMC drv(eps, M, Lmin, Lmax, N0);
    if (payoff->estimator == MLMC_ANTITHETIC)  // two fine paths per sample: 2 M^l + M^(l-1) steps
        for (int l = 1; l < MLMC_MAX_LEVELS; ++l) drv.set_cost_scale(l, (2.0 * M + 1.0) / (M + 1.0));
    double kernel_ms = 0.0;
    uint64_t launches = 0, d2h_bytes = 0;
    while (drv.active()) {
        const std::vector<uint64_t> dN = drv.next_samples();
        const int L = drv.finest_level();
        if ((e = cudaEventRecord(ev0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = rs.fork(sc)) != cudaSuccess) return cuda_fail(e, "fork of the round's streams");
        for (int l = L; l >= 0; --l) {
            if (!dN[l]) continue;
            Plan plan;
            rc = plan_problem(l, M, dN[l], precision, model, payoff, nullptr, &plan);
            if (!rc && plan.blocks > ws_blocks) plan.blocks = ws_blocks;
            if (rc) {
                free_scratch(sc);  // waits for the launches already queued on the set's streams
                return rc;
            }
            LevelParams p;
            fill_params(p, l, M, dN[l], drv.samples_taken(l), model, payoff, seed, MLMC_TAG_PATHS, plan.lanes,
                        precision);
            p.out = d_sums + 4 * l;
            const int k = rs.take();
            rc = launch_level(plan, p, rs.slot[k], rs.stream[k]);
            if (rc) {
                free_scratch(sc);  // waits for the launches already queued on the set's streams
                return rc;
            }
            ++launches;
        }
        if ((e = rs.join(sc)) != cudaSuccess) return cuda_fail(e, "join of the round's streams");
        if ((e = cudaEventRecord(ev1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        e = cudaMemcpyAsync(h_sums, d_sums, (L + 1) * 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
        d2h_bytes += (L + 1) * 4 * sizeof(double);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "level round");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) kernel_ms += ms;
        for (int l = 0; l <= L; ++l) {
            if (!dN[l]) continue;
            for (int k = 0; k < 4; ++k) {
                if (!std::isfinite(h_sums[4 * l + k])) {
                    cleanup();
                    return fail(MLMC_ENONFINITE, "level %d sums are not finite (the scheme diverged)", l);
                }
            }
        }
        drv.absorb(h_sums);
    }
    cleanup();

    std::memset(out, 0, sizeof(*out));
    drv.fill(out);
    out->kernel_ms = kernel_ms;
    out->launches = launches;
    out->d2h_bytes = d2h_bytes;
    out->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (!out->converged) {
        fail(MLMC_ENOTCONV, "bias test still failing at Lmax = %d", Lmax);
        return MLMC_ENOTCONV;
    }
    return MLMC_OK;
}
