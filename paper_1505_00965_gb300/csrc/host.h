// host.h -- host-side helpers shared by the C ABI translation units (defined in api.cu).
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <cstddef>
#include <cstdint>

#include "engine.h"
#include "mlmc.h"

namespace mlmcgb {

// Record a message for mlmc_last_error() on this host thread and return `code`.
int fail(int code, const char *fmt, ...);

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return ::mlmcgb::fail(MLMC_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

long ipow(long b, int e);
int check_problem(const mlmc_model *model, const mlmc_payoff *payoff);
int check_level(int level, int M);
int check_tag(int tag);
int device_sms(int *sms);
int max_resident_blocks(const void *kernel, int threads, int *out);

// Launch shape and kernel of one level.
struct Plan {
    const void *kernel;
    int threads, lanes, blocks;
    int ns = 1;  // samples per thread (2: the two-sample kernel)
};
int plan_level(int level, int M, uint64_t N, int precision, int payoff, int scheme, const mlmc_launch *launch,
               Plan *plan);
// plan_level for GBM, the one-thread-per-sample plan of the QUINTIC_ODE kernel otherwise.
// Whether every fine and coarse step factor 1 + d of a GBM path on this level is positive for any
// normal the stream can produce (the split lookback kernels then keep no running minimum).
bool positive_step_factors(const mlmc_model *m, int level, int M);
// Device-side rounds of mlmc_estimate (graph_driver.cu): mode, coverage, the estimate (MLMC_ENOTIMPL
// with nothing launched where the graph cannot be built), and release of a device's cached graphs.
int graph_driver_mode();
bool graph_driver_covers(const mlmc_model *model, const mlmc_payoff *payoff);
int estimate_on_device(double eps, int M, int Lmin, int Lmax, uint64_t N0, const mlmc_model *model,
                       const mlmc_payoff *payoff, uint64_t seed, int precision, cudaStream_t st, mlmc_result *out,
                       std::chrono::steady_clock::time_point t_start);
void graph_driver_release(int dev);
int plan_problem(int level, int M, uint64_t N, int precision, const mlmc_model *model, const mlmc_payoff *payoff,
                 const mlmc_launch *launch, Plan *plan);
void fill_params(LevelParams &p, int level, int M, uint64_t N, uint64_t first,
                 const mlmc_model *m, const mlmc_payoff *pay, uint64_t seed, int tag, int lanes, int precision);
double level_cost(int level, int M);
// Euler--Maruyama steps of one sample of the payoff's estimator (level_cost for the coupled one).
double problem_cost(int level, int M, const mlmc_payoff *payoff);
int launch_level(const Plan &plan, LevelParams &p, void *ws, cudaStream_t st);
int check_estimate_args(double eps, int M, int Lmin, int Lmax, uint64_t N0, int precision);

// Launch shape found by the autotuner for (precision, payoff, M, level) at the size class of N.
struct TunedShape {
    int threads, lanes, oversub;
    double ns_per_sample;
    int ns = 0;  // samples per thread (0 = not tuned: the planner's default)
};
bool tuned_lookup(int precision, int payoff, int M, int level, uint64_t N, TunedShape *out);

// Buffers of one adaptive-driver call, pooled per device between calls: a workspace of at least
// ws_bytes (zero tickets), device and pinned host sums (kDriverSumsPerLevel doubles per level),
// two timing events, and kDriverStreams - 1 streams with their fork and join events, over which
// (with the caller's stream) a round spreads its level launches.  acquire_scratch takes a set
// from the pool or makes one; release_scratch returns it; free_scratch destroys a set that met
// a CUDA error.
constexpr int kDriverSumsPerLevel = 16;
constexpr int kDriverStreams = 4;
struct DriverScratch {
    int device = -1;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    double *d_sums = nullptr;
    double *h_sums = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t aux[kDriverStreams - 1] = {};
    cudaEvent_t fork = nullptr, join[kDriverStreams - 1] = {};
};
int acquire_scratch(size_t ws_bytes, DriverScratch **out);
void release_scratch(DriverScratch *s);
void free_scratch(DriverScratch *s);

// The streams of one driver call and their workspace slots: slot k (slot_bytes from the set's
// workspace, which holds kDriverStreams of them) belongs to stream k, the caller's stream for
// k = 0 and the set's own streams after it, so launches that share a slot are ordered.  A round
// forks the set's streams from the caller's stream, takes streams in turn, and joins them back.
struct RoundStreams {
    cudaStream_t stream[kDriverStreams];
    void *slot[kDriverStreams];
    int next = 0;

    RoundStreams(const DriverScratch *sc, cudaStream_t st, size_t slot_bytes)
    {
        for (int k = 0; k < kDriverStreams; ++k) {
            stream[k] = k ? sc->aux[k - 1] : st;
            slot[k] = (char *)sc->ws + slot_bytes * k;
        }
    }
    // zero every slot's completion ticket (in the caller's stream's order)
    cudaError_t clear_tickets(size_t ticket_bytes) const
    {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kDriverStreams && e == cudaSuccess; ++k)
            e = cudaMemsetAsync(slot[k], 0, ticket_bytes, stream[0]);
        return e;
    }
    cudaError_t fork(const DriverScratch *sc)
    {
        next = 0;
        cudaError_t e = cudaEventRecord(sc->fork, stream[0]);
        for (int k = 1; k < kDriverStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(stream[k], sc->fork, 0);
        return e;
    }
    int take() { return next++ % kDriverStreams; }
    cudaError_t join(const DriverScratch *sc)
    {
        cudaError_t e = cudaSuccess;
        for (int k = 1; k < kDriverStreams && e == cudaSuccess; ++k) {
            e = cudaEventRecord(sc->join[k - 1], stream[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(stream[0], sc->join[k - 1], 0);
        }
        return e;
    }
};

}  // namespace mlmcgb
