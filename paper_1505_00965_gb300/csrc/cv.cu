// cv.cu -- the learned control variate: training on the GPU, the control-variate level and mean
// estimators, and the adaptive driver that uses them (host side of the C ABI).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cv_kernels.cuh"
#include "train_kernel.cuh"
#include "driver.h"
#include "engine.h"
#include "host.h"
#include "mlmc.h"

using namespace mlmcgb;

struct mlmc_cv {
    int M;
    mlmc_model model;
    mlmc_payoff payoff;
    int device;
    float *d_params[MLMC_CV_MAX_LEVELS];
    float h_params[MLMC_CV_MAX_LEVELS][kNumParams];
    mlmc_cv_level_info info[MLMC_CV_MAX_LEVELS];
    mlmc_cv_train_stats train;  // zero unless made by mlmc_cv_train
};

namespace {

static_assert(kNumParams == MLMC_CV_PARAMS && kInputs == MLMC_CV_INPUTS, "network shape of the C ABI");
constexpr int kCvThreads = 256;
constexpr double kMinKappa = 1.0 / 64.0, kMaxKappa = 4096.0;  // mean points per path sample

const void *cv_data_kernel_for(int payoff)
{
    switch (payoff) {
    case kEuropean: return (const void *)cv_data_kernel<kEuropean>;
    case kAsian: return (const void *)cv_data_kernel<kAsian>;
    case kLookback: return (const void *)cv_data_kernel<kLookback>;
    case kDigital: return (const void *)cv_data_kernel<kDigital>;
    case kLinear: return (const void *)cv_data_kernel<kLinear>;
    case kGeoAsian: return (const void *)cv_data_kernel<kGeoAsian>;
    default: return nullptr;
    }
}

int grid_for(const void *kernel, uint64_t items, int *blocks)
{
    int resident = 0;
    int rc = max_resident_blocks(kernel, kCvThreads, &resident);
    if (rc) return rc;
    const double need = std::ceil((double)std::max<uint64_t>(items, 1) / kCvThreads);
    *blocks = (int)std::max(1.0, std::min<double>(need, resident));
    return MLMC_OK;
}

// Grid of the tcgen05 level kernel, in waves of the blocks an SM holds by shared memory,
// registers, threads and tensor memory (64 columns of 512 per block).  The occupancy query reports
// one block per SM for this kernel although six run at once (a launch of six blocks per SM runs
// 2.2 times faster than one of one block per SM), so the count comes from the kernel's attributes.
// Up to four waves when every block still gets at least 32 tiles (the blocks of an SM then fall
// out of step: 5% faster than one wave at 4e7 samples); one wave otherwise, since each block pays
// for loading the network and for the FP64 warp reductions of its eight sums (with 8.6 tiles per
// block these kept the FP64 pipe 20% busy).
int cv_level_grid(int payoff, int level, int M, uint64_t items, int *blocks)
{
    const void *k = cv_level_kernel_fp32(payoff, level, M);
    if (!k) return fail(MLMC_EINVAL, "payoff %d has no control-variate kernel", payoff);
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, reserved = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    cudaFuncAttributes fa;
    CUDA_TRY(cudaFuncGetAttributes(&fa, k));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const int warps = kCvTcThreads / 32;
    const int regs_block = warps * ((fa.numRegs * 32 + 255) / 256) * 256;  // 256-register warp granules
    int per_sm = std::min({smem_sm / std::max(1, (int)fa.sharedSizeBytes + reserved), regs_sm / std::max(1, regs_block),
                           thr_sm / kCvTcThreads, 512 / (int)kTcCols});
    per_sm = std::max(per_sm, 1);
    const double need = std::ceil((double)std::max<uint64_t>(items, 1) / kCvTcThreads);
    const double slots = (double)per_sm * sms;
    const double waves = std::min(4.0, std::max(1.0, std::floor(need / (32.0 * slots))));
    *blocks = (int)std::max(1.0, std::min(need, waves * slots));
    return MLMC_OK;
}

// Workspace for a kernel that sums NV doubles: ticket word (256 bytes) then NV per block.
size_t sums_workspace(int blocks, int nv) { return kTicketBytes + (size_t)blocks * nv * sizeof(double); }

int check_cv_level(const mlmc_cv *cv, int level)
{
    if (!cv) return fail(MLMC_EINVAL, "cv must not be NULL");
    if (level < 0 || level >= MLMC_CV_MAX_LEVELS) return fail(MLMC_EINVAL, "level %d outside 0..%d", level,
                                                              MLMC_CV_MAX_LEVELS - 1);
    return MLMC_OK;
}

int check_trained(const mlmc_cv *cv, int level)
{
    int rc = check_cv_level(cv, level);
    if (rc) return rc;
    if (!cv->d_params[level]) return fail(MLMC_EINVAL, "level %d has no network", level);
    return MLMC_OK;
}

// Launch the control-variate level kernel; ws holds sums_workspace(blocks, 8) bytes with a zero
// ticket.
int launch_cv_level(const mlmc_cv *cv, int level, uint64_t N, uint64_t first, uint64_t seed, double *d_sums8,
                    float *d_r, float *d_g, void *ws, int blocks, cudaStream_t st)
{
    LevelParams p;
    fill_params(p, level, cv->M, N, first, &cv->model, &cv->payoff, seed, MLMC_TAG_PATHS, 1, MLMC_FP32_PATH);
    p.ticket = (unsigned *)ws;
    p.partials = (double *)((char *)ws + kTicketBytes);
    const float *params = cv->d_params[level];
    void *args[] = {&p, (void *)&params, &d_sums8, &d_r, &d_g};
    CUDA_TRY(cudaLaunchKernel(cv_level_kernel_fp32(cv->payoff.kind, level, cv->M), dim3(blocks), dim3(kCvTcThreads), args, 0, st));
    return MLMC_OK;
}

// Replicates a launch of the lattice mean kernel can take in a workspace of ws_bytes: one FP64
// partial per block, kChunksPerReplicate blocks per replicate.
uint64_t mean_replicates_per_launch(size_t ws_bytes)
{
    return ws_bytes > kTicketBytes ? (ws_bytes - kTicketBytes) / (sizeof(double) * kChunksPerReplicate) : 0;
}

// Lattice mean sample: replicates [first, first + R) of `level`; d_sums2 = (sum Q_r, sum Q_r^2)
// (added to its old values when `accumulate` is set); d_g [R][n] or NULL.  ws (ws_bytes, zero
// ticket) holds the block partials; more replicates than fit run as consecutive launches.
int launch_cv_mean(const mlmc_cv *cv, int level, uint64_t R, uint64_t first, uint64_t seed, double *d_sums2,
                   float *d_g, void *ws, size_t ws_bytes, bool accumulate, cudaStream_t st)
{
    const uint64_t cap = mean_replicates_per_launch(ws_bytes);
    if (!cap) return fail(MLMC_EINVAL, "workspace too small for one replicate");
    for (uint64_t done = 0; done < R;) {
        const uint64_t nr = std::min(cap, R - done);
        LevelParams p;
        fill_params(p, level, cv->M, nr, first + done, &cv->model, &cv->payoff, seed, MLMC_TAG_CV_MEAN, 1,
                    MLMC_FP32_PATH);
        p.ticket = (unsigned *)ws;
        p.partials = (double *)((char *)ws + kTicketBytes);
        const float *params = cv->d_params[level];
        float *g = d_g ? d_g + done * kLatticeN : nullptr;
        int acc = (accumulate || done > 0) ? 1 : 0;
        void *args[] = {&p, (void *)&params, &d_sums2, &g, &acc};
        CUDA_TRY(cudaLaunchKernel((const void *)cv_mean_tc_kernel, dim3((unsigned)(nr * kChunksPerReplicate)),
                                  dim3(kMeanTcThreads), args, 0, st));
        done += nr;
    }
    return MLMC_OK;
}

// Replicates of the lattice mean sample that go with dN path samples at ratio kappa (mean
// points per path sample), at least kMinReplicates in all.
constexpr uint64_t kMinReplicates = 8;
uint64_t mean_replicates(double kappa, uint64_t dN, uint64_t have)
{
    uint64_t dR = (uint64_t)std::ceil(kappa * (double)dN / (double)kLatticeN);
    if (have + dR < kMinReplicates) dR = kMinReplicates - have;
    return dR;
}

// Run `body(ws)` with a zeroed stream-ordered workspace of `bytes`, then synchronise.
template <class F> int with_workspace(size_t bytes, cudaStream_t st, F body)
{
    void *ws = nullptr;
    CUDA_TRY(cudaMallocAsync(&ws, bytes, st));
    cudaError_t e = cudaMemsetAsync(ws, 0, bytes, st);
    int rc = e == cudaSuccess ? body(ws) : fail(MLMC_ECUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
    cudaFreeAsync(ws, st);
    e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = fail(MLMC_ECUDA, "control-variate kernel failed: %s", cudaGetErrorString(e));
    return rc;
}

// Initial weights: uniform in +-1/sqrt(fan-in) from a splitmix64 sequence; biases zero.
void init_params(float *w, uint64_t seed)
{
    uint64_t state = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1p-53 * 2.0 - 1.0;
    };
    std::fill(w, w + kNumParams, 0.f);
    for (int i = 0; i < kHidden * kInputs; ++i) w[kOffW1 + i] = (float)(next() / std::sqrt((double)kInputs));
    for (int i = 0; i < kHidden * kHidden; ++i) w[kOffW2 + i] = (float)(next() / std::sqrt((double)kHidden));
    for (int i = 0; i < kHidden; ++i) w[kOffW3 + i] = (float)(next() / std::sqrt((double)kHidden));
}

// Launch the training kernel (train) or one gradient evaluation (!train) for `jobs` networks, one
// thread-block cluster of `cluster` CTAs each.
int launch_training(const TrainArgs &args, int jobs, int cluster, bool train, cudaStream_t st)
{
    const void *k = train ? (const void *)train_cluster_kernel<true> : (const void *)train_cluster_kernel<false>;
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)));
    if (cluster > 8) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cluster * jobs));
    cfg.blockDim = dim3(kTrainThreads);
    cfg.dynamicSmemBytes = sizeof(TrainSmem);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TrainArgs a = args;
    void *kargs[] = {&a};
    CUDA_TRY(cudaLaunchKernelExC(&cfg, k, kargs));
    return MLMC_OK;
}

// Whether a cluster of `cluster` training CTAs fits on this GPU (the SMs of one GPC must hold it).
bool training_cluster_fits(int cluster, bool train)
{
    const void *k = train ? (const void *)train_cluster_kernel<true> : (const void *)train_cluster_kernel<false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)) != cudaSuccess)
        return false;
    if (cluster > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3(kTrainThreads);
    cfg.dynamicSmemBytes = sizeof(TrainSmem);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

// Largest cluster (16, 8, 4 or 2 CTAs; at least `least`) that fits and splits B rows into slices
// of whole 16-row tiles; 0 if none.
int training_cluster(int B, int least, bool train)
{
    for (int c = kTrainMaxCluster; c >= least; c /= 2)
        if (B % (16 * c) == 0 && training_cluster_fits(c, train)) return c;
    return 0;
}

double seconds_per_sample(cudaEvent_t a, cudaEvent_t b, uint64_t n)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms * 1e-3 / (double)n;
}

}  // namespace

extern "C" {

int mlmc_cv_create(int M, const mlmc_model *model, const mlmc_payoff *payoff, mlmc_cv **out)
{
    int rc = check_problem(model, payoff);
    if (rc) return rc;
    if (model->kind != MLMC_MODEL_GBM) return fail(MLMC_ENOTIMPL, "the control variate is built for GBM");
    if (model->scheme != MLMC_EULER_MARUYAMA || payoff->estimator != MLMC_COUPLED)
        return fail(MLMC_EINVAL, "the control variate runs the coupled Euler--Maruyama estimator");
    if (M != 2 && M != 4 && M != 8) return fail(MLMC_EINVAL, "M must be 2, 4 or 8");
    if (!out) return fail(MLMC_EINVAL, "out must not be NULL");
    mlmc_cv *cv = new (std::nothrow) mlmc_cv();
    if (!cv) return fail(MLMC_ENOMEM, "cannot allocate the control-variate handle");
    cv->M = M;
    cv->model = *model;
    cv->payoff = *payoff;
    cudaError_t e = cudaGetDevice(&cv->device);
    if (e != cudaSuccess) {
        delete cv;
        return fail(MLMC_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    }
    *out = cv;
    return MLMC_OK;
}

int mlmc_cv_free(mlmc_cv *cv)
{
    if (!cv) return MLMC_OK;
    for (int l = 0; l < MLMC_CV_MAX_LEVELS; ++l)
        if (cv->d_params[l]) cudaFree(cv->d_params[l]);
    delete cv;
    return MLMC_OK;
}

int mlmc_cv_info(const mlmc_cv *cv, int level, mlmc_cv_level_info *out)
{
    int rc = check_cv_level(cv, level);
    if (rc) return rc;
    if (!out) return fail(MLMC_EINVAL, "out must not be NULL");
    *out = cv->info[level];
    return MLMC_OK;
}

int mlmc_cv_get_params(const mlmc_cv *cv, int level, float *params)
{
    int rc = check_trained(cv, level);
    if (rc) return rc;
    if (!params) return fail(MLMC_EINVAL, "params must not be NULL");
    std::memcpy(params, cv->h_params[level], sizeof(float) * kNumParams);
    return MLMC_OK;
}

int mlmc_cv_set_params(mlmc_cv *cv, int level, const float *params, double kappa)
{
    int rc = check_cv_level(cv, level);
    if (rc) return rc;
    if (!params) return fail(MLMC_EINVAL, "params must not be NULL");
    if (!(kappa >= kMinKappa && kappa <= kMaxKappa))
        return fail(MLMC_EINVAL, "kappa must lie in [%g, %g]", kMinKappa, kMaxKappa);
    if (!cv->d_params[level]) CUDA_TRY(cudaMalloc(&cv->d_params[level], sizeof(float) * kNumParams));
    CUDA_TRY(cudaMemcpy(cv->d_params[level], params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
    std::memcpy(cv->h_params[level], params, sizeof(float) * kNumParams);
    cv->info[level] = mlmc_cv_level_info();
    cv->info[level].trained = 1;
    cv->info[level].used = 1;
    cv->info[level].kappa = kappa;
    return MLMC_OK;
}

int mlmc_cv_level_sums(const mlmc_cv *cv, int level, uint64_t N, uint64_t first, uint64_t seed, double *d_sums8,
                       float *d_r, float *d_g, void *stream)
{
    int rc = check_trained(cv, level);
    if (rc) return rc;
    if (!d_sums8) return fail(MLMC_EINVAL, "d_sums8 must not be NULL");
    if (first + N < first) return fail(MLMC_EINVAL, "first + N overflows 64 bits");
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0) {
        CUDA_TRY(cudaMemsetAsync(d_sums8, 0, 8 * sizeof(double), st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return MLMC_OK;
    }
    int blocks = 0;
    rc = cv_level_grid(cv->payoff.kind, level, cv->M, N, &blocks);
    if (rc) return rc;
    return with_workspace(sums_workspace(blocks, 8), st, [&](void *ws) {
        return launch_cv_level(cv, level, N, first, seed, d_sums8, d_r, d_g, ws, blocks, st);
    });
}

int mlmc_cv_mean_sums(const mlmc_cv *cv, int level, uint64_t R, uint64_t first, uint64_t seed, double *d_sums2,
                      float *d_g, void *stream)
{
    int rc = check_trained(cv, level);
    if (rc) return rc;
    if (!d_sums2) return fail(MLMC_EINVAL, "d_sums2 must not be NULL");
    if (first + R < first) return fail(MLMC_EINVAL, "first + R overflows 64 bits");
    cudaStream_t st = (cudaStream_t)stream;
    if (R == 0) {
        CUDA_TRY(cudaMemsetAsync(d_sums2, 0, 2 * sizeof(double), st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return MLMC_OK;
    }
    const size_t bytes = kTicketBytes + std::min<uint64_t>(R, 1024) * kChunksPerReplicate * sizeof(double);
    return with_workspace(bytes, st, [&](void *ws) {
        return launch_cv_mean(cv, level, R, first, seed, d_sums2, d_g, ws, bytes, false, st);
    });
}

int mlmc_cv_training_data(const mlmc_cv *cv, int level, uint64_t N, uint64_t first, uint64_t seed, float *d_X,
                          float *d_Y, void *stream)
{
    int rc = check_cv_level(cv, level);
    if (rc) return rc;
    if (!d_X || !d_Y) return fail(MLMC_EINVAL, "d_X and d_Y must not be NULL");
    if (first + N < first) return fail(MLMC_EINVAL, "first + N overflows 64 bits");
    if (ipow(cv->M, level) > (1L << 24)) return fail(MLMC_EINVAL, "level %d too deep", level);
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0) return MLMC_OK;
    const void *k = cv_data_kernel_for(cv->payoff.kind);
    int blocks = 0;
    rc = grid_for(k, N, &blocks);
    if (rc) return rc;
    LevelParams p;
    fill_params(p, level, cv->M, N, first, &cv->model, &cv->payoff, seed, MLMC_TAG_CV_TRAIN, 1, MLMC_FP32_PATH);
    void *args[] = {&p, &d_X, &d_Y};
    CUDA_TRY(cudaLaunchKernel(k, dim3(blocks), dim3(kCvThreads), args, 0, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return MLMC_OK;
}

int mlmc_mlp_forward(const float *params, const float *d_X, uint64_t N, float *d_G, void *stream)
{
    if (!params || !d_X || !d_G) return fail(MLMC_EINVAL, "params, d_X and d_G must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (N == 0) return MLMC_OK;
    int blocks = 0;
    int rc = grid_for((const void *)mlp_forward_kernel, N, &blocks);
    if (rc) return rc;
    float *d_params = nullptr;
    CUDA_TRY(cudaMallocAsync(&d_params, sizeof(float) * kNumParams, st));
    cudaError_t e = cudaMemcpyAsync(d_params, params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, st);
    const float *cp = d_params;
    void *args[] = {(void *)&cp, (void *)&d_X, &N, &d_G};
    if (e == cudaSuccess) e = cudaLaunchKernel((const void *)mlp_forward_kernel, dim3(blocks), dim3(kCvThreads), args, 0, st);
    cudaFreeAsync(d_params, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(MLMC_ECUDA, "network forward failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return MLMC_OK;
}

int mlmc_mlp_grad(const float *params, const float *d_X, const float *d_Y, uint64_t N, float *grad, double *loss,
                  void *stream)
{
    if (!params || !d_X || !d_Y || !grad || !loss) return fail(MLMC_EINVAL, "NULL argument");
    if (N == 0 || N % 32 || N > 65536) return fail(MLMC_EINVAL, "N must be a positive multiple of 32, at most 65536");
    cudaStream_t st = (cudaStream_t)stream;
    const int cluster = training_cluster((int)N, 2, false);
    if (!cluster) return fail(MLMC_ECUDA, "no thread-block cluster for the gradient kernel fits this GPU");
    float *d_buf = nullptr;  // parameters, gradient, then N outputs g
    CUDA_TRY(cudaMallocAsync(&d_buf, sizeof(float) * (2 * kNumParams + N), st));
    TrainArgs a = {};
    a.job[0] = TrainJob{d_X, d_Y, d_buf, 0.f, 1.f};
    a.B = (int)N;
    a.steps = 1;
    a.epochs = 1;
    a.lr = 0.f;
    a.grad_out = d_buf + kNumParams;
    a.g_out = d_buf + 2 * kNumParams;
    std::vector<float> g(N), y(N);
    cudaError_t e = cudaMemcpyAsync(d_buf, params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, st);
    int rc = e == cudaSuccess ? launch_training(a, 1, cluster, false, st)
                              : fail(MLMC_ECUDA, "upload failed: %s", cudaGetErrorString(e));
    if (!rc) {
        e = cudaMemcpyAsync(grad, a.grad_out, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.data(), a.g_out, sizeof(float) * N, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(y.data(), d_Y, sizeof(float) * N, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(MLMC_ECUDA, "network gradient failed: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(d_buf, st);
    if (rc) return rc;
    double acc = 0.0;
    for (uint64_t i = 0; i < N; ++i) acc += ((double)g[i] - y[i]) * ((double)g[i] - y[i]);
    *loss = acc / (double)N;
    return MLMC_OK;
}

int mlmc_cv_train(int M, const mlmc_model *model, const mlmc_payoff *payoff, uint64_t seed,
                  const mlmc_cv_options *opts, void *stream, mlmc_cv **out)
{
    if (!out) return fail(MLMC_EINVAL, "out must not be NULL");
    mlmc_cv_options o = opts ? *opts : mlmc_cv_options();
    if (o.reserved != 0) return fail(MLMC_EINVAL, "mlmc_cv_options.reserved must be 0");
    const int levels = o.levels ? o.levels : 4;
    const int epochs = o.epochs ? o.epochs : 20;
    const int B = o.batch ? o.batch : 4096;
    const uint64_t n_train = o.n_train ? o.n_train : 1000000;
    const float lr = (float)(o.lr > 0 ? o.lr : 1e-3);
    if (levels < 1 || levels > MLMC_CV_MAX_LEVELS) return fail(MLMC_EINVAL, "levels must be 1..%d", MLMC_CV_MAX_LEVELS);
    if (epochs < 1 || B < 256 || B % 256 || B > 65536) return fail(MLMC_EINVAL, "need epochs >= 1 and batch a multiple of 256 up to 65536");
    const uint64_t n_fit = n_train / 10 * 9, n_val = n_train - n_fit;
    if (n_fit < (uint64_t)B || n_val < 256) return fail(MLMC_EINVAL, "n_train too small for the batch size");
    if (ipow(M, levels - 1) > (1L << 16)) return fail(MLMC_EINVAL, "levels too deep for training");
    mlmc_cv *cv = nullptr;
    int rc = mlmc_cv_create(M, model, payoff, &cv);
    if (rc) return rc;
    // training runs on a private stream once `stream` has drained
    const auto t_begin = std::chrono::steady_clock::now();
    cudaStream_t st = nullptr;
    {
        cudaError_t e0 = cudaStreamSynchronize((cudaStream_t)stream);
        if (e0 == cudaSuccess) e0 = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e0 != cudaSuccess) {
            mlmc_cv_free(cv);
            return fail(MLMC_ECUDA, "training stream: %s", cudaGetErrorString(e0));
        }
    }
    const int cluster = training_cluster(B, kTrainMinClusterAdam, true);
    if (!cluster) {
        cudaStreamDestroy(st);
        mlmc_cv_free(cv);
        return fail(MLMC_ECUDA, "no thread-block cluster of %d or more training CTAs fits this GPU", kTrainMinClusterAdam);
    }
    float *d_X = nullptr, *d_Y = nullptr, *d_Gv = nullptr, *d_P = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    auto cleanup = [&](int code) {
        if (d_X) cudaFree(d_X);
        if (d_Y) cudaFree(d_Y);
        if (d_Gv) cudaFree(d_Gv);
        if (d_P) cudaFree(d_P);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (st) cudaStreamDestroy(st);
        st = nullptr;
        if (code) mlmc_cv_free(cv);
        return code;
    };
#define CV_TRY(expr)                                                                                \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess) return cleanup(fail(MLMC_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_))); \
    } while (0)
    CV_TRY(cudaMalloc(&d_X, sizeof(float) * kInputs * n_train * levels));
    CV_TRY(cudaMalloc(&d_Y, sizeof(float) * n_train * levels));
    CV_TRY(cudaMalloc(&d_Gv, sizeof(float) * n_train));
    CV_TRY(cudaMalloc(&d_P, sizeof(float) * kNumParams * levels));
    CV_TRY(cudaEventCreate(&ev0));
    CV_TRY(cudaEventCreate(&ev1));
    std::vector<float> hY(n_train * levels), hG(n_val);
    std::vector<double> mu(levels), sd(levels);
    // 1. training data of every level from the method itself (independent tag), target
    // standardisation, initial weights
    TrainArgs targs = {};
    for (int l = 0; l < levels; ++l) {
        float *X = d_X + kInputs * n_train * l, *Yd = d_Y + n_train * l;
        rc = mlmc_cv_training_data(cv, l, n_train, 0, seed, X, Yd, st);
        if (rc) return cleanup(rc);
        const float *hy = hY.data() + n_train * l;
        CV_TRY(cudaMemcpy((void *)hy, Yd, sizeof(float) * n_train, cudaMemcpyDeviceToHost));
        double m = 0.0, v = 0.0;
        for (uint64_t i = 0; i < n_fit; ++i) m += hy[i];
        m /= (double)n_fit;
        for (uint64_t i = 0; i < n_fit; ++i) v += (hy[i] - m) * (hy[i] - m);
        mu[l] = m;
        sd[l] = std::sqrt(std::max(v / (double)n_fit, 1e-300));
        float w[kNumParams];
        init_params(w, o.init_seed + 7919ull * (uint64_t)l);
        CV_TRY(cudaMemcpy(d_P + kNumParams * l, w, sizeof(w), cudaMemcpyHostToDevice));
        targs.job[l] = TrainJob{X, Yd, d_P + kNumParams * l, (float)m, (float)(1.0 / sd[l])};
    }
    const auto t_data = std::chrono::steady_clock::now();
    // 2. every level's network trained side by side: one cluster per level, one launch
    targs.B = B;
    targs.steps = (int)(n_fit / (uint64_t)B);
    targs.epochs = epochs;
    targs.lr = lr;
    CV_TRY(cudaEventRecord(ev0, st));
    rc = launch_training(targs, levels, cluster, true, st);
    if (rc) return cleanup(rc);
    CV_TRY(cudaEventRecord(ev1, st));
    CV_TRY(cudaEventSynchronize(ev1));
    float train_kernel_ms = 0.f;
    CV_TRY(cudaEventElapsedTime(&train_kernel_ms, ev0, ev1));
    const auto t_trained = std::chrono::steady_clock::now();
    double eval_ms = 0.0, cost_ms = 0.0;
    for (int l = 0; l < levels; ++l) {
        const auto t_eval0 = std::chrono::steady_clock::now();
        float w[kNumParams];
        // 4. undo the target standardisation in the last layer: g = sd * net + mu
        CV_TRY(cudaMemcpy(w, d_P + kNumParams * l, sizeof(w), cudaMemcpyDeviceToHost));
        for (int i = 0; i < kHidden; ++i) w[kOffW3 + i] = (float)(w[kOffW3 + i] * sd[l]);
        w[kOffB3] = (float)(w[kOffB3] * sd[l] + mu[l]);
        rc = mlmc_cv_set_params(cv, l, w, 1.0);
        if (rc) return cleanup(rc);
        const float *d_Xl = d_X + kInputs * n_train * l;
        const float *hYl = hY.data() + n_train * l;
        // 5. held-out variance ratio
        rc = mlmc_mlp_forward(w, d_Xl + kInputs * n_fit, n_val, d_Gv, st);
        if (rc) return cleanup(rc);
        CV_TRY(cudaMemcpy(hG.data(), d_Gv, sizeof(float) * n_val, cudaMemcpyDeviceToHost));
        double sy = 0, syy = 0, sr = 0, srr = 0, sg = 0, sgg = 0;
        for (uint64_t i = 0; i < n_val; ++i) {
            const double y = hYl[n_fit + i], g = hG[i], r = y - g;
            sy += y; syy += y * y; sr += r; srr += r * r; sg += g; sgg += g * g;
        }
        const double nv = (double)n_val;
        mlmc_cv_level_info &inf = cv->info[l];
        inf.var_plain = std::max(syy / nv - (sy / nv) * (sy / nv), 0.0);
        inf.var_resid = std::max(srr / nv - (sr / nv) * (sr / nv), 0.0);
        inf.var_g = std::max(sgg / nv - (sg / nv) * (sg / nv), 0.0);
        inf.train_loss = inf.var_resid / (sd[l] * sd[l]);
        const auto t_cost0 = std::chrono::steady_clock::now();
        eval_ms += std::chrono::duration<double, std::milli>(t_cost0 - t_eval0).count();
        // 6. measured cost per sample of the plain, control-variate and mean kernels, each timed
        // once after a small warm-up launch (sizes that keep every timed launch near half a
        // millisecond or more: small launches would measure launch latency and idle SMs, not the
        // cost per sample)
        const uint64_t nt = std::max<uint64_t>(1u << 21, (uint64_t)(1u << 29) >> std::min(2 * l, 20));
        const uint64_t nc = 1u << 23;
        constexpr uint64_t kWarmSamples = 4096, kWarmReplicates = 8;
        {
            Plan plan, warm_plan;
            rc = plan_level(l, M, nt, MLMC_FP32_PATH, payoff->kind, MLMC_EULER_MARUYAMA, nullptr, &plan);
            if (!rc) rc = plan_level(l, M, kWarmSamples, MLMC_FP32_PATH, payoff->kind, MLMC_EULER_MARUYAMA, nullptr,
                                     &warm_plan);
            if (rc) return cleanup(rc);
            int cvb = 0;
            rc = cv_level_grid(payoff->kind, l, M, nc, &cvb);
            if (rc) return cleanup(rc);
            // the lattice statistics use kStatReplicates replicates (2^23 points)
            constexpr uint64_t kStatReplicates = 128;
            const size_t wbytes = std::max<size_t>(sums_workspace(std::max(plan.blocks, cvb), 8),
                                                   kTicketBytes + kStatReplicates * kChunksPerReplicate * sizeof(double));
            double *d_out = nullptr;
            CV_TRY(cudaMalloc(&d_out, 16 * sizeof(double)));
            double hq[2] = {0.0, 0.0};
            rc = with_workspace(wbytes, st, [&](void *ws) {
                for (int rep = 0; rep < 2; ++rep) {  // a small warm-up pass (lazily loaded kernels), then the timed one
                    const Plan &pl = rep ? plan : warm_plan;
                    const uint64_t n1 = rep ? nt : kWarmSamples, n2 = rep ? nc : kWarmSamples;
                    const uint64_t R = rep ? kStatReplicates : kWarmReplicates;
                    LevelParams p;
                    fill_params(p, l, M, n1, 0, model, payoff, seed, MLMC_TAG_PATHS, pl.lanes, MLMC_FP32_PATH);
                    p.out = d_out;
                    CUDA_TRY(cudaEventRecord(ev0, st));
                    int r2 = launch_level(pl, p, ws, st);
                    if (r2) return r2;
                    CUDA_TRY(cudaEventRecord(ev1, st));
                    CUDA_TRY(cudaEventSynchronize(ev1));
                    inf.t_plain = seconds_per_sample(ev0, ev1, n1);
                    CUDA_TRY(cudaEventRecord(ev0, st));
                    r2 = launch_cv_level(cv, l, n2, 0, seed, d_out, nullptr, nullptr, ws, cvb, st);
                    if (r2) return r2;
                    CUDA_TRY(cudaEventRecord(ev1, st));
                    CUDA_TRY(cudaEventSynchronize(ev1));
                    inf.t_cv = seconds_per_sample(ev0, ev1, n2);
                    CUDA_TRY(cudaEventRecord(ev0, st));
                    // replicates far from those of any estimate (which count from 0)
                    r2 = launch_cv_mean(cv, l, R, 1ull << 40, seed, d_out + 8, nullptr, ws, wbytes, false, st);
                    if (r2) return r2;
                    CUDA_TRY(cudaEventRecord(ev1, st));
                    CUDA_TRY(cudaEventSynchronize(ev1));
                    inf.t_mean = seconds_per_sample(ev0, ev1, R * kLatticeN);
                }
                CUDA_TRY(cudaMemcpy(hq, d_out + 8, sizeof(hq), cudaMemcpyDeviceToHost));
                return (int)MLMC_OK;
            });
            cudaFree(d_out);
            if (rc) return cleanup(rc);
            // per-point variance of the lattice mean: n times the variance of a replicate mean
            const double R = (double)kStatReplicates, mq = hq[0] / R;
            inf.var_lattice = (double)kLatticeN * std::max(hq[1] - R * mq * mq, 0.0) / (R - 1.0);
        }
        // 7. mean points per path sample minimising (Vr + Vq / k)(t_cv + k t_mean), Vq the
        // per-point variance of the lattice mean, and the decision
        const double vr = std::max(inf.var_resid, 1e-300);
        double kappa = std::sqrt(inf.var_lattice * inf.t_cv / (vr * std::max(inf.t_mean, 1e-15)));
        kappa = std::min(std::max(kappa, kMinKappa), kMaxKappa);
        inf.kappa = kappa;
        inf.work_ratio = (inf.var_resid + inf.var_lattice / kappa) * (inf.t_cv + kappa * inf.t_mean) /
                         std::max(inf.var_plain * inf.t_plain, 1e-300);
        inf.used = inf.work_ratio < 1.0 ? 1 : 0;
        inf.trained = 1;
        cost_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_cost0).count();
    }
#undef CV_TRY
    cleanup(MLMC_OK);
    mlmc_cv_train_stats &ts = cv->train;
    ts.data_ms = std::chrono::duration<double, std::milli>(t_data - t_begin).count();
    ts.train_ms = std::chrono::duration<double, std::milli>(t_trained - t_data).count();
    ts.train_kernel_ms = train_kernel_ms;
    ts.eval_ms = eval_ms;
    ts.cost_ms = cost_ms;
    ts.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_begin).count();
    ts.steps = (int64_t)targs.steps * epochs;
    ts.cluster = cluster;
    ts.levels = levels;
    *out = cv;
    return MLMC_OK;
}

int mlmc_cv_train_info(const mlmc_cv *cv, mlmc_cv_train_stats *out)
{
    if (!cv || !out) return fail(MLMC_EINVAL, "cv and out must not be NULL");
    *out = cv->train;
    return MLMC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ estimate with the control variate

extern "C" int mlmc_estimate_cv(double eps, int M, int Lmin, int Lmax, uint64_t N0, const mlmc_model *model,
                                const mlmc_payoff *payoff, uint64_t seed, const mlmc_cv *cv, void *stream,
                                mlmc_result *out)
{
    const auto t_start = std::chrono::steady_clock::now();
    int rc = check_problem(model, payoff);
    if (rc) return rc;
    if (model->kind != MLMC_MODEL_GBM) return fail(MLMC_ENOTIMPL, "the control variate is built for GBM");
    if (!out || !cv) return fail(MLMC_EINVAL, "out and cv must not be NULL");
    rc = check_estimate_args(eps, M, Lmin, Lmax, N0, MLMC_FP32_PATH);
    if (rc) return rc;
    if (cv->M != M || std::memcmp(&cv->model, model, sizeof(*model)) ||
        std::memcmp(&cv->payoff, payoff, sizeof(*payoff)))
        return fail(MLMC_EINVAL, "the control variate was made for another problem");
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0;
    rc = device_sms(&sms);
    if (rc) return rc;
    const int ws_blocks = sms * 32;
    const size_t ws_bytes = sums_workspace(ws_blocks, 8);
    const int stride = 16;  // doubles per level in the round buffer: 8 level sums + 2 mean sums
    static_assert(stride <= kDriverSumsPerLevel, "round buffer");
    // a round's launches spread over `st` and the set's own streams as in mlmc_estimate; a
    // control-variate level's path kernel and lattice-mean kernel take one turn each
    const size_t ws_slot = (ws_bytes + 255) / 256 * 256;
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
    cudaError_t e = rs.clear_tickets(kTicketBytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");

    AdaptiveMLMC drv(eps, M, Lmin, Lmax, N0);
    auto uses = [&](int l) { return l < MLMC_CV_MAX_LEVELS && cv->d_params[l] && cv->info[l].used; };
    // control-variate levels: cumulative sums of r, r^2 (N path samples) and of the lattice
    // replicate means Q, Q^2 (nrep replicates)
    std::vector<double> sr(MLMC_MAX_LEVELS, 0.0), srr(MLMC_MAX_LEVELS, 0.0), sq(MLMC_MAX_LEVELS, 0.0),
        sqq(MLMC_MAX_LEVELS, 0.0), vs0(MLMC_MAX_LEVELS, 0.0), vs1(MLMC_MAX_LEVELS, 0.0);
    std::vector<uint64_t> nrep(MLMC_MAX_LEVELS, 0), drep(MLMC_MAX_LEVELS, 0);
    for (int l = 0; l < MLMC_MAX_LEVELS; ++l)
        if (uses(l)) {
            const mlmc_cv_level_info &inf = cv->info[l];
            const double t_plain = inf.t_plain > 0 ? inf.t_plain : 1.0;
            const double t_cv = inf.t_cv > 0 ? inf.t_cv : 1.0, t_mean = inf.t_mean > 0 ? inf.t_mean : 1.0;
            drv.set_cost_scale(l, inf.t_plain > 0 ? (t_cv + inf.kappa * t_mean) / t_plain : 1.0 + inf.kappa);
        }
    std::vector<double> round(MLMC_MAX_LEVELS * 4);
    double kernel_ms = 0.0;
    uint64_t launches = 0, d2h_bytes = 0;
    while (drv.active()) {
        const std::vector<uint64_t> dN = drv.next_samples();
        const int L = drv.finest_level();
        if ((e = cudaEventRecord(ev0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = rs.fork(sc)) != cudaSuccess) return cuda_fail(e, "fork of the round's streams");
        for (int l = L; l >= 0; --l) {
            if (!dN[l]) continue;
            const int k = rs.take();
            void *ws = rs.slot[k];
            const cudaStream_t sk = rs.stream[k];
            if (uses(l)) {
                drep[l] = mean_replicates(cv->info[l].kappa, dN[l], nrep[l]);
                int cb = 0;
                rc = cv_level_grid(payoff->kind, l, M, dN[l], &cb);
                if (!rc)
                    rc = launch_cv_level(cv, l, dN[l], drv.samples_taken(l), seed, d_sums + stride * l, nullptr,
                                         nullptr, ws, std::min(cb, ws_blocks), sk);
                // the lattice mean is independent of the path kernel: the next stream and its slot
                const int km = rs.take();
                if (!rc)
                    rc = launch_cv_mean(cv, l, drep[l], nrep[l], seed, d_sums + stride * l + 8, nullptr, rs.slot[km],
                                        ws_bytes, false, rs.stream[km]);
                launches += 1 + (drep[l] + mean_replicates_per_launch(ws_bytes) - 1) / mean_replicates_per_launch(ws_bytes);
            } else {
                Plan plan;
                rc = plan_level(l, M, dN[l], MLMC_FP32_PATH, payoff->kind, MLMC_EULER_MARUYAMA, nullptr, &plan);
                if (!rc && plan.blocks > ws_blocks) plan.blocks = ws_blocks;
                if (!rc) {
                    LevelParams p;
                    fill_params(p, l, M, dN[l], drv.samples_taken(l), model, payoff, seed, MLMC_TAG_PATHS, plan.lanes,
                                MLMC_FP32_PATH);
                    p.out = d_sums + stride * l;
                    rc = launch_level(plan, p, ws, sk);
                }
                launches += 1;
            }
            if (rc) {
                free_scratch(sc);  // waits for the launches already queued on the set's streams
                return rc;
            }
        }
        if ((e = rs.join(sc)) != cudaSuccess) return cuda_fail(e, "join of the round's streams");
        if ((e = cudaEventRecord(ev1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        e = cudaMemcpyAsync(h_sums, d_sums, (L + 1) * stride * sizeof(double), cudaMemcpyDeviceToHost, st);
        d2h_bytes += (L + 1) * stride * sizeof(double);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "level round");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) kernel_ms += ms;
        std::fill(round.begin(), round.end(), 0.0);
        for (int l = 0; l <= L; ++l) {
            if (!dN[l]) continue;
            const double *h = h_sums + stride * l;
            if (uses(l)) {
                // level estimate mean(r) + mean of the replicate means Q: its variance per path
                // sample is Var(r) + N Var(Q) / R; hand the driver the sums of a sample with that
                // mean and variance (as differences from the previous round's totals)
                sr[l] += h[0];
                srr[l] += h[1];
                sq[l] += h[8];
                sqq[l] += h[9];
                nrep[l] += drep[l];
                const double n = (double)(drv.samples_taken(l) + dN[l]), R = (double)nrep[l];
                const double mr = sr[l] / n, mq = sq[l] / R;
                const double vr = std::max(srr[l] / n - mr * mr, 0.0);
                const double vq = R > 1.0 ? std::max(sqq[l] - R * mq * mq, 0.0) / (R - 1.0) : 0.0;
                const double m = mr + mq, v = vr + vq * n / R;
                const double s0 = n * m, s1 = n * (v + m * m);
                round[4 * l + 0] = s0 - vs0[l];
                round[4 * l + 1] = s1 - vs1[l];
                vs0[l] = s0;
                vs1[l] = s1;
            } else {
                for (int k = 0; k < 4; ++k) round[4 * l + k] = h[k];
            }
        }
        drv.absorb(round.data());
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
