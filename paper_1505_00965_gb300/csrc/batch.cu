// batch.cu -- many adaptive MLMC problems per round: chunk lists, the persistent kernel, the
// fixed-order reduction and the CUDA graph that replays each round.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "driver.h"
#include "engine.h"
#include "host.h"
#include "mlmc.h"

namespace mlmcgb {

// Sum each task's chunk partials in chunk order; thread 0 also rearms the chunk counter for
// the next round.
__global__ void batch_reduce(const BatchRange *__restrict__ ranges, const BatchHeader *__restrict__ header,
                             const double *__restrict__ chunk_sums, double *task_sums, unsigned *counter)
{
    const unsigned task = blockIdx.x * blockDim.x + threadIdx.x;
    if (task == 0) *counter = 0u;
    if (task >= header->n_tasks) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned c = ranges[task].begin; c < ranges[task].end; ++c) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += chunk_sums[4 * (size_t)c + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) task_sums[4 * (size_t)task + k] = acc[k];
}

const void *batch_reduce_kernel() { return (const void *)batch_reduce; }

namespace {

constexpr int kBatchThreads = 256;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Lanes per path for a deep-level chunk of `spc` samples: enough groups to fill a block,
// chunks of whole Philox blocks and coarse steps.
int batch_lanes(long nf, int M, uint64_t spc)
{
    if (nf < 8) return 1;
    const long unit = std::max(M, 4);
    int P = 1;
    while (P < 32 && spc * (uint64_t)P < (uint64_t)kBatchThreads && nf % (2L * P) == 0 &&
           (nf / (2L * P)) % unit == 0 && nf / (2L * P) >= 32)
        P *= 2;
    return P;
}

struct BatchBuffers {
    size_t cap_tasks = 0, cap_chunks = 0;
    size_t off_ranges = 0, off_tasks = 0, off_chunks = 0, stage_bytes = 0;
    char *h_stage = nullptr, *d_stage = nullptr;
    double *d_chunk_sums = nullptr, *d_task_sums = nullptr, *h_task_sums = nullptr;
    unsigned *d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    void release()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (h_stage) cudaFreeHost(h_stage);
        if (h_task_sums) cudaFreeHost(h_task_sums);
        if (d_stage) cudaFree(d_stage);
        if (d_chunk_sums) cudaFree(d_chunk_sums);
        if (d_task_sums) cudaFree(d_task_sums);
        if (d_counter) cudaFree(d_counter);
        *this = BatchBuffers();
    }

    int reserve(size_t tasks, size_t chunks)
    {
        if (tasks <= cap_tasks && chunks <= cap_chunks) return MLMC_OK;
        release();
        cap_tasks = std::max<size_t>(tasks * 2, 64);
        cap_chunks = std::max<size_t>(chunks * 2, 4096);
        off_ranges = align256(sizeof(BatchHeader));
        off_tasks = off_ranges + align256(cap_tasks * sizeof(BatchRange));
        off_chunks = off_tasks + align256(cap_tasks * sizeof(LevelParams));
        stage_bytes = off_chunks + align256(cap_chunks * sizeof(BatchChunk));
        CUDA_TRY(cudaMallocHost(&h_stage, stage_bytes));
        CUDA_TRY(cudaMallocHost(&h_task_sums, cap_tasks * 4 * sizeof(double)));
        CUDA_TRY(cudaMalloc(&d_stage, stage_bytes));
        CUDA_TRY(cudaMalloc(&d_chunk_sums, cap_chunks * 4 * sizeof(double)));
        CUDA_TRY(cudaMalloc(&d_task_sums, cap_tasks * 4 * sizeof(double)));
        CUDA_TRY(cudaMalloc(&d_counter, sizeof(unsigned)));
        CUDA_TRY(cudaMemset(d_counter, 0, sizeof(unsigned)));
        return MLMC_OK;
    }

    BatchHeader *header() { return (BatchHeader *)h_stage; }
    BatchRange *ranges() { return (BatchRange *)(h_stage + off_ranges); }
    LevelParams *tasks() { return (LevelParams *)(h_stage + off_tasks); }
    BatchChunk *chunks() { return (BatchChunk *)(h_stage + off_chunks); }

    // Upload, persistent kernel, reduction, download: captured once per capacity.
    int capture(cudaStream_t st, const void *kernel, int blocks)
    {
        if (exec) return MLMC_OK;
        const LevelParams *d_tasks = (const LevelParams *)(d_stage + off_tasks);
        const BatchChunk *d_chunks = (const BatchChunk *)(d_stage + off_chunks);
        const BatchRange *d_ranges = (const BatchRange *)(d_stage + off_ranges);
        const BatchHeader *d_header = (const BatchHeader *)d_stage;
        CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemcpyAsync(d_stage, h_stage, stage_bytes, cudaMemcpyHostToDevice, st);
        void *kargs[] = {(void *)&d_tasks, (void *)&d_chunks, (void *)&d_header, (void *)&d_counter,
                         (void *)&d_chunk_sums};
        if (e == cudaSuccess) e = cudaLaunchKernel(kernel, dim3(blocks), dim3(kBatchThreads), kargs, 0, st);
        void *rargs[] = {(void *)&d_ranges, (void *)&d_header, (void *)&d_chunk_sums, (void *)&d_task_sums,
                         (void *)&d_counter};
        const unsigned rblocks = (unsigned)((cap_tasks + 255) / 256);
        if (e == cudaSuccess) e = cudaLaunchKernel(batch_reduce_kernel(), dim3(rblocks), dim3(256), rargs, 0, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_task_sums, d_task_sums, cap_tasks * 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaError_t e2 = cudaStreamEndCapture(st, &graph);
        if (e != cudaSuccess) return fail(MLMC_ECUDA, "capturing the batch round failed: %s", cudaGetErrorString(e));
        if (e2 != cudaSuccess) return fail(MLMC_ECUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(e2));
        CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
        return MLMC_OK;
    }

    // The same round as direct launches (upload, kernel, reduction, download of n_tasks sums).
    int launch_direct(cudaStream_t st, const void *kernel, int blocks, size_t n_tasks)
    {
        const LevelParams *d_tasks = (const LevelParams *)(d_stage + off_tasks);
        const BatchChunk *d_chunks = (const BatchChunk *)(d_stage + off_chunks);
        const BatchRange *d_ranges = (const BatchRange *)(d_stage + off_ranges);
        const BatchHeader *d_header = (const BatchHeader *)d_stage;
        CUDA_TRY(cudaMemcpyAsync(d_stage, h_stage, stage_bytes, cudaMemcpyHostToDevice, st));
        void *kargs[] = {(void *)&d_tasks, (void *)&d_chunks, (void *)&d_header, (void *)&d_counter,
                         (void *)&d_chunk_sums};
        CUDA_TRY(cudaLaunchKernel(kernel, dim3(blocks), dim3(kBatchThreads), kargs, 0, st));
        void *rargs[] = {(void *)&d_ranges, (void *)&d_header, (void *)&d_chunk_sums, (void *)&d_task_sums,
                         (void *)&d_counter};
        CUDA_TRY(cudaLaunchKernel(batch_reduce_kernel(), dim3((unsigned)((n_tasks + 255) / 256)), dim3(256), rargs, 0,
                                  st));
        CUDA_TRY(cudaMemcpyAsync(h_task_sums, d_task_sums, n_tasks * 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        return MLMC_OK;
    }
};

// Fine steps per chunk of a round with `total` fine steps of new work: about four chunks per
// resident block, at least 2^14 and at most 2^22 steps.
double chunk_steps(double total, int blocks)
{
    return std::min(std::max(total / (4.0 * blocks), 16384.0), 4194304.0);
}

// Append one task (samples [first, first + N) of `level` of one problem) and its chunks of about
// W fine steps to a round.  y_out (device or NULL) receives Y of the task's samples in order.
void add_task(std::vector<LevelParams> &tasks, std::vector<BatchChunk> &chunks, std::vector<BatchRange> &ranges,
              const mlmc_problem &pr, int level, int M, uint64_t first, uint64_t N, double W, int precision,
              double *y_out)
{
    const long nf = ipow(M, level);
    const uint64_t spc = (uint64_t)std::max(1.0, std::floor(W / (double)nf));
    LevelParams p;
    fill_params(p, level, M, N, first, &pr.model, &pr.payoff, pr.seed, MLMC_TAG_PATHS, batch_lanes(nf, M, spc),
                precision);
    p.y_out = y_out;
    BatchRange r;
    r.begin = (uint32_t)chunks.size();
    for (uint64_t off = 0; off < N; off += spc) {
        BatchChunk c;
        c.first = first + off;
        c.task = (uint32_t)tasks.size();
        c.count = (uint32_t)std::min<uint64_t>(spc, N - off);
        chunks.push_back(c);
    }
    r.end = (uint32_t)chunks.size();
    ranges.push_back(r);
    tasks.push_back(p);
}

// Checks shared by the batched entry points: GBM, the coupled Euler--Maruyama estimator.
int check_batch_problem(const mlmc_problem &pr, int i)
{
    int rc = check_problem(&pr.model, &pr.payoff);
    if (!rc && pr.model.kind != MLMC_MODEL_GBM) rc = fail(MLMC_ENOTIMPL, "batches run GBM problems");
    if (!rc && (pr.model.scheme != MLMC_EULER_MARUYAMA || pr.payoff.estimator != MLMC_COUPLED))
        rc = fail(MLMC_EINVAL, "batches run the coupled Euler--Maruyama estimator");
    if (rc) {
        std::string msg = mlmc_last_error();
        return fail(rc, "problem %d: %s", i, msg.c_str());
    }
    return MLMC_OK;
}

}  // namespace
}  // namespace mlmcgb

using namespace mlmcgb;

extern "C" int mlmc_estimate_batch(int n, const mlmc_problem *problems, int M, int Lmin, int Lmax, uint64_t N0,
                                   int precision, void *stream, mlmc_result *results)
{
    const auto t_start = std::chrono::steady_clock::now();
    if (n < 1 || !problems || !results) return fail(MLMC_EINVAL, "need n >= 1 and non-NULL problems and results");
    int rc = check_estimate_args(1.0, M, Lmin, Lmax, N0, precision);
    if (rc) return rc;
    if (precision == MLMC_FP64_STREAM32) return fail(MLMC_EINVAL, "batches run MLMC_FP64 or MLMC_FP32_PATH");
    for (int i = 0; i < n; ++i) {
        rc = check_batch_problem(problems[i], i);
        if (!rc && !(problems[i].eps > 0 && std::isfinite(problems[i].eps)))
            rc = fail(MLMC_EINVAL, "problem %d: eps must be positive and finite", i);
        if (rc) return rc;
    }
    const int mt = M == 4 ? 4 : 0;
    const void *kernel = precision == MLMC_FP32_PATH ? batch_kernel_fp32(mt) : batch_kernel_fp64(mt);
    int blocks = 0;
    rc = max_resident_blocks(kernel, kBatchThreads, &blocks);
    if (rc) return rc;

    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    cudaStream_t st = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    BatchBuffers buf;
    auto cleanup = [&]() {
        buf.release();
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (st) cudaStreamDestroy(st);
    };
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        cleanup();
        return fail(MLMC_ECUDA, "%s failed: %s", what, cudaGetErrorString(e));
    };
    cudaError_t e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");

    std::vector<AdaptiveMLMC> drv;
    drv.reserve(n);
    for (int i = 0; i < n; ++i) drv.emplace_back(problems[i].eps, M, Lmin, Lmax, N0);

    struct TaskRef {
        int problem, level;
    };
    std::vector<TaskRef> refs;
    std::vector<LevelParams> tasks;
    std::vector<BatchChunk> chunks;
    std::vector<BatchRange> ranges;
    std::vector<double> sums(MLMC_MAX_LEVELS * 4);
    double kernel_ms = 0.0;
    uint64_t launches = 0, d2h_bytes = 0;
    int rounds = 0;
    for (;;) {
        refs.clear();
        tasks.clear();
        chunks.clear();
        ranges.clear();
        // total new work of the round sets the chunk size: about 4 chunks per resident block
        double total = 0.0;
        for (int i = 0; i < n; ++i) {
            if (!drv[i].active()) continue;
            const std::vector<uint64_t> &dN = drv[i].next_samples();
            for (int l = 0; l <= drv[i].finest_level(); ++l) total += (double)dN[l] * (double)ipow(M, l);
        }
        if (total == 0.0) break;
        const double W = chunk_steps(total, blocks);
        for (int i = 0; i < n; ++i) {
            if (!drv[i].active()) continue;
            const std::vector<uint64_t> &dN = drv[i].next_samples();
            for (int l = 0; l <= drv[i].finest_level(); ++l) {
                if (!dN[l]) continue;
                add_task(tasks, chunks, ranges, problems[i], l, M, drv[i].samples_taken(l), dN[l], W, precision,
                         nullptr);
                refs.push_back({i, l});
            }
        }
        rc = buf.reserve(tasks.size(), chunks.size());
        if (rc) {
            cleanup();
            return rc;
        }
        buf.header()->n_tasks = (uint32_t)tasks.size();
        buf.header()->n_chunks = (uint32_t)chunks.size();
        std::memcpy(buf.ranges(), ranges.data(), ranges.size() * sizeof(BatchRange));
        std::memcpy(buf.tasks(), tasks.data(), tasks.size() * sizeof(LevelParams));
        std::memcpy(buf.chunks(), chunks.data(), chunks.size() * sizeof(BatchChunk));
        rc = buf.capture(st, kernel, blocks);
        if (rc) {
            cleanup();
            return rc;
        }
        if ((e = cudaEventRecord(ev0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaGraphLaunch(buf.exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        if ((e = cudaEventRecord(ev1, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "batch round");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) kernel_ms += ms;
        launches += 2;
        d2h_bytes += buf.cap_tasks * 4 * sizeof(double);
        ++rounds;
        // hand each problem its round sums, level by level
        size_t t = 0;
        while (t < refs.size()) {
            const int i = refs[t].problem;
            std::fill(sums.begin(), sums.end(), 0.0);
            while (t < refs.size() && refs[t].problem == i) {
                for (int k = 0; k < 4; ++k) sums[4 * refs[t].level + k] = buf.h_task_sums[4 * t + k];
                ++t;
            }
            drv[i].absorb(sums.data());
        }
    }
    cleanup();
    const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    bool all = true;
    for (int i = 0; i < n; ++i) {
        std::memset(&results[i], 0, sizeof(mlmc_result));
        drv[i].fill(&results[i]);
        results[i].kernel_ms = kernel_ms;
        results[i].wall_ms = wall;
        results[i].launches = launches;
        results[i].d2h_bytes = d2h_bytes;
        all = all && results[i].converged;
    }
    if (!all) {
        fail(MLMC_ENOTCONV, "some problems reached Lmax = %d before their bias test passed", Lmax);
        return MLMC_ENOTCONV;
    }
    return MLMC_OK;
}

extern "C" int mlmc_level_sums_batch(int n, const mlmc_level_task *tasks, int M, int precision, double *sums,
                                     double *d_y, void *stream)
{
    if (n < 1 || !tasks || !sums) return fail(MLMC_EINVAL, "need n >= 1 and non-NULL tasks and sums");
    if (M != 2 && M != 4 && M != 8) return fail(MLMC_EINVAL, "M must be 2, 4 or 8");
    if (precision != MLMC_FP64 && precision != MLMC_FP32_PATH)
        return fail(MLMC_EINVAL, "batches run MLMC_FP64 or MLMC_FP32_PATH");
    int rc = MLMC_OK;
    double total = 0.0;
    uint64_t n_y = 0;
    for (int i = 0; i < n; ++i) {
        rc = check_batch_problem(tasks[i].problem, i);
        if (!rc) rc = check_level(tasks[i].level, M);
        if (!rc && tasks[i].reserved != 0) rc = fail(MLMC_EINVAL, "task %d: reserved must be 0", i);
        if (!rc && tasks[i].first + tasks[i].N < tasks[i].first) rc = fail(MLMC_EINVAL, "task %d: first + N overflows", i);
        if (!rc && tasks[i].N > 0xFFFFFFFFull) rc = fail(MLMC_EINVAL, "task %d: N above 2^32 - 1", i);
        if (rc) return rc;
        total += (double)tasks[i].N * (double)ipow(M, tasks[i].level);
        n_y += tasks[i].N;
    }
    const int mt = M == 4 ? 4 : 0;
    const void *kernel = precision == MLMC_FP32_PATH ? batch_kernel_fp32(mt) : batch_kernel_fp64(mt);
    int blocks = 0;
    rc = max_resident_blocks(kernel, kBatchThreads, &blocks);
    if (rc) return rc;
    std::vector<LevelParams> lp;
    std::vector<BatchChunk> chunks;
    std::vector<BatchRange> ranges;
    const double W = chunk_steps(total, blocks);
    uint64_t y_off = 0;
    std::vector<int> real;  // tasks with samples, in order
    for (int i = 0; i < n; ++i) {
        if (tasks[i].N == 0) continue;
        add_task(lp, chunks, ranges, tasks[i].problem, tasks[i].level, M, tasks[i].first, tasks[i].N, W, precision,
                 d_y ? d_y + y_off : nullptr);
        y_off += tasks[i].N;
        real.push_back(i);
    }
    std::memset(sums, 0, sizeof(double) * 4 * (size_t)n);
    (void)n_y;
    if (real.empty()) return MLMC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    BatchBuffers buf;
    rc = buf.reserve(lp.size(), chunks.size());
    if (!rc) {
        buf.header()->n_tasks = (uint32_t)lp.size();
        buf.header()->n_chunks = (uint32_t)chunks.size();
        std::memcpy(buf.ranges(), ranges.data(), ranges.size() * sizeof(BatchRange));
        std::memcpy(buf.tasks(), lp.data(), lp.size() * sizeof(LevelParams));
        std::memcpy(buf.chunks(), chunks.data(), chunks.size() * sizeof(BatchChunk));
        rc = buf.launch_direct(st, kernel, blocks, lp.size());
    }
    if (!rc) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(MLMC_ECUDA, "batched level sums failed: %s", cudaGetErrorString(e));
    }
    if (!rc)
        for (size_t t = 0; t < real.size(); ++t)
            for (int k = 0; k < 4; ++k) sums[4 * real[t] + k] = buf.h_task_sums[4 * t + k];
    buf.release();
    return rc;
}
