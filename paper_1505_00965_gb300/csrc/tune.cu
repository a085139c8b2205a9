// tune.cu -- the autotuner: measured choice of the level kernel's launch shape.
//
// For each (precision, payoff, M, level) and size class (N rounded down to a power of two) it
// times candidate shapes -- threads per block, lanes per path (the time-parallel split), samples
// per thread (one, or two in lockstep: the FP32 one-thread-per-sample kernels), and a grid of one
// or two waves of resident blocks -- with CUDA events and keeps the fastest.  The
// planner uses the table whenever the caller leaves the launch shape to the library.  Results
// do not depend on the grid; a different lanes_per_path changes path roundoff only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "engine.h"
#include "host.h"
#include "mlmc.h"

namespace mlmcgb {
namespace {

using Key = std::tuple<int, int, int, int, int>;  // precision, payoff, M, level, log2 N
std::mutex g_tune_mutex;
std::map<Key, TunedShape> g_table;
bool g_env_loaded = false;

int log2_floor(uint64_t n)
{
    int k = 0;
    while (n > 1) {
        n >>= 1;
        ++k;
    }
    return k;
}

int load_file(const char *path, int *entries)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return fail(MLMC_EINVAL, "cannot open %s", path);
    char line[512];
    int n = 0;
    while (std::fgets(line, sizeof(line), f)) {
        int prec, pay, M, level, lg, threads, lanes, oversub, spt = 1;
        double ns;
        // entries written before the samples-per-thread field existed read as one sample per thread
        const int got = std::sscanf(line,
                                    " {\"precision\": %d, \"payoff\": %d, \"M\": %d, \"level\": %d, \"log2N\": %d, "
                                    "\"threads\": %d, \"lanes\": %d, \"oversub\": %d, \"ns_per_sample\": %lf, "
                                    "\"samples_per_thread\": %d}",
                                    &prec, &pay, &M, &level, &lg, &threads, &lanes, &oversub, &ns, &spt);
        if (got >= 9 && spt >= 1 && spt <= 2) {
            g_table[Key(prec, pay, M, level, lg)] = TunedShape{threads, lanes, oversub, ns, spt};
            ++n;
        }
    }
    std::fclose(f);
    if (entries) *entries = n;
    return MLMC_OK;
}

}  // namespace

bool tuned_lookup(int precision, int payoff, int M, int level, uint64_t N, TunedShape *out)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (!g_env_loaded) {
        g_env_loaded = true;
        const char *path = std::getenv("MLMC_AUTOTUNE_CACHE");
        if (path && *path) {
            int n = 0;
            load_file(path, &n);
        }
    }
    if (g_table.empty()) return false;
    // the largest tuned size class at or below N, else the smallest one above it
    const int lg = log2_floor(std::max<uint64_t>(N, 1));
    const TunedShape *below = nullptr, *above = nullptr;
    for (auto it = g_table.lower_bound(Key(precision, payoff, M, level, -1)); it != g_table.end(); ++it) {
        const Key &k = it->first;
        if (std::get<0>(k) != precision || std::get<1>(k) != payoff || std::get<2>(k) != M || std::get<3>(k) != level)
            break;
        if (std::get<4>(k) <= lg) below = &it->second;
        else if (!above) above = &it->second;
    }
    const TunedShape *best = below ? below : above;
    if (!best) return false;
    *out = *best;
    return true;
}

}  // namespace mlmcgb

using namespace mlmcgb;

extern "C" {

int mlmc_autotune(int M, int max_level, int precision, int payoff, void *stream, int *entries)
{
    int rc = check_level(max_level, M);
    if (rc) return rc;
    if (precision != MLMC_FP64 && precision != MLMC_FP32_PATH && precision != MLMC_FP64_STREAM32)
        return fail(MLMC_EINVAL, "precision must be MLMC_FP64, MLMC_FP32_PATH or MLMC_FP64_STREAM32");
    mlmc_model model{MLMC_MODEL_GBM, 0, 100.0, 0.05, 0.2, 1.0};
    mlmc_payoff pay{payoff, 0, 100.0, 1.0};
    rc = check_problem(&model, &pay);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0;
    rc = device_sms(&sms);
    if (rc) return rc;
    const int max_blocks = sms * 32 * 2;
    const size_t ws_bytes = workspace_bytes_for_blocks(max_blocks);
    void *ws = nullptr;
    double *d_sums = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (ws) cudaFree(ws);
        if (d_sums) cudaFree(d_sums);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&ws, ws_bytes);
    if (e == cudaSuccess) e = cudaMemset(ws, 0, ws_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_sums, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return fail(MLMC_ECUDA, "autotuner setup failed: %s", cudaGetErrorString(e));
    }
    int added = 0;
    for (int level = 0; level <= max_level; ++level) {
        const long nf = ipow(M, level);
        const int unit = std::max(M, 4);
        std::vector<int> lanes_set = {1};
        for (int P = 2; P <= 32; P *= 2)
            if (nf >= 8 && nf % P == 0 && (nf / P) % unit == 0) lanes_set.push_back(P);
        for (int lg = 10; lg <= 26; lg += 3) {
            const uint64_t N = 1ull << lg;
            if ((double)N * (double)nf > 2.0e9) break;
            TunedShape best{256, 1, 1, 1e300, 1};
            for (int threads : {128, 256, 512}) {
                for (int lanes : lanes_set) {
                  for (int spt : {1, 2}) {
                    // two samples per thread: FP32 whole paths of levels with M^l >= 4
                    if (spt == 2 && (lanes > 1 || nf < 4 || precision != MLMC_FP32_PATH || threads > kNs2MaxThreads))
                        continue;
                    for (int oversub : {1, 2}) {
                        Plan plan;
                        mlmc_launch probe{threads, lanes, 0, spt};
                        rc = plan_level(level, M, N, precision, payoff, MLMC_EULER_MARUYAMA, &probe, &plan);
                        if (rc) continue;
                        int resident = 0;
                        if (max_resident_blocks(plan.kernel, threads, &resident)) continue;
                        const double items = nf < 4 ? std::ceil((double)N * nf / 4.0) + 1.0
                                                    : std::ceil((double)N * lanes / spt);
                        const int blocks = (int)std::max(1.0, std::min(std::ceil(items / threads),
                                                                       (double)resident * oversub));
                        if (oversub == 2 && blocks <= resident) continue;  // same grid as one wave
                        mlmc_launch shape{threads, lanes, std::min(blocks, max_blocks), spt};
                        float ms = 0.f;
                        for (int rep = 0; rep < 2 && rc == MLMC_OK; ++rep) {
                            e = cudaEventRecord(e0, st);
                            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                                rc = mlmc_level_sums_async(level, M, N, 0, &model, &pay, 1, precision,
                                                           MLMC_TAG_PATHS, &shape, d_sums, ws, ws_bytes, nullptr,
                                                           st);
                                if (rc) break;
                            }
                            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                            if (e != cudaSuccess) {
                                cleanup();
                                return fail(MLMC_ECUDA, "autotuner timing failed: %s", cudaGetErrorString(e));
                            }
                        }
                        if (rc) {
                            cleanup();
                            return rc;
                        }
                        const double ns = 1e6 * ms / 3.0 / (double)N;
                        if (ns < best.ns_per_sample) best = TunedShape{threads, lanes, oversub, ns, spt};
                    }
                  }
                }
            }
            if (best.ns_per_sample < 1e300) {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                g_table[Key(precision, payoff, M, level, lg)] = best;
                ++added;
            }
        }
    }
    cleanup();
    if (entries) *entries = added;
    return MLMC_OK;
}

int mlmc_autotune_save(const char *path)
{
    if (!path) return fail(MLMC_EINVAL, "path must not be NULL");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE *f = std::fopen(path, "w");
    if (!f) return fail(MLMC_EINVAL, "cannot write %s", path);
    std::fprintf(f, "{\"entries\": [\n");
    size_t i = 0;
    for (const auto &kv : g_table) {
        const Key &k = kv.first;
        const TunedShape &s = kv.second;
        std::fprintf(f,
                     " {\"precision\": %d, \"payoff\": %d, \"M\": %d, \"level\": %d, \"log2N\": %d, \"threads\": %d, "
                     "\"lanes\": %d, \"oversub\": %d, \"ns_per_sample\": %.6g, \"samples_per_thread\": %d}%s\n",
                     std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), s.threads,
                     s.lanes, s.oversub, s.ns_per_sample, s.ns > 0 ? s.ns : 1, ++i < g_table.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return MLMC_OK;
}

int mlmc_autotune_load(const char *path, int *entries)
{
    if (!path) return fail(MLMC_EINVAL, "path must not be NULL");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_env_loaded = true;
    return load_file(path, entries);
}

int mlmc_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_table.clear();
    g_env_loaded = true;
    return MLMC_OK;
}

int mlmc_autotune_lookup(int precision, int payoff, int M, int level, uint64_t N, mlmc_launch *out)
{
    if (!out) return fail(MLMC_EINVAL, "out must not be NULL");
    TunedShape s;
    if (!tuned_lookup(precision, payoff, M, level, N, &s)) return fail(MLMC_EINVAL, "no tuned shape");
    out->threads_per_block = s.threads;
    out->lanes_per_path = s.lanes;
    out->blocks = s.oversub;
    out->samples_per_thread = s.ns > 0 ? s.ns : 1;
    return MLMC_OK;
}

int mlmc_autotune_entries(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    return (int)g_table.size();
}

}  // extern "C"
