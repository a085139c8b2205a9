// graph_driver.cu -- the adaptive driver's rounds on the device (Sec. 5, the Theorem's
// algorithm): one CUDA graph per estimate whose WHILE node repeats {driver kernel -> level
// kernels} until the driver ends the loop, so that no round waits for the host.
//
// The driver kernel (one warp) is the device form of AdaptiveMLMC (driver.h), with the same FP64
// formulas in the same order: it adds the last round's level sums, re-estimates means,
// variances and the rates alpha, beta, sets N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k
// sqrt(V_k C_k)), applies the bias test and adds a level.  It then plans each level of the next
// round with the host planner's launch model (lanes per path from the same wave model, the same
// grid) and configures the level kernel nodes through device-side graph updates: the node of
// the chosen kernel variant gets its sample range, lanes and grid, every other node is disabled.
// The level kernels, grids and reduction orders are those of the host-driven rounds, so both
// forms add the same samples in the same order; only CUDA's FP64 log and pow (against the host
// library's) could move a decision at an exact boundary.
//
// Device-side node updates persist across launches of the graph, so each launch gives a node the
// call's parameters (seed, model, payoff) the first time the node runs in that launch, and every
// finished launch leaves all level nodes disabled.  The loop is bounded: a driver that reaches
// kGdMaxIterations stops it with an error status.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "driver.h"
#include "engine.h"
#include "host.h"
#include "mlmc.h"

namespace mlmcgb {

constexpr int kGdVariants = 3;  // per level: one thread per path (or the small / antithetic kernel), split, split long
constexpr int kGdNodes = MLMC_MAX_LEVELS * kGdVariants;
constexpr int kGdThreads = 256;
constexpr int kGdMaxIterations = 4096;  // estimates take tens of rounds
constexpr double kGdLoneWaveCost = 0.25;

enum : int { kGdRunning = 0, kGdDone = 1, kGdNonFinite = 2, kGdDeviceError = 3, kGdTooManyRounds = 4 };
enum : int { kVarWhole = 0, kVarSplit = 1, kVarSplitLong = 2 };

struct GdNode {
    cudaGraphDeviceNode_t dev;  // device handle of the kernel node; NULL where the variant does not exist
    int resident;               // the grid cap of this variant: resident blocks of the kernel the host planner sizes it by
    int pad;
};

// The estimate's configuration (written by the host before every launch) and state, in device
// memory.
struct GdState {
    double eps;
    int M, Lmin, Lmax;
    int small_levels;   // levels l < small_levels have M^l < 4 (4 / M^l samples per Philox block)
    int antithetic;     // one thread per sample, no split
    int ws_blocks;      // grid cap: blocks of a level's workspace slot
    uint64_t N0;
    int res1[MLMC_MAX_LEVELS], resp[MLMC_MAX_LEVELS];  // residencies the lanes model compares
    double C[MLMC_MAX_LEVELS];                         // C_l, cost of one sample
    GdNode node[kGdNodes];                             // node l * kGdVariants + variant
    LevelParams tmpl[MLMC_MAX_LEVELS];                 // the call's parameters of each level
    // state
    int L, rounds, status, iter, converged, pad;
    double alpha, beta;
    uint64_t N[MLMC_MAX_LEVELS], dN[MLMC_MAX_LEVELS];
    double S[MLMC_MAX_LEVELS][4];
    double mean[MLMC_MAX_LEVELS], var[MLMC_MAX_LEVELS];
    double sums[MLMC_MAX_LEVELS][4];  // this round's level sums, written by the level kernels
    uint64_t launches;
    // per node: whether it is enabled (device-side updates persist across launches: nodes start
    // enabled after instantiation and every finished launch leaves them disabled; the host
    // passes the state in), and whether this launch has set its full parameters (a node gets
    // them the first time it runs in a launch)
    int enabled[kGdNodes], full_set[kGdNodes];
};

// std::max of the host driver, NaN handling included: (a < b) ? b : a.
__device__ __forceinline__ double hmax(double a, double b) { return (a < b) ? b : a; }

__device__ double gd_lsq_slope(int n, const double *y)  // x = 1..n
{
    double mx = 0, my = 0;
    for (int i = 0; i < n; ++i) {
        mx += (double)(i + 1);
        my += y[i];
    }
    mx /= n;
    my /= n;
    double sxy = 0, sxx = 0;
    for (int i = 0; i < n; ++i) {
        sxy += ((double)(i + 1) - mx) * (y[i] - my);
        sxx += ((double)(i + 1) - mx) * ((double)(i + 1) - mx);
    }
    return sxy / sxx;
}

// vf = floored variances of levels 0..L and mf = floored means (as AdaptiveMLMC::floored), with
// Ma = M^alpha and Mb = M^beta.  One lane (a chain over the levels).
__device__ void gd_floored(const GdState &s, double Ma, double Mb, double *mf, double *vf)
{
    for (int l = 0; l <= s.L; ++l) {
        mf[l] = s.mean[l];
        vf[l] = s.var[l];
    }
    for (int l = 2; l <= s.L; ++l) {
        mf[l] = hmax(fabs(mf[l]), 0.5 * fabs(mf[l - 1]) / Ma);
        vf[l] = hmax(vf[l], 0.5 * vf[l - 1] / Mb);
    }
}

__device__ double gd_bias(const GdState &s, double Ma, const double *mf)
{
    return hmax(fabs(mf[s.L]), fabs(mf[s.L - 1]) / Ma) / (Ma - 1.0);
}

// dN_l for levels 0..nl-1 from variances V (as AdaptiveMLMC::extra_samples), the whole warp:
// lane l forms level l's square roots and its count, lane 0 adds the square roots in level order.
__device__ void gd_extra_samples(GdState &s, const double *V, int nl, double *root)
{
    const int lane = threadIdx.x;
    double q = 0.0;
    if (lane < nl) {
        root[lane] = sqrt(V[lane] * s.C[lane]);
        q = sqrt(V[lane] / s.C[lane]);
    }
    __syncwarp();
    double tot = 0;
    for (int l = 0; l < nl; ++l) tot += root[l];
    if (lane < MLMC_MAX_LEVELS) {
        if (lane < nl) {
            const double n = ceil(2.0 / (s.eps * s.eps) * q * tot);
            const uint64_t want = n > 9.0e18 ? (uint64_t)9.0e18 : (uint64_t)n;
            const uint64_t done = s.N[lane];
            s.dN[lane] = want > done ? want - done : 0;
        } else {
            s.dN[lane] = 0;
        }
    }
    __syncwarp();
}

// Launch plan of `dN` samples of level l (the host planner's automatic shape: 256 threads, the
// lanes wave model, grid capped by the kernel's residency and the workspace).
__device__ void gd_plan(const GdState &s, int l, uint64_t dN, int &variant, int &lanes, int &blocks)
{
    long nf = 1;
    for (int i = 0; i < l; ++i) nf *= s.M;
    const int unit = s.M > 4 ? s.M : 4;
    const double threads = (double)kGdThreads;
    const double Nd = (double)(dN > 0 ? dN : 1);
    lanes = 1;
    variant = kVarWhole;
    double need;
    if (l < s.small_levels) {
        need = ceil((ceil(Nd * (double)nf / 4.0) + 1.0) / threads);
    } else {
        if (nf >= 8 && !s.antithetic) {
            double best = 0.0;
            for (int P = 1; P <= 32; P *= 2) {
                if (P > 1 && (nf % P != 0 || (nf / P) % unit != 0 || nf / P < 256)) break;
                const double T = (double)(P == 1 ? s.res1[l] : s.resp[l]) * threads;
                const double w = Nd * P / T;
                const double full = floor(w);
                const double waves = w < 1.0 ? fmax(fmin(1.0, 3.0 * w), kGdLoneWaveCost)
                                             : full + fmin(1.0, kLanesTailSlope * (w - full) + kLanesTailBase);
                const double per_step = P > 1 ? kLanesSplitStep : 1.0;
                const double cost = waves * ((double)nf / P + 12.0) * per_step;
                if (P == 1 || cost < 0.99 * best) {
                    best = cost;
                    lanes = P;
                }
            }
        }
        if (lanes > 1) variant = nf / lanes > kLongLaneSteps ? kVarSplitLong : kVarSplit;
        need = ceil(ceil(Nd * (double)lanes) / threads);
    }
    const int cap = s.node[l * kGdVariants + variant].resident;
    double b = fmin(need, (double)cap);
    if (b < 1.0) b = 1.0;
    blocks = (int)b;
    if (blocks > s.ws_blocks) blocks = s.ws_blocks;
}

// One iteration of the graph's loop: absorb the last round (after the first iteration), plan the
// next one, configure the level nodes, and set the loop's condition.  One warp.
__global__ void __launch_bounds__(32) gd_driver_kernel(GdState *sp, cudaGraphConditionalHandle cond)
{
    __shared__ double lm[MLMC_MAX_LEVELS], lv[MLMC_MAX_LEVELS];
    __shared__ double mf[MLMC_MAX_LEVELS + 1], vf[MLMC_MAX_LEVELS + 1], root[MLMC_MAX_LEVELS], powM[2];
    __shared__ int phase_ok, grow;
    // the update list (raw storage: the struct's union holds a dim3 and has no default constructor)
    __shared__ __align__(16) unsigned char upd_raw[kGdNodes * 5 * sizeof(cudaGraphKernelNodeUpdate)];
    cudaGraphKernelNodeUpdate *upd = reinterpret_cast<cudaGraphKernelNodeUpdate *>(upd_raw);
    __shared__ uint64_t range[MLMC_MAX_LEVELS][2];
    __shared__ int lanes_of[MLMC_MAX_LEVELS], variant_of[MLMC_MAX_LEVELS], blocks_of[MLMC_MAX_LEVELS];
    __shared__ int active_sh;
    // the state in shared memory for the iteration (each scalar step of the driver would otherwise
    // wait on a global load): copied in by the warp, worked on, copied back at the end
    __shared__ __align__(16) GdState s;
    static_assert(sizeof(GdState) % sizeof(uint64_t) == 0, "the state copies in 8-byte words");
    const int lane = threadIdx.x;
    for (size_t i = lane; i < sizeof(GdState) / sizeof(uint64_t); i += 32)
        reinterpret_cast<uint64_t *>(&s)[i] = reinterpret_cast<const uint64_t *>(sp)[i];
    __syncwarp();
    const int iter = s.iter;
    if (iter == 0) {
        if (lane == 0) phase_ok = 1;
        __syncwarp();
    } else {
        // absorb the round (AdaptiveMLMC::absorb); per-level arithmetic one level per lane
        if (lane == 0) {
            phase_ok = 1;
            for (int l = 0; l <= s.L; ++l) {
                if (!s.dN[l]) continue;
                for (int k = 0; k < 4; ++k)
                    if (!isfinite(s.sums[l][k])) phase_ok = 0;
            }
            if (phase_ok) ++s.rounds;
            else s.status = kGdNonFinite;
        }
        __syncwarp();
        if (phase_ok) {
            const int l = lane;
            if (l <= s.L) {
                if (s.dN[l]) {
                    for (int k = 0; k < 4; ++k) s.S[l][k] += s.sums[l][k];
                    s.N[l] += s.dN[l];
                }
                s.mean[l] = s.S[l][0] / (double)s.N[l];
                s.var[l] = hmax(s.S[l][1] / (double)s.N[l] - s.mean[l] * s.mean[l], 0.0);
                // the rates' least-squares inputs
                if (l >= 1) {
                    const double tiny = 1e-300, lnM = log((double)s.M);
                    lm[l - 1] = log(hmax(fabs(s.mean[l]), tiny)) / lnM;
                    lv[l - 1] = log(hmax(s.var[l], tiny)) / lnM;
                }
            }
            __syncwarp();
            if (lane == 0) s.alpha = hmax(0.5, -gd_lsq_slope(s.L, lm));
            if (lane == 1) s.beta = hmax(0.5, -gd_lsq_slope(s.L, lv));
            __syncwarp();
            if (lane == 0) powM[0] = pow((double)s.M, s.alpha);
            if (lane == 1) powM[1] = pow((double)s.M, s.beta);
            __syncwarp();
            if (lane == 0) gd_floored(s, powM[0], powM[1], mf, vf);
            __syncwarp();
            gd_extra_samples(s, vf, s.L + 1, root);
            if (lane == 0) {
                bool settled = true;
                for (int q = 0; q <= s.L; ++q)
                    if ((double)s.dN[q] > 0.01 * (double)s.N[q]) settled = false;
                grow = settled && gd_bias(s, powM[0], mf) > s.eps / sqrt(2.0) && s.L < s.Lmax;
                if (grow) {
                    s.L += 1;
                    vf[s.L] = vf[s.L - 1] / powM[1];
                    s.N[s.L] = 0;
                    for (int k = 0; k < 4; ++k) s.S[s.L][k] = 0.0;
                }
            }
            __syncwarp();
            if (grow) gd_extra_samples(s, vf, s.L + 1, root);
        }
    }
    // the next round: the node of each level's kernel variant, every other node disabled
    int n_upd = 0;
    if (lane == 0) {
        bool active = false;
        if (s.status == kGdRunning) {
            for (int l = 0; l <= s.L; ++l) active = active || s.dN[l] > 0;
            if (iter + 1 >= kGdMaxIterations) {
                s.status = kGdTooManyRounds;
                active = false;
            }
        }
        if (!active && s.status == kGdRunning) {
            s.status = kGdDone;
            const double Ma = pow((double)s.M, s.alpha), Mb = pow((double)s.M, s.beta);
            gd_floored(s, Ma, Mb, mf, vf);
            s.converged = gd_bias(s, Ma, mf) <= s.eps / sqrt(2.0) ? 1 : 0;
        }
        active_sh = active ? 1 : 0;
    }
    __syncwarp();
    const bool active = active_sh != 0;
    if (lane < MLMC_MAX_LEVELS) {  // each level's launch plan on its own lane
        const int l = lane;
        int variant = -1, lanes = 1, blocks = 1;
        if (active && l <= s.L && s.dN[l] > 0) gd_plan(s, l, s.dN[l], variant, lanes, blocks);
        variant_of[l] = variant;
        lanes_of[l] = lanes;
        blocks_of[l] = blocks;
        range[l][0] = s.N[l];
        range[l][1] = s.dN[l];
    }
    __syncwarp();
    if (lane == 0) {
        for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
            const int variant = variant_of[l], blocks = blocks_of[l];
            for (int v = 0; v < kGdVariants; ++v) {
                const int id = l * kGdVariants + v;
                const GdNode &nd = s.node[id];
                if (!nd.dev) continue;
                const bool on = v == variant;
                if (on != (s.enabled[id] != 0)) {
                    cudaGraphKernelNodeUpdate &e = upd[n_upd++];
                    e.node = nd.dev;
                    e.field = cudaGraphKernelNodeFieldEnabled;
                    e.updateData.isEnabled = on ? 1u : 0u;
                    s.enabled[id] = on ? 1 : 0;
                }
                if (!on) continue;
                if (!s.full_set[id]) {
                    cudaGraphKernelNodeUpdate &f = upd[n_upd++];
                    f.node = nd.dev;
                    f.field = cudaGraphKernelNodeFieldParam;
                    f.updateData.param.pValue = &s.tmpl[l];
                    f.updateData.param.offset = 0;
                    f.updateData.param.size = sizeof(LevelParams);
                    s.full_set[id] = 1;
                }
                cudaGraphKernelNodeUpdate &gdim = upd[n_upd++];
                gdim.node = nd.dev;
                gdim.field = cudaGraphKernelNodeFieldGridDim;
                gdim.updateData.gridDim = dim3((unsigned)blocks, 1, 1);
                cudaGraphKernelNodeUpdate &pr = upd[n_upd++];
                pr.node = nd.dev;
                pr.field = cudaGraphKernelNodeFieldParam;
                pr.updateData.param.pValue = &range[l][0];
                pr.updateData.param.offset = offsetof(LevelParams, first);
                pr.updateData.param.size = 2 * sizeof(uint64_t);
                cudaGraphKernelNodeUpdate &pl = upd[n_upd++];
                pl.node = nd.dev;
                pl.field = cudaGraphKernelNodeFieldParam;
                pl.updateData.param.pValue = &lanes_of[l];
                pl.updateData.param.offset = offsetof(LevelParams, lanes);
                pl.updateData.param.size = sizeof(int);
                ++s.launches;
            }
        }
        bool go = active;
        if (cudaGraphKernelNodeUpdatesApply(upd, (size_t)n_upd) != cudaSuccess) {
            s.status = kGdDeviceError;
            go = false;
            // a failed update may have left nodes enabled: disable every node one by one
            for (int v = 0; v < kGdNodes; ++v)
                if (s.node[v].dev) cudaGraphKernelNodeSetEnabled(s.node[v].dev, false);
        }
        s.iter = iter + 1;
        cudaGraphSetConditional(cond, go ? 1u : 0u);
    }
    __syncwarp();
    for (size_t i = lane; i < sizeof(GdState) / sizeof(uint64_t); i += 32)
        reinterpret_cast<uint64_t *>(sp)[i] = reinterpret_cast<const uint64_t *>(&s)[i];
}

namespace {

// One instantiated graph with its device state and workspace slots, for one problem shape.
struct GdCache {
    int device = -1;
    int key[10] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GdState *d_state = nullptr, *h_state = nullptr;
    void *slots = nullptr;
    size_t slot_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    GdNode nodes[kGdNodes] = {};
    int res1[MLMC_MAX_LEVELS] = {}, resp[MLMC_MAX_LEVELS] = {};
    int ws_blocks = 0;
    bool launched = false;  // a finished launch left every node disabled

    void release()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (d_state) cudaFree(d_state);
        if (h_state) cudaFreeHost(h_state);
        if (slots) cudaFree(slots);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        *this = GdCache();
    }
};

std::mutex g_gd_mutex;
std::vector<GdCache *> g_gd_pool;
// The host rounds are the default: on GB300 a host round trip (copy, synchronisation, the
// host's FP64 update, launches) takes about 16 us, while the driver kernel's FP64 update alone
// takes about 23 us (a chain of dependent FP64 divisions, logarithms and powers on a pipe of 2
// operations per SM per clock), plus 6 us of planning and 2-9 us of graph updates per round.
int g_driver_mode = MLMC_DRIVER_HOST;

// Kernel of `variant` on level l for the problem (nullptr where the variant does not exist), the
// residency its grid is capped by, and the lanes model's inputs (as plan_level and plan_problem).
struct LevelKernels {
    const void *k[kGdVariants];
    int resident[kGdVariants];
    int res1, resp;
};

int level_kernels(int l, int M, int precision, const mlmc_model *model, const mlmc_payoff *payoff, LevelKernels *out)
{
    *out = LevelKernels{};
    const long nf = ipow(M, l);
    const int pay = payoff->kind, scheme = model->scheme;
    const bool anti = payoff->estimator == MLMC_ANTITHETIC;
    auto pick = [&](int mt, bool split, bool long_lanes, bool positive) {
        return precision == MLMC_FP32_PATH ? level_kernel_fp32(pay, mt, split, scheme, long_lanes, positive)
                                           : level_kernel_fp64(pay, mt, split, scheme, long_lanes, positive);
    };
    int rc;
    if (nf < 4) {
        out->k[kVarWhole] = pick(-1, false, false, false);
        if (!out->k[kVarWhole]) return fail(MLMC_EINVAL, "no kernel for payoff %d", pay);
        return max_resident_blocks(out->k[kVarWhole], kGdThreads, &out->resident[kVarWhole]);
    }
    const int mt = M == 4 ? 4 : 0;
    // whole paths: the two-sample kernel where plan_level takes it by default (same grid rule)
    const bool ns2 = !anti && precision == MLMC_FP32_PATH && scheme == MLMC_EULER_MARUYAMA && M == 4 &&
                     nf >= kNs2MinSteps && kGdThreads <= kNs2MaxThreads;
    const void *whole = ns2 ? level_ns2_kernel_fp32(pay, mt, nf > kLongLaneSteps)
                            : pick(mt, false, nf > kLongLaneSteps, false);
    if (!whole) return fail(MLMC_EINVAL, "no kernel for payoff %d", pay);
    rc = max_resident_blocks(whole, kGdThreads, &out->resident[kVarWhole]);
    if (rc) return rc;
    out->k[kVarWhole] = whole;
    if (anti) {
        const void *ak = precision == MLMC_FP32_PATH ? level_anti_kernel_fp32(pay, mt, scheme, nf > kLongLaneSteps)
                                                     : level_anti_kernel_fp64(pay, mt, scheme, nf > kLongLaneSteps);
        if (!ak) return fail(MLMC_EINVAL, "no antithetic kernel for payoff %d", pay);
        int ra = 0;
        rc = max_resident_blocks(ak, kGdThreads, &ra);
        if (rc) return rc;
        out->k[kVarWhole] = ak;
        out->resident[kVarWhole] = std::min(out->resident[kVarWhole], ra);
        return MLMC_OK;
    }
    if (nf < 8) return MLMC_OK;
    // the lanes model's residencies: one-thread-per-path and split kernels without long lanes
    const void *k1 = pick(mt, false, false, false), *kp = pick(mt, true, false, false);
    rc = max_resident_blocks(k1, kGdThreads, &out->res1);
    if (!rc) rc = max_resident_blocks(kp, kGdThreads, &out->resp);
    if (rc) return rc;
    const bool pos = pay == kLookback && positive_step_factors(model, l, M);
    out->k[kVarSplit] = pick(mt, true, false, pos);
    out->resident[kVarSplit] = out->resp;
    if (nf / 2 > kLongLaneSteps) {
        const void *kl = pick(mt, true, true, false);
        int rl = 0;
        rc = max_resident_blocks(kl, kGdThreads, &rl);
        if (rc) return rc;
        out->k[kVarSplitLong] = pos ? pick(mt, true, false, true) : kl;
        out->resident[kVarSplitLong] = rl;
    }
    return MLMC_OK;
}

#define GD_TRY(expr)                                                                                        \
    do {                                                                                                    \
        cudaError_t e_ = (expr);                                                                            \
        if (e_ != cudaSuccess) {                                                                            \
            cudaGetLastError();                                                                             \
            return fail(MLMC_ENOTIMPL, "device-side rounds unavailable: %s: %s", #expr, cudaGetErrorString(e_)); \
        }                                                                                                   \
    } while (0)

// Build the graph of one problem shape into `c` (kernels, residencies, nodes, slots, state).
int gd_build(GdCache &c, int dev, const int key[10], int M, int Lmax, int precision, const mlmc_model *model,
             const mlmc_payoff *payoff)
{
    c.device = dev;
    std::memcpy(c.key, key, sizeof(c.key));
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    c.ws_blocks = sms * 32;
    c.slot_bytes = (workspace_bytes_for_blocks(c.ws_blocks) + 255) / 256 * 256;
    GD_TRY(cudaMalloc(&c.d_state, sizeof(GdState)));
    GD_TRY(cudaMallocHost(&c.h_state, sizeof(GdState)));
    GD_TRY(cudaMalloc(&c.slots, c.slot_bytes * (size_t)(Lmax + 1)));
    GD_TRY(cudaMemset(c.slots, 0, c.slot_bytes * (size_t)(Lmax + 1)));
    GD_TRY(cudaEventCreate(&c.ev0));
    GD_TRY(cudaEventCreate(&c.ev1));
    GD_TRY(cudaGraphCreate(&c.graph, 0));
    cudaGraphConditionalHandle cond;
    GD_TRY(cudaGraphConditionalHandleCreate(&cond, c.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    GD_TRY(cudaGraphAddNode(&wnode, c.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    GdState *dst = c.d_state;
    void *dargs[] = {(void *)&dst, (void *)&cond};
    cudaKernelNodeParams dk = {};
    dk.func = (void *)gd_driver_kernel;
    dk.gridDim = dim3(1);
    dk.blockDim = dim3(32);
    dk.kernelParams = dargs;
    cudaGraphNode_t dnode;
    GD_TRY(cudaGraphAddKernelNode(&dnode, body, nullptr, 0, &dk));
    for (int l = 0; l <= Lmax; ++l) {
        LevelKernels lk;
        rc = level_kernels(l, M, precision, model, payoff, &lk);
        if (rc) return rc;
        c.res1[l] = lk.res1;
        c.resp[l] = lk.resp;
        for (int v = 0; v < kGdVariants; ++v) {
            if (!lk.k[v]) continue;
            size_t off = 1, size = 0;
            GD_TRY(cudaFuncGetParamInfo(lk.k[v], 0, &off, &size));
            if (off != 0 || size != sizeof(LevelParams))
                return fail(MLMC_ENOTIMPL, "device-side rounds unavailable: unexpected kernel parameter layout");
            // instantiation parameters: a valid one-sample launch into this level's own slot and
            // sums (the driver kernel gives every node the call's parameters before it first runs
            // and disables the others; a node that ran on these would still stay in bounds)
            LevelParams p;
            fill_params(p, l, M, 1, 0, model, payoff, 1, MLMC_TAG_PATHS, 1, precision);
            p.out = &c.d_state->sums[l][0];
            p.ticket = (unsigned *)((char *)c.slots + c.slot_bytes * (size_t)l);
            p.partials = (double *)((char *)c.slots + c.slot_bytes * (size_t)l + kTicketBytes);
            void *kargs[] = {&p};
            cudaKernelNodeParams kp = {};
            kp.func = const_cast<void *>(lk.k[v]);
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(kGdThreads);
            kp.kernelParams = kargs;
            cudaGraphNode_t kn;
            GD_TRY(cudaGraphAddKernelNode(&kn, body, &dnode, 1, &kp));
            cudaKernelNodeAttrValue av = {};
            av.deviceUpdatableKernelNode.deviceUpdatable = 1;
            GD_TRY(cudaGraphKernelNodeSetAttribute(kn, cudaLaunchAttributeDeviceUpdatableKernelNode, &av));
            cudaKernelNodeAttrValue got = {};
            GD_TRY(cudaGraphKernelNodeGetAttribute(kn, cudaLaunchAttributeDeviceUpdatableKernelNode, &got));
            if (!got.deviceUpdatableKernelNode.devNode)
                return fail(MLMC_ENOTIMPL, "device-side rounds unavailable: no device handle for a kernel node");
            c.nodes[l * kGdVariants + v].dev = got.deviceUpdatableKernelNode.devNode;
            c.nodes[l * kGdVariants + v].resident = lk.resident[v];
        }
    }
    GD_TRY(cudaGraphInstantiate(&c.exec, c.graph, 0));
    return MLMC_OK;
}

void shape_key(int out[10], int M, int Lmin, int Lmax, int precision, const mlmc_model *model, const mlmc_payoff *payoff)
{
    // the graph depends on the kernels of every level: M, Lmax, precision, payoff, scheme,
    // estimator and (through the lookback's positive-factor kernels) sigma, r and T
    int pos = 0;
    for (int l = 0; l <= Lmax && l < 31; ++l)
        if (payoff->kind == kLookback && positive_step_factors(model, l, M)) pos |= 1 << l;
    const int k[10] = {M, Lmin, Lmax, precision, payoff->kind, model->scheme, payoff->estimator, pos, model->kind, 0};
    std::memcpy(out, k, sizeof(k));
}

}  // namespace

// Free every cached graph of the current device (mlmc_shutdown).
void graph_driver_release(int dev)
{
    std::lock_guard<std::mutex> lock(g_gd_mutex);
    for (size_t i = 0; i < g_gd_pool.size();) {
        if (g_gd_pool[i]->device == dev) {
            g_gd_pool[i]->release();
            delete g_gd_pool[i];
            g_gd_pool.erase(g_gd_pool.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

int graph_driver_mode()
{
    std::lock_guard<std::mutex> lock(g_gd_mutex);
    return g_driver_mode;
}

// Whether the device form covers this problem (GBM; coupled or antithetic; any precision).
bool graph_driver_covers(const mlmc_model *model, const mlmc_payoff *payoff)
{
    return model->kind == MLMC_MODEL_GBM &&
           (payoff->estimator == MLMC_COUPLED || payoff->estimator == MLMC_ANTITHETIC);
}

// mlmc_estimate with the rounds on the device.  MLMC_ENOTIMPL (nothing launched) where the
// graph cannot be built on this device; the caller then runs the host rounds.
int estimate_on_device(double eps, int M, int Lmin, int Lmax, uint64_t N0, const mlmc_model *model,
                       const mlmc_payoff *payoff, uint64_t seed, int precision, cudaStream_t st, mlmc_result *out,
                       std::chrono::steady_clock::time_point t_start)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    int key[10];
    shape_key(key, M, Lmin, Lmax, precision, model, payoff);
    GdCache *c = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_gd_mutex);
        for (size_t i = 0; i < g_gd_pool.size(); ++i) {
            if (g_gd_pool[i]->device == dev && std::memcmp(g_gd_pool[i]->key, key, sizeof(key)) == 0) {
                c = g_gd_pool[i];
                g_gd_pool.erase(g_gd_pool.begin() + (long)i);
                break;
            }
        }
    }
    if (!c) {
        c = new GdCache();
        const int rc = gd_build(*c, dev, key, M, Lmax, precision, model, payoff);
        if (rc) {
            c->release();
            delete c;
            return rc;
        }
    }
    auto give_back = [&](bool keep) {
        if (!keep) {
            c->release();
            delete c;
            return;
        }
        std::lock_guard<std::mutex> lock(g_gd_mutex);
        g_gd_pool.push_back(c);
    };
    // configuration and initial state (AdaptiveMLMC's constructor: warm-up N0 on levels 0..Lmin)
    GdState &h = *c->h_state;
    std::memset(&h, 0, sizeof(h));
    h.eps = eps;
    h.M = M;
    h.Lmin = Lmin;
    h.Lmax = Lmax;
    h.N0 = N0;
    int small = 0;
    while (small <= Lmax && ipow(M, small) < 4) ++small;
    h.small_levels = small;
    h.antithetic = payoff->estimator == MLMC_ANTITHETIC ? 1 : 0;
    h.ws_blocks = c->ws_blocks;
    AdaptiveMLMC costs(eps, M, Lmin, Lmax, N0);  // C_l with the estimator's cost scale
    if (h.antithetic)
        for (int l = 1; l < MLMC_MAX_LEVELS; ++l) costs.set_cost_scale(l, (2.0 * M + 1.0) / (M + 1.0));
    for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
        h.res1[l] = c->res1[l];
        h.resp[l] = c->resp[l];
        h.C[l] = costs.cost_of(l);
    }
    std::memcpy(h.node, c->nodes, sizeof(h.node));
    for (int v = 0; v < kGdNodes; ++v) h.enabled[v] = (c->nodes[v].dev && !c->launched) ? 1 : 0;
    for (int l = 0; l <= Lmax; ++l) {
        LevelParams &p = h.tmpl[l];
        fill_params(p, l, M, 0, 0, model, payoff, seed, MLMC_TAG_PATHS, 1, precision);
        p.out = &c->d_state->sums[l][0];
        p.ticket = (unsigned *)((char *)c->slots + c->slot_bytes * (size_t)l);
        p.partials = (double *)((char *)c->slots + c->slot_bytes * (size_t)l + kTicketBytes);
    }
    h.L = Lmin;
    h.alpha = h.beta = 0.5;
    for (int l = 0; l <= Lmin; ++l) h.dN[l] = N0;
    cudaError_t e = cudaMemcpyAsync(c->d_state, c->h_state, sizeof(GdState), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(c->exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_state, c->d_state, sizeof(GdState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        give_back(false);
        return fail(MLMC_ECUDA, "device-side rounds failed: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    const GdState r = h;  // copy before the cache goes back to the pool
    // a launch that did not finish may have left nodes enabled: such a cache is not reused
    c->launched = true;
    give_back(r.status == kGdDone);
    if (r.status == kGdNonFinite)
        return fail(MLMC_ENONFINITE, "level sums of round %d are not finite (the scheme diverged)", r.rounds + 1);
    if (r.status == kGdDeviceError) return fail(MLMC_ECUDA, "a device-side graph update failed");
    if (r.status == kGdTooManyRounds) return fail(MLMC_ECUDA, "the device-side driver stopped after %d rounds", r.rounds);
    if (r.status != kGdDone) return fail(MLMC_ECUDA, "the device-side driver ended in state %d", r.status);
    // the result, as AdaptiveMLMC::fill
    std::memset(out, 0, sizeof(*out));
    out->eps = eps;
    out->L = r.L;
    out->converged = r.converged;
    out->rounds = r.rounds;
    out->device_rounds = 1;
    double P = 0.0, total = 0.0, steps = 0.0;
    for (int l = 0; l <= r.L; ++l) {
        out->N[l] = r.N[l];
        for (int k = 0; k < 4; ++k) out->sums[l][k] = r.S[l][k];
        out->mean[l] = r.mean[l];
        out->var[l] = r.var[l];
        out->cost[l] = (double)r.N[l] * r.C[l];
        P += r.mean[l];
        total += out->cost[l];
        steps += (double)r.N[l] * (double)ipow(M, l);
    }
    out->P = P;
    out->alpha = r.alpha;
    out->beta = r.beta;
    out->total_cost = total;
    out->path_steps = steps;
    out->kernel_ms = ms;
    out->launches = r.launches + (uint64_t)r.iter;  // level kernels and driver iterations
    out->d2h_bytes = sizeof(GdState);
    out->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (!out->converged) {
        fail(MLMC_ENOTCONV, "bias test still failing at Lmax = %d", Lmax);
        return MLMC_ENOTCONV;
    }
    return MLMC_OK;
}

}  // namespace mlmcgb

extern "C" int mlmc_set_driver_mode(int mode, int *previous)
{
    if (mode != MLMC_DRIVER_AUTO && mode != MLMC_DRIVER_HOST && mode != MLMC_DRIVER_DEVICE)
        return mlmcgb::fail(MLMC_EINVAL, "mode must be MLMC_DRIVER_AUTO, MLMC_DRIVER_HOST or MLMC_DRIVER_DEVICE");
    std::lock_guard<std::mutex> lock(mlmcgb::g_gd_mutex);
    if (previous) *previous = mlmcgb::g_driver_mode;
    mlmcgb::g_driver_mode = mode;
    return MLMC_OK;
}
