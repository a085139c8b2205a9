/*
 * mlmc.h -- C ABI of the GB300 multilevel Monte Carlo level engine.
 *
 * The engine computes, on one GPU, the level estimators of multilevel Monte Carlo for option
 * valuation (D. J. Higham, "An Introduction to Multilevel Monte Carlo for Option Valuation",
 * Sec. 5): for level l it simulates N coupled pairs of Euler--Maruyama paths (Sec. 2, Eq. em)
 * of geometric Brownian motion, the fine path with step T / M^l and the coarse path with
 * step T / M^(l-1) driven by sums of M consecutive fine increments (Sec. 5, Fig. 2), and
 * returns sum Y, sum Y^2, sum Y^3, sum Y^4 of Y = P_l - P_{l-1} (Eq. Yldef; Y = P_0 on
 * level 0, Eq. mlmc:Yzero).  The adaptive driver combines the levels by the telescoping sum
 * of Eq. (mlmc:ident).
 *
 * Conventions for every function below:
 *   - Return value: an mlmc_status; 0 (MLMC_OK) on success.  On failure the outputs are left
 *     untouched and mlmc_last_error() returns a message for the calling host thread.
 *   - Pointers documented as "host" are caller-owned host memory, read or written only during
 *     the call.  Pointers documented as "device" are caller-owned device memory on the current
 *     CUDA device; the engine only reads or writes them in work queued on the given stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Functions with host outputs synchronise `stream` before returning.  Functions with the
 *     _async suffix only queue work on `stream` and never synchronise.
 *   - All floating-point arguments are FP64; the path arithmetic precision is chosen by an
 *     mlmc_precision argument.
 *   - Random numbers: sample s of level l draws Philox4x32-10 blocks with key = (seed low,
 *     seed high) and counter = ((tag << 16) | l, j, s high, s low), j = 0, 1, ...  Block j
 *     gives normals 4j..4j+3 by two Box--Muller pairs; fine step k takes normal k,
 *     dW_k = sqrt(T / M^l) z_k.  Every level and every sample index therefore has its own,
 *     independent numbers (Sec. 5: fresh random numbers on every level), and a sample range
 *     [first, first + N) can be computed in any order, on any device, with identical results.
 */
#ifndef MLMC_GB300_H
#define MLMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mlmc_status {
    MLMC_OK = 0,
    MLMC_EINVAL = 1,      /* an argument is out of range or a required pointer is NULL */
    MLMC_ECUDA = 2,       /* a CUDA call failed; the message carries the CUDA error string */
    MLMC_ENOMEM = 3,      /* a device or host allocation failed */
    MLMC_ENOTCONV = 4,    /* the driver reached Lmax before the bias test passed */
    MLMC_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
    MLMC_ENOTIMPL = 6,    /* the combination of options is not implemented */
    MLMC_ENONFINITE = 7   /* a level's sums are not finite: the scheme diverged (the driver stops) */
} mlmc_status;

/* Models:
 *   GBM          geometric Brownian motion dS = r S dt + sigma S dW, S(0) = S0, on [0, T]
 *                (the SDE of Sec. 2, Eq. sde, with f(x) = r x and g(x) = sigma x as in Sec. 6).
 *   QUINTIC_ODE  the counterexample cited in Sec. 5 (Eq. count): dX = -X^5 dt with a standard
 *                normal X(0), on [0, T].  Only T is read (S0, r, sigma must be finite and are
 *                ignored).  Sample s of a level draws X(0) as normal (s mod 4) of Philox block 0
 *                of counter index floor(s / 4) (counter word as below); its fine and coarse paths
 *                both start from that X(0).  Paired with MLMC_SECOND_MOMENT, E[X(T)^2]. */
typedef enum mlmc_model_kind { MLMC_MODEL_GBM = 0, MLMC_MODEL_QUINTIC_ODE = 1 } mlmc_model_kind;
/* Time-stepping scheme on both grids, with drift f and step h:
 *   EULER_MARUYAMA  X + h f(X) + g(X) dW (Sec. 2, Eq. em); both models.
 *   MILSTEIN        (GBM) adds sigma^2 X (dW^2 - dt) / 2, the coarse step using the summed
 *                   increment and its own dt (Sec. 5, the strongly more accurate scheme).
 *   TAMED_EM        (QUINTIC_ODE) X + h f(X) / (1 + h |f(X)|): the tamed method that Sec. 5
 *                   cites as recovering multilevel convergence where explicit Euler--Maruyama
 *                   diverges. */
typedef enum mlmc_scheme { MLMC_EULER_MARUYAMA = 0, MLMC_MILSTEIN = 1, MLMC_TAMED_EM = 2 } mlmc_scheme;
typedef struct mlmc_model {
    int32_t kind;          /* mlmc_model_kind */
    int32_t scheme;        /* mlmc_scheme */
    double S0, r, sigma, T; /* GBM: S0 > 0, sigma > 0, T > 0, all finite; QUINTIC_ODE: T > 0 */
} mlmc_model;

/* Payoffs, discounted by exp(-r T) (Sec. 6):
 *   EUROPEAN  max(S_n - K, 0)                                   (Sec. 5, Sec. 6)
 *   ASIAN     max(A - K, 0), A = (1/n) sum_{i<n} (S_i + S_{i+1}) / 2 on the path's own grid
 *   LOOKBACK  max(max_{0<=i<=n} S_i - K, 0)  (fixed strike, discrete monitoring)
 *   DIGITAL   cash * 1{S_n > K}, cash / 2 when S_n == K        (Sec. 6)
 *   LINEAR_TEST     S_n, not discounted (test payoff with exact Euler--Maruyama moments)
 *   GEO_ASIAN_TEST  max(exp((1/n) sum (log S_i + log S_{i+1}) / 2) - K, 0) (closed-form test)
 *   SECOND_MOMENT   X_n^2, not discounted (the quantity of Sec. 5, Eq. count; QUINTIC_ODE only,
 *                   and the only payoff of that model)
 * The paper names the Asian and lookback options (Sec. 7) without defining them; the
 * definitions above are this library's reading. */
typedef enum mlmc_payoff_kind {
    MLMC_EUROPEAN = 0, MLMC_ASIAN = 1, MLMC_LOOKBACK = 2, MLMC_DIGITAL = 3, MLMC_SECOND_MOMENT = 4,
    MLMC_LINEAR_TEST = 100, MLMC_GEO_ASIAN_TEST = 101
} mlmc_payoff_kind;
/* What a level sample returns: the coupled difference Y = P_l - P_{l-1} of multilevel Monte
 * Carlo (Eq. Yldef); P_l alone -- standard Monte Carlo with Euler--Maruyama at step T / M^l
 * (Sec. 3), the comparison of Sec. 6; or the antithetic difference (Sec. 7: antithetic
 * variables inside multilevel Monte Carlo, after Giles and Szpruch)
 * Y = (P_l + P_l^a) / 2 - P_{l-1}, where the antithetic fine path P_l^a takes the same fine
 * increments with the M increments of every coarse step in reverse order (M = 2: swapped), so
 * it has the fine path's law and E[Y] is unchanged.  GBM with M = 2 or 4, one thread per
 * sample; cost 2 M^l + M^(l-1) steps.  Under GBM the step factors commute, so payoffs of S(T)
 * alone are unchanged; the trapezoid average and the maximum gain. */
typedef enum mlmc_estimator { MLMC_COUPLED = 0, MLMC_SINGLE_LEVEL = 1, MLMC_ANTITHETIC = 2 } mlmc_estimator;
typedef struct mlmc_payoff {
    int32_t kind;          /* mlmc_payoff_kind */
    int32_t estimator;     /* mlmc_estimator (mlmc_estimate: COUPLED or ANTITHETIC; batch and
                              control variate: COUPLED) */
    double K;              /* strike, finite */
    double cash;           /* digital cash amount (Sec. 6 uses 100), finite */
} mlmc_payoff;

/* Path arithmetic precision.  Moment sums are FP64 in all three. */
typedef enum mlmc_precision {
    MLMC_FP64 = 0,         /* FP64 normals (32-bit uniforms) and FP64 paths */
    MLMC_FP32_PATH = 1,    /* FP32 normals (23-bit uniforms) and FP32 paths */
    MLMC_FP64_STREAM32 = 2 /* FP64 arithmetic on the FP32 stream's 23-bit uniforms: the same samples
                              as MLMC_FP32_PATH, so the two differ by FP32 roundoff alone */
} mlmc_precision;

/* Random-number stream tags (the `tag` field of the Philox counter). */
enum { MLMC_TAG_PATHS = 0, MLMC_TAG_CV_MEAN = 1, MLMC_TAG_CV_TRAIN = 2 };

/* Launch shape of one level kernel.  Zero in a field means "choose automatically".
 *   threads_per_block  multiple of 32, 32..1024 (at most 512 with samples_per_thread = 2)
 *   lanes_per_path     1 (one thread per sample) or a power of two up to 32: that many lanes of
 *                      one warp split the time steps of one sample into equal chunks and join
 *                      them by a product scan (GBM's step is multiplicative); requires
 *                      M^l / lanes_per_path to be a multiple of max(M, 4); GBM only (QUINTIC_ODE
 *                      paths are nonlinear and run one thread per sample)
 *   blocks             grid size, blocks x threads_per_block below 2^31; the kernel strides
 *                      over the samples */
typedef struct mlmc_launch {
    int32_t threads_per_block;
    int32_t lanes_per_path;
    int32_t blocks;
    int32_t samples_per_thread;  /* 1 or 2 (0 = automatic): with 2, each thread of a one-thread-
                              per-sample launch steps two samples' paths in lockstep (two
                              independent Philox and step chains for the scheduler to interleave);
                              FP32 Euler--Maruyama paths of the coupled or single-level estimator
                              with M^l >= 4 and lanes_per_path = 1 only.  Thread t of a grid of
                              T threads takes samples t, t + T, ... as with 1, in pairs, and runs
                              an unpaired last sample alone; the automatic grid is the same.  The
                              samples and their Y are the same; the FP32 moment sums add them in
                              another order.  Automatic: 2 for FP32 Euler--Maruyama whole paths
                              with M = 4 and M^l >= 16, else 1 (or the autotuner's choice). */
} mlmc_launch;

/* Message describing the last failure on this host thread ("" if none). */
const char *mlmc_last_error(void);

/* Library version string. */
const char *mlmc_version(void);

/*
 * mlmc_level_sums -- the level estimator of Sec. 5, Eq. (Yldef) (Eq. mlmc:Yzero at l = 0),
 * in its short form: samples [0, N), FP32 paths, tag MLMC_TAG_PATHS, default stream.
 *   level   0..12, with M^level <= 2^24
 *   M       refinement factor of Eq. (mlmc:Dtl): 2, 4 or 8
 *   N       number of samples (0 gives zero sums and cost)
 *   model, payoff   host, read only
 *   seed    64-bit Philox key
 *   sums    host, 4 doubles written: sum over samples of Y, Y^2, Y^3, Y^4
 *   cost    host, 1 double written: N * C_l with C_0 = 1, C_l = M^l + M^(l-1), the number of
 *           Euler--Maruyama steps taken (the cost measure of Sec. 3)
 * Errors: MLMC_EINVAL for out-of-range arguments or NULL pointers; MLMC_ECUDA if a CUDA call
 * fails (no device, launch failure).
 */
int mlmc_level_sums(int level, int M, uint64_t N, const mlmc_model *model,
                    const mlmc_payoff *payoff, uint64_t seed, double sums[4], double *cost);

/*
 * mlmc_level_sums_ex -- the same estimator over samples [first, first + N) with explicit
 * precision, random-stream tag, launch shape (NULL = automatic) and stream.  Adaptive drivers
 * pass first = the number of samples already taken on this level, so that every round draws
 * new samples.  Host outputs as in mlmc_level_sums; synchronises `stream`.  The engine
 * allocates its small reduction workspace with stream-ordered allocation on `stream`.
 * Errors: as mlmc_level_sums; MLMC_EINVAL also if first + N overflows 64 bits or the launch
 * shape is invalid for this level.
 */
int mlmc_level_sums_ex(int level, int M, uint64_t N, uint64_t first, const mlmc_model *model,
                       const mlmc_payoff *payoff, uint64_t seed, int precision, int tag,
                       const mlmc_launch *launch, void *stream, double sums[4], double *cost);

/* Bytes of device workspace that mlmc_level_sums_async needs for this launch shape
 * (NULL = automatic shape); 0 on invalid arguments. */
size_t mlmc_level_workspace_bytes(int level, int M, uint64_t N, int precision,
                                  const mlmc_launch *launch);

/*
 * mlmc_level_sums_async -- queue the level estimator on `stream` with device outputs:
 *   d_sums       device, 4 doubles overwritten with sum Y^k, k = 1..4
 *   d_workspace  device, at least mlmc_level_workspace_bytes(...) bytes, 256-byte aligned.
 *                Its first 256 bytes hold a completion counter that must be zero before the
 *                first launch; every launch leaves it zero again.  The rest holds per-block
 *                partial sums and needs no initial value.  One workspace may serve launches of
 *                any level and grid size as long as they are ordered (same stream).
 *   d_y          device or NULL: if not NULL, N doubles receive Y of each sample in order
 * Never synchronises and allocates nothing.  Errors: MLMC_EINVAL (also for a workspace that is
 * too small or misaligned), MLMC_ECUDA for a failed launch.
 */
int mlmc_level_sums_async(int level, int M, uint64_t N, uint64_t first,
                          const mlmc_model *model, const mlmc_payoff *payoff, uint64_t seed,
                          int precision, int tag, const mlmc_launch *launch, double *d_sums,
                          void *d_workspace, size_t workspace_bytes, double *d_y, void *stream);

/*
 * mlmc_level_sums_noalloc -- mlmc_level_sums_async for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant of the level estimator.
 * Some callers must not allocate at run time: latency-critical loops where a cudaMalloc or
 * cudaFree would synchronise the device or take an unpredictable time, processes whose device
 * memory is already claimed by another allocator, and deployments whose rules forbid dynamic
 * allocation after start-up.  This entry point allocates nothing: its reduction scratch is a
 * fixed array in the library's device memory, 2048 blocks of partial sums plus a completion
 * word (64 KiB + 256 bytes), which every GPU that loads the library holds until the process
 * exits.
 *   Arguments as mlmc_level_sums_async, without the workspace.  d_sums (device, 4 doubles)
 *   is overwritten; d_y (device or NULL) receives Y per sample.
 *   A grid that the planner sizes above 2048 blocks (small blocks on a large range) is cut
 *   to 2048 blocks, each striding over more samples: the samples and d_y are those of
 *   mlmc_level_sums_async, and the sums equal its sums bit for bit only when its grid has at
 *   most 2048 blocks; otherwise they add the same samples in another order (FP32 batches of
 *   32 and block partials), within the oracle tolerances of both.
 *   The first call on each device looks up the array's device address (with that device
 *   current) and caches it; make that first call before any stream capture.  mlmc_shutdown
 *   forgets the cached address of the current device: call it before resetting the device
 *   (a reset or a new primary context moves the array), so that the next call looks it up
 *   again.
 *   All calls share the one array: each call clears the completion word on `stream` before
 *   its launch, and calls whose work overlaps on the GPU (different streams, or different
 *   host threads without ordering) race on it.
 * Errors: MLMC_EINVAL as mlmc_level_sums_async, and for an explicit launch->blocks above 2048
 * (the message states the scratch needed and the scratch held); MLMC_ECUDA for a failed lookup
 * or launch.
 */
int mlmc_level_sums_noalloc(int level, int M, uint64_t N, uint64_t first, const mlmc_model *model,
                            const mlmc_payoff *payoff, uint64_t seed, int precision, int tag,
                            const mlmc_launch *launch, double *d_sums, double *d_y, void *stream);

/* Result of one adaptive estimate (Sec. 5).  Arrays are indexed by level 0..L. */
#define MLMC_MAX_LEVELS 16
typedef struct mlmc_result {
    double P;                        /* estimate sum_l mean_l, Eq. (mlmc:ident) */
    double eps;                      /* requested root-mean-square accuracy */
    int32_t L;                       /* finest level used */
    int32_t converged;               /* 1 if the bias test passed */
    int32_t rounds;                  /* sampling rounds taken */
    int32_t device_rounds;           /* 1 if the rounds ran on the device (one graph launch), 0 if
                                        the host ran them (mlmc_set_driver_mode) */
    uint64_t N[MLMC_MAX_LEVELS];      /* samples per level */
    double sums[MLMC_MAX_LEVELS][4];  /* sum Y^k per level */
    double mean[MLMC_MAX_LEVELS];     /* sample mean of Y_l */
    double var[MLMC_MAX_LEVELS];      /* sample variance of Y_l */
    double cost[MLMC_MAX_LEVELS];     /* N_l C_l */
    double alpha, beta;              /* fitted weak and variance rates (base M) */
    double total_cost;               /* sum_l N_l C_l */
    double path_steps;               /* sum_l N_l M^l: coupled fine steps simulated */
    double kernel_ms;                /* device time of the level kernels (device rounds: of the whole
                                        graph, driver kernels included) */
    double wall_ms;                  /* host wall time of the call */
    uint64_t launches;               /* kernel launches made (device rounds: level kernels and
                                        driver iterations) */
    uint64_t d2h_bytes;              /* bytes copied device to host (host rounds: the round sums;
                                        device rounds: the final state, once) */
} mlmc_result;

/* Where mlmc_estimate runs its rounds.  The paper has no counterpart (host/device placement of
 * the driver's arithmetic).
 *   MLMC_DRIVER_HOST (default): every round's sums come back to the host, which decides the next
 *     round (on GB300 with its Grace host the faster form: a round trip costs about 16 us, the
 *     device form's driver kernel about 35 us, most of it the FP64 update's dependent chain);
 *   MLMC_DRIVER_DEVICE: on the device or MLMC_ENOTIMPL (no host round trip: the whole estimate
 *     is one graph launch, for callers whose host must not take part between rounds);
 *   MLMC_DRIVER_AUTO: on the device where the device form covers the problem (GBM, coupled or
 *     antithetic estimator), on the host otherwise or where the device form cannot be built.
 * Device rounds: one CUDA graph per problem shape (cached per device until mlmc_shutdown) whose
 * WHILE node repeats a one-warp driver kernel -- the host driver's FP64 update of means,
 * variances, rates, N_l, the bias test and the added level, in the same order -- and the level
 * kernels it configures by device-side graph updates (sample range, lanes per path, grid; the
 * host planner's built-in shapes, not an autotuned table).  The host launches the graph once and
 * reads the final state once.  Both forms run the same kernels on the same ranges and grids, so
 * their estimates agree; only a decision taken exactly at a rounding boundary of CUDA's FP64 log
 * or pow could differ.  Process-wide; *previous (host, may be NULL) receives the mode it replaces.
 * MLMC_EINVAL for an unknown mode (the mode is then unchanged). */
enum { MLMC_DRIVER_AUTO = 0, MLMC_DRIVER_HOST = 1, MLMC_DRIVER_DEVICE = 2 };
int mlmc_set_driver_mode(int mode, int *previous);

/*
 * mlmc_estimate -- adaptive multilevel Monte Carlo estimate of E[h(X(T))] to root-mean-square
 * accuracy eps (Sec. 5; mean-square error bound of the Theorem in Sec. 5).
 *   Start with levels 0..Lmin and N0 samples each.  After every round of sampling, estimate
 *   V_l and set N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)) (the variance target
 *   eps^2 / 2 at least cost, the pre-processing optimisation remarked on in Sec. 5).  When no
 *   level needs more than 1% more samples, test the bias estimate
 *   max(|m_L|, |m_{L-1}| / M^alpha) / (M^alpha - 1) against eps / sqrt(2) and add a level
 *   (variance extrapolated as V_{L-1} / M^beta) if it fails.  alpha, beta are least-squares
 *   slopes over levels 1..L, floored at 1/2; for l >= 2 the means and variances used in these
 *   formulas are floored at half the extrapolation from the level below.
 *   eps > 0; M in {2, 4, 8}; 1 <= Lmin <= Lmax < MLMC_MAX_LEVELS, M^Lmax <= 2^24; N0 >= 2.
 *   model, payoff  host, read only.  out  host, written on success and on MLMC_ENOTCONV.
 *   stream  void* cudaStream_t (NULL = default); synchronised before return.  A round's level
 *           launches run on `stream` and on three streams of the library's own, which wait for
 *           the work queued on `stream` before the round and which `stream` waits for after it;
 *           results do not depend on how the launches overlap.
 * Errors: MLMC_EINVAL, MLMC_ECUDA, MLMC_ENOMEM; MLMC_ENOTCONV when Lmax is reached first
 * (out then holds the estimate at L = Lmax); MLMC_ENONFINITE when a round's level sums are
 * not finite (explicit Euler--Maruyama on QUINTIC_ODE, Sec. 5), out left untouched.
 */
int mlmc_estimate(double eps, int M, int Lmin, int Lmax, uint64_t N0, const mlmc_model *model,
                  const mlmc_payoff *payoff, uint64_t seed, int precision, void *stream,
                  mlmc_result *out);

/* One problem of a batch: model, payoff, accuracy and seed. */
typedef struct mlmc_problem {
    mlmc_model model;
    mlmc_payoff payoff;
    double eps;                      /* requested root-mean-square accuracy, > 0 */
    uint64_t seed;                   /* Philox key of this problem's samples */
} mlmc_problem;

/*
 * mlmc_estimate_batch -- n independent adaptive estimates (each as mlmc_estimate, Sec. 5),
 * computed together.  Every round gathers the new samples of all unfinished problems on all
 * their levels into one list of chunks of about equal work; one persistent kernel works through
 * the list (each block claims the next chunk from a counter; deep levels with few samples split
 * every path over several lanes), and a second kernel adds each (problem, level)'s chunk sums in
 * a fixed order, so results do not depend on scheduling.  The round's upload, both kernels and
 * the download are captured once in a CUDA graph and replayed every round.
 *   n >= 1; problems host [n], read only; M, Lmin, Lmax, N0, precision as mlmc_estimate and
 *   shared by all problems; stream as mlmc_estimate (the batch runs on its own stream after
 *   `stream` has drained, and is finished on return).
 *   results host [n], written for every problem.  kernel_ms, wall_ms, launches and d2h_bytes
 *   describe the whole batch (the same values in every result).
 * GBM problems only (other models: MLMC_ENOTIMPL).
 * Returns MLMC_OK when every problem converged, MLMC_ENOTCONV when some reached Lmax first
 * (their results carry converged = 0 and the estimate at Lmax), MLMC_EINVAL for a bad argument
 * (the message names the problem), MLMC_ECUDA or MLMC_ENOMEM for device failures.
 */
int mlmc_estimate_batch(int n, const mlmc_problem *problems, int M, int Lmin, int Lmax, uint64_t N0,
                        int precision, void *stream, mlmc_result *results);

/* One level range of a batch: samples [first, first + N) of `level` of one problem (its eps is
 * not used). */
typedef struct mlmc_level_task {
    mlmc_problem problem;
    int32_t level;
    int32_t reserved;                /* must be 0 */
    uint64_t first, N;               /* N at most 2^32 - 1 */
} mlmc_level_task;

/*
 * mlmc_level_sums_batch -- the level estimator (Sec. 5, Eq. Yldef; Eq. mlmc:Yzero at l = 0) for
 * n ranges at once, through the batched driver's own round: the same chunk list of about equal
 * work, persistent kernel and fixed-order per-task reduction as one round of
 * mlmc_estimate_batch (launched directly, not from a graph).
 *   tasks host [n]; M and precision (MLMC_FP64 or MLMC_FP32_PATH) shared by all tasks.
 *   sums host [n][4]: sum Y^k, k = 1..4, of each task's samples (zeros for N = 0).
 *   d_y device or NULL: if not NULL, Y of every sample, task after task in order (sum of N
 *   doubles); deep levels split paths over lanes as the batched rounds do, so Y carries that
 *   split's roundoff.  Synchronises `stream`.
 * GBM problems with the coupled Euler--Maruyama estimator only.  Errors as mlmc_estimate_batch.
 */
int mlmc_level_sums_batch(int n, const mlmc_level_task *tasks, int M, int precision, double *sums,
                          double *d_y, void *stream);

/*
 * ---------------------------------------------------------------- learned control variate
 * A control variate replaces E[Y_l] by E[Y_l - g] + E[g] (Sec. 5 "Exploiting Structure":
 * compute E[X - Y] and add E[Y]).  Here g is a network 16 -> 64 -> 64 -> 1 of the sample's
 * Brownian path, trained per level on (inputs, Y_l) pairs the method itself generates:
 *   x = the Brownian-bridge (Levy) coordinates of the path on the T/16 grid (iid N(0,1)):
 *   x_0 = W(T) / sqrt(T), then stage by stage (intervals of 16, 8, 4, 2 grid steps) and left to
 *   right (W(m) - (W(l) + W(r)) / 2) / sqrt((r - l) / 4), m the midpoint of [l, r]; on levels with
 *   M^l < 16 the T/16 grid is refined from the path's grid by Brownian-bridge midpoints (stage by
 *   stage, left to right) taken from the Philox blocks of the sample's counter that its path does
 *   not read, from block max(1, M^l / 4) on;
 *   g(x) = w3 . GELU(W2 GELU(W1 x + b1) + b2) + b3, GELU(z) = z/2 (1 + tanh(sqrt(2/pi)
 *   (z + 0.044715 z^3))); products on the tensor cores with bfloat16 operands and FP32
 *   accumulation (rounded: x, W1, W2, GELU(z1)); everything else FP32;
 *   packed parameters (MLMC_CV_PARAMS floats): W1 [64][16] (row = output unit), b1 [64],
 *   W2 [64][64], b2 [64], w3 [64], b3.
 * The level estimator with the control variate is mean over N samples of (Y - g(x)) plus an
 * independent estimate of E[g]: the average of R replicate means Q_r of a randomly shifted
 * rank-1 lattice rule (Sloan and Joe 1994; random shift after Cranley and Patterson 1976).
 * Replicate r has the n = MLMC_CV_LATTICE_POINTS points i = 0 .. n-1 with coordinates, k = 0..15,
 *   v_k = ((i z_k mod n) 2^16 + D_k) mod 2^32,  z_k = a^k mod n (a = MLMC_CV_LATTICE_A),
 *   w_k = 2 v_k if v_k < 2^31, else 2 (2^32 - 1 - v_k)  (the baker's, or tent, transform
 *         u -> 1 - |2u - 1|, which keeps points uniform and suits non-periodic integrands),
 *   u_k = (floor(w_k / 2^9) + 1/2) 2^-23,  x_k = Phi^{-1}(u_k),
 * where D_0..D_15 are the words of Philox blocks 0..3 of counter r under tag
 * MLMC_TAG_CV_MEAN (the random shift, as 32-bit fractions).  Every point is uniform whatever
 * the shift, so Q_r is unbiased for E[g] for any g, and replicates are independent; the lattice
 * makes Var(Q_r) far smaller than Var(g) / n for a smooth g.  kappa is the number of lattice
 * points per path sample (R = ceil(kappa N / n), at least 8 replicates).  A level uses the
 * control variate only while its measured work-weighted variance
 * (Var(Y - g) + var_lattice / kappa) (t_cv + kappa t_mean) stays below Var(Y) t_plain, with
 * var_lattice = n Var(Q_r); otherwise the plain estimator runs.  FP32 paths only.
 */
#define MLMC_CV_PARAMS 5313
#define MLMC_CV_INPUTS 16              /* network inputs: the Levy coordinates of the T/16 grid */
#define MLMC_CV_LATTICE_POINTS 65536   /* points n of one mean-sample replicate */
#define MLMC_CV_LATTICE_A 43833        /* Korobov multiplier a of the mean-sample lattice */
#define MLMC_CV_MAX_LEVELS 8
typedef struct mlmc_cv mlmc_cv;   /* opaque; owns device memory */

typedef struct mlmc_cv_options {
    int32_t levels;        /* train levels 0 .. levels-1, 1..8 (0 = 4) */
    int32_t epochs;        /* passes over the training set (0 = 20) */
    int32_t batch;         /* mini-batch rows, a multiple of 256 (0 = 4096) */
    int32_t reserved;      /* must be 0 */
    uint64_t n_train;      /* samples per level (0 = 10^6); the last tenth is held out */
    double lr;             /* Adam step size (0 = 1e-3) */
    uint64_t init_seed;    /* seed of the initial weights */
} mlmc_cv_options;

typedef struct mlmc_cv_level_info {
    int32_t trained;       /* 1 if this level has a network */
    int32_t used;          /* 1 if the estimator uses the control variate on this level */
    double var_plain;      /* Var(Y) on the held-out samples */
    double var_resid;      /* Var(Y - g) on the held-out samples */
    double var_g;          /* Var(g) on the held-out samples */
    double kappa;          /* lattice points per path sample, in [1/64, 4096] */
    double t_plain, t_cv, t_mean;   /* measured seconds per path sample (plain, control variate)
                                       and per lattice point (mean) */
    double work_ratio;     /* (var_resid + var_lattice / kappa)(t_cv + kappa t_mean) / (var_plain t_plain) */
    double train_loss;     /* final mean training loss (standardised targets) */
    double var_lattice;    /* n Var(Q_r) over 128 replicates: per-point variance of the lattice mean
                              (var_g / var_lattice is the lattice rule's gain over plain sampling) */
} mlmc_cv_level_info;

/* Where the time of one mlmc_cv_train call went (host clock, milliseconds) and how it trained. */
typedef struct mlmc_cv_train_stats {
    double data_ms;        /* training data of every level, target standardisation, initial weights */
    double train_ms;       /* the training launch (host clock, launch to completion) */
    double train_kernel_ms;/* the same launch timed by CUDA events on the training stream */
    double eval_ms;        /* held-out variance ratios */
    double cost_ms;        /* timed kernel costs and the lattice statistics of every level */
    double total_ms;       /* the whole call */
    int64_t steps;         /* Adam steps per network (epochs x batches per epoch) */
    int32_t cluster;       /* CTAs per thread-block cluster: one cluster trains one level's network */
    int32_t levels;        /* networks trained side by side in the one launch */
} mlmc_cv_train_stats;

/* Create a control variate for one problem with no trained level (every level plain).
 * M as mlmc_estimate; model, payoff host, read only.  *out receives the handle. */
int mlmc_cv_create(int M, const mlmc_model *model, const mlmc_payoff *payoff, mlmc_cv **out);

/* Train networks for levels 0 .. opts->levels - 1 (opts NULL = defaults) on samples drawn under
 * tag MLMC_TAG_CV_TRAIN with `seed`, then measure each level's variance ratio and kernel costs
 * and decide which levels use it.  Synchronises `stream`.  *out receives the handle.
 * Training minimises the mean squared error of g against the standardised Y with Adam
 * (beta1 0.9, beta2 0.999, 1e-8) over mini-batches taken in order, `epochs` passes over the
 * first nine tenths of the samples; all levels train at once in one launch (one thread-block
 * cluster of 16 CTAs per level where the GPU can place it, else 8), forward, backward, gradient
 * and update of every step inside it.  MLMC_ECUDA if no cluster of 8 fits. */
int mlmc_cv_train(int M, const mlmc_model *model, const mlmc_payoff *payoff, uint64_t seed,
                  const mlmc_cv_options *opts, void *stream, mlmc_cv **out);

/* Timings and shape of the mlmc_cv_train call that made `cv` (zeros for a handle from
 * mlmc_cv_create).  The paper has no counterpart (cost accounting of the learned part). */
int mlmc_cv_train_info(const mlmc_cv *cv, mlmc_cv_train_stats *out);

/* Release a handle (NULL is ignored). */
int mlmc_cv_free(mlmc_cv *cv);

/* Statistics of one level (host output). */
int mlmc_cv_info(const mlmc_cv *cv, int level, mlmc_cv_level_info *out);

/* Read / install the packed FP32 parameters of one level (host arrays of MLMC_CV_PARAMS).
 * Installing marks the level trained and used with the given kappa (lattice points per path
 * sample, in [1/64, 4096]); the statistics are left at zero. */
int mlmc_cv_get_params(const mlmc_cv *cv, int level, float *params);
int mlmc_cv_set_params(mlmc_cv *cv, int level, const float *params, double kappa);

/* Control-variate level sums over samples [first, first + N) of `level` (tag MLMC_TAG_PATHS):
 * d_sums8 device, 8 doubles: sum r, r^2, r^3, r^4 (r = Y - g(x)), sum Y, Y^2, sum g, g^2.
 * d_r, d_g device or NULL: per-sample r and g (float).  Synchronises `stream`. */
int mlmc_cv_level_sums(const mlmc_cv *cv, int level, uint64_t N, uint64_t first, uint64_t seed,
                       double *d_sums8, float *d_r, float *d_g, void *stream);

/* The lattice mean sample of `level`, replicates [first, first + R): d_sums2 device, 2 doubles
 * (sum Q_r, sum Q_r^2, Q_r the mean of g over replicate r's n points); d_g device [R][n] (g of
 * every point) or NULL.  Synchronises `stream`. */
int mlmc_cv_mean_sums(const mlmc_cv *cv, int level, uint64_t R, uint64_t first, uint64_t seed,
                      double *d_sums2, float *d_g, void *stream);

/* Training data of `level`: d_X device [N][16] network inputs, d_Y device [N] Y values, for
 * samples [first, first + N) under tag MLMC_TAG_CV_TRAIN.  Synchronises `stream`. */
int mlmc_cv_training_data(const mlmc_cv *cv, int level, uint64_t N, uint64_t first, uint64_t seed,
                          float *d_X, float *d_Y, void *stream);

/* The network on given inputs: params host [MLMC_CV_PARAMS]; d_X device [N][16]; d_G device [N].
 * mlmc_mlp_grad: loss (1/N) sum (g - Y)^2 and its gradient (host outputs) for rows d_X, d_Y
 * (device); N a multiple of 32, at most 65536.  The gradient comes from the training kernel's
 * own forward and backward code (one step, no update).  Both synchronise `stream`. */
int mlmc_mlp_forward(const float *params, const float *d_X, uint64_t N, float *d_G, void *stream);
int mlmc_mlp_grad(const float *params, const float *d_X, const float *d_Y, uint64_t N, float *grad,
                  double *loss, void *stream);

/* mlmc_estimate with the control variate on the levels `cv` uses (FP32 paths; the problem must be
 * the one cv was made for).  Level means are mean(Y - g) + mean'(g) on those levels. */
int mlmc_estimate_cv(double eps, int M, int Lmin, int Lmax, uint64_t N0, const mlmc_model *model,
                     const mlmc_payoff *payoff, uint64_t seed, const mlmc_cv *cv, void *stream,
                     mlmc_result *out);

/*
 * ---------------------------------------------------------------- autotuner
 * mlmc_autotune -- time candidate launch shapes of the level kernel (threads per block in
 * {128, 256, 512}, every valid lanes_per_path, one or two samples per thread where the two-sample
 * kernel applies, one or two waves of resident blocks) for
 * levels 0..max_level of (precision, payoff, M) at N = 2^10, 2^13, ... (up to 2e9 fine steps per
 * launch), keeping the fastest per size class.  Whenever a caller leaves launch fields at zero
 * the library then uses the tuned values of the nearest size class at or below N.  A different
 * lanes_per_path changes path roundoff, not the samples.  The paper has no counterpart (launch
 * tuning).  entries (host, may be NULL) receives the number of table entries added.
 * The table is process-wide.  MLMC_AUTOTUNE_CACHE names a file loaded on first use.
 */
int mlmc_autotune(int M, int max_level, int precision, int payoff, void *stream, int *entries);
/* Write the table as JSON (one entry per line) / read such a file (adds to the table). */
int mlmc_autotune_save(const char *path);
int mlmc_autotune_load(const char *path, int *entries);
/* Empty the table (the library returns to its built-in launch heuristic). */
int mlmc_autotune_clear(void);
/* Number of table entries. */
int mlmc_autotune_entries(void);
/* Tuned shape for (precision, payoff, M, level, N): threads_per_block, lanes_per_path,
 * samples_per_thread, and in `blocks` the number of waves of resident blocks; MLMC_EINVAL if the
 * table has none. */
int mlmc_autotune_lookup(int precision, int payoff, int M, int level, uint64_t N, mlmc_launch *out);

/* Number of streaming multiprocessors of the current device, or -1 with an error message. */
int mlmc_device_sm_count(void);

/* Release every device resource the library holds on the current device (the adaptive drivers'
 * pooled buffers) and forget the cached address of the allocation-free entry point's scratch.
 * Call it before cudaDeviceReset or any other teardown of the device's primary context. */
int mlmc_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_GB300_H */
