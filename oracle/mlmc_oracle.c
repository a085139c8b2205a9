/*
 * mlmc_oracle.c -- plain, slow FP64 CPU reference of one multilevel Monte Carlo level.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no source with the CUDA path: the random stream is re-implemented here from its
 * published definition, and every formula is written out in the order the paper states it.
 *
 * Method (D. J. Higham, "An Introduction to Multilevel Monte Carlo for Option Valuation"):
 *   - SDE dX = f(X) dt + g(X) dW                                   (Sec. 2, Eq. sde)
 *   - Euler--Maruyama  X_{n+1} = X_n + f(X_n) dt + g(X_n) dW_n     (Sec. 2, Eq. em)
 *     for GBM f(x) = r x, g(x) = sigma x                           (Sec. 6 uses this model)
 *   - level step sizes dt_l = M^{-l} T                             (Sec. 5, Eq. mlmc:Dtl)
 *   - Y_0 = mean of P_0, Y_l = mean of P_l - P_{l-1}               (Sec. 5, Eqs. mlmc:Yzero, Yldef)
 *   - P_l and P_{l-1} come from the same Brownian path; the coarse increments are sums of
 *     M consecutive fine increments                                (Sec. 5, Fig. 2)
 *   - fresh, independent random numbers on every level             (Sec. 5, after Eq. Yldef)
 *   - cost per path proportional to the number of f, g evaluations (Sec. 3)
 *   - discounted call and digital payoffs, h(K) = half the cash    (Sec. 6)
 *
 * Readings where the paper is silent (the Asian and lookback payoffs are only named in Sec. 7;
 * the random stream is not specified at all):
 *   - Random stream: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Key = (seed low 32
 *     bits, seed high 32 bits).  Counter = ((tag << 16) | level, j, s high, s low) where j is
 *     the call index inside one sample and s the sample index inside the level.  Call j gives
 *     four words x0..x3; the pairs (x0,x1) and (x2,x3) each give two normals by Box--Muller.
 *   - Uniforms from a 32-bit word x: FP64 stream u = (x + 1) 2^-32; FP32 stream
 *     u = 1 - (x mod 2^23) 2^-23 (the low 23 bits, exactly a float mantissa).  Both lie in
 *     (0, 1], so log(u) is finite.
 *   - Box--Muller: rho = sqrt(-2 log u1), z0 = rho cos(2 pi u2), z1 = rho sin(2 pi u2).
 *   - Fine step k of sample s (k < M^l) takes normal k of the sample: dW_k = sqrt(dt_l) z_k,
 *     where the sample's normals are those of its blocks j = 0, 1, ... in order.  When
 *     M^l < 4 (level 0, and level 1 for M = 2), G = 4 / M^l consecutive samples share one
 *     block: sample s takes normals (s mod G) M^l .. (s mod G) M^l + M^l - 1 of block j = 0 of
 *     counter index floor(s / G) (in place of s).
 *   - The Brownian path on the T/16 grid (the learned control variate's inputs) is the running
 *     sum of the fine increments when M^l >= 16.  On coarser levels it is refined from the
 *     fine-grid values by Brownian-bridge midpoints, stage by stage and left to right; the
 *     midpoints take the normals of the sample's own counter from block b0 = max(1, M^l / 4)
 *     on, the first block its fine path does not read.  The fine path never depends on whether
 *     the grid is built.
 *   - Arithmetic Asian: trapezoid average (1/n) sum_{i<n} (S_i + S_{i+1}) / 2 on each path's own
 *     grid.  Lookback: fixed strike, max over the grid points S_0..S_n.  Both discounted.
 *   - Cost of one level-l sample: C_0 = 1, C_l = M^l + M^{l-1} Euler--Maruyama steps.
 *   - Antithetic mode (Sec. 7, the antithetic multilevel estimator of Giles and Szpruch): a
 *     second fine path takes the M fine increments of every coarse step in reverse order (for
 *     M = 2, swapped); the coarse path is unchanged and Y = (P_f + P_f^a) / 2 - P_c.  Cost
 *     C_l = 2 M^l + M^{l-1}.  On level 0 it is the plain estimator.
 *   - Milstein scheme (Sec. 5, the strongly more accurate scheme that gives beta > gamma): for
 *     g(x) = sigma x the step adds (1/2) g g' (dW^2 - dt) = (1/2) sigma^2 X (dW^2 - dt); the coarse
 *     step uses the coarse increment (the sum of the fine ones) and its own step size.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

enum { PAY_EUROPEAN = 0, PAY_ASIAN = 1, PAY_LOOKBACK = 2, PAY_DIGITAL = 3,
       PAY_LINEAR = 100, PAY_GEO_ASIAN = 101 };
enum { STREAM_FP64 = 0, STREAM_FP32 = 1 };
enum { MODE_COUPLED = 0, MODE_FINE_ONLY = 1, MODE_ANTITHETIC = 2 };

/* ---------------------------------------------------------------- random stream ---------- */

/* Philox4x32-10 bijection of a 128-bit counter under a 64-bit key (SC'11 definition). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {                       /* Weyl key schedule between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double oracle_uniform(uint32_t x, int stream)
{
    if (stream == STREAM_FP32)
        return 1.0 - (double)(x & 0x7FFFFFu) * 0x1p-23;
    return ((double)x + 1.0) * 0x1p-32;
}

/* The first n normals of sample s at this level (n a multiple of 4). */
void oracle_normals(uint64_t seed, int level, int tag, uint64_t s, int stream, int n, double *z)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int j = 0; 4 * j < n; ++j) {
        uint32_t ctr[4] = { ((uint32_t)tag << 16) | (uint32_t)level, (uint32_t)j, (uint32_t)(s >> 32),
                            (uint32_t)s };
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = oracle_uniform(x[2 * pair], stream);
            double u2 = oracle_uniform(x[2 * pair + 1], stream);
            double rho = sqrt(-2.0 * log(u1));
            z[4 * j + 2 * pair]     = rho * cos(2.0 * ORACLE_PI * u2);
            z[4 * j + 2 * pair + 1] = rho * sin(2.0 * ORACLE_PI * u2);
        }
    }
}

/* ---------------------------------------------------------------- paths and payoffs ------ */

static long ipow(long b, int e) { long p = 1; while (e-- > 0) p *= b; return p; }

/* The M^l normals of sample s's fine increments (the packing rule above). */
void oracle_sample_normals(uint64_t seed, int level, int M, int tag, uint64_t s, int stream,
                           double *z)
{
    long nf = ipow(M, level);
    if (nf < 4) {
        long group = 4 / nf;
        double z4[4];
        oracle_normals(seed, level, tag, s / (uint64_t)group, stream, 4, z4);
        long slot = (long)(s % (uint64_t)group);
        for (long k = 0; k < nf; ++k)
            z[k] = z4[slot * nf + k];
    } else {
        oracle_normals(seed, level, tag, s, stream, (int)nf, z);
    }
}

/* Euler--Maruyama for GBM over n steps of size h driven by the given increments (Eq. em). */
void oracle_em_path(int n, double S0, double r, double sigma, double h, const double *dW,
                    double *path)
{
    path[0] = S0;
    for (int i = 0; i < n; ++i) {
        double X = path[i];
        path[i + 1] = X + r * X * h + sigma * X * dW[i];
    }
}

/* Milstein for GBM: the Euler--Maruyama step plus (1/2) sigma^2 X (dW^2 - h). */
void oracle_milstein_path(int n, double S0, double r, double sigma, double h, const double *dW,
                          double *path)
{
    path[0] = S0;
    for (int i = 0; i < n; ++i) {
        double X = path[i];
        path[i + 1] = X + r * X * h + sigma * X * dW[i] + 0.5 * sigma * sigma * X * (dW[i] * dW[i] - h);
    }
}

/* Discounted payoff of a path S_0..S_n on [0, T]. */
double oracle_payoff(int payoff, double K, double Q, double r, double T, const double *path,
                     int n)
{
    double disc = exp(-r * T);
    double ST = path[n];
    switch (payoff) {
    case PAY_EUROPEAN:
        return disc * (ST > K ? ST - K : 0.0);
    case PAY_ASIAN: {
        double acc = 0.0;
        for (int i = 0; i < n; ++i)
            acc += 0.5 * (path[i] + path[i + 1]);
        double A = acc / n;
        return disc * (A > K ? A - K : 0.0);
    }
    case PAY_LOOKBACK: {
        double mx = path[0];
        for (int i = 1; i <= n; ++i)
            if (path[i] > mx) mx = path[i];
        return disc * (mx > K ? mx - K : 0.0);
    }
    case PAY_DIGITAL:
        if (ST > K) return disc * Q;
        if (ST == K) return disc * 0.5 * Q;
        return 0.0;
    case PAY_LINEAR:
        return ST;
    case PAY_GEO_ASIAN: {
        double acc = 0.0;
        for (int i = 0; i < n; ++i)
            acc += 0.5 * (log(path[i]) + log(path[i + 1]));
        double G = exp(acc / n);
        return disc * (G > K ? G - K : 0.0);
    }
    default:
        return NAN;
    }
}

typedef struct {
    double S0, r, sigma, T;
    int payoff;
    double K, Q;
    int scheme;  /* 0 Euler--Maruyama, 1 Milstein */
} oracle_problem;

static void scheme_path(const oracle_problem *p, int n, double h, const double *dW, double *path)
{
    if (p->scheme == 1)
        oracle_milstein_path(n, p->S0, p->r, p->sigma, h, dW, path);
    else
        oracle_em_path(n, p->S0, p->r, p->sigma, h, dW, path);
}

/*
 * One coupled sample of level l: fills the fine increments (M^l), the fine path (M^l + 1
 * values) and, for l > 0, the coarse path (M^{l-1} + 1 values) built from sums of M
 * consecutive fine increments (Fig. 2).  Returns the number of fine steps.
 */
int oracle_sample_paths(int level, int M, uint64_t s, int tag, const oracle_problem *p,
                        uint64_t seed, int stream, double *dWf, double *fine, double *coarse)
{
    long nf = ipow(M, level);
    double *z = (double *)malloc(sizeof(double) * (size_t)nf);
    oracle_sample_normals(seed, level, M, tag, s, stream, z);
    double sqrt_h = sqrt(p->T / (double)nf);
    for (long k = 0; k < nf; ++k)
        dWf[k] = sqrt_h * z[k];
    free(z);
    double hf = p->T / (double)nf;
    scheme_path(p, (int)nf, hf, dWf, fine);
    if (level > 0 && coarse) {
        long nc = nf / M;
        double *dWc = (double *)malloc(sizeof(double) * (size_t)nc);
        for (long c = 0; c < nc; ++c) {
            double acc = 0.0;
            for (int q = 0; q < M; ++q)
                acc += dWf[c * M + q];
            dWc[c] = acc;
        }
        scheme_path(p, (int)nc, hf * M, dWc, coarse);
        free(dWc);
    }
    return (int)nf;
}

/* Brownian values W(k T / 16), k = 1..16, of one sample (the T/16 grid of the stream). */
void oracle_grid_brownian(int level, int M, uint64_t s, int tag, double T, uint64_t seed,
                          int stream, double W16[16])
{
    long nf = ipow(M, level);
    double *z = (double *)malloc(sizeof(double) * (size_t)(nf > 16 ? nf : 16));
    oracle_sample_normals(seed, level, M, tag, s, stream, z);
    double sqrt_h = sqrt(T / (double)nf);
    if (nf >= 16) {
        long per16 = nf / 16;
        double W = 0.0;
        for (int k = 0; k < 16; ++k) {
            for (long q = 0; q < per16; ++q)
                W += sqrt_h * z[k * per16 + q];
            W16[k] = W;
        }
    } else {
        /* grid[i] = W(i T / 16), i = 0..16; known at multiples of 16 / nf, then bridged.  The
         * midpoints take the normals of the sample's own blocks from b0 on: the first block
         * after the path's own (b0 = M^l / 4 when M^l >= 4; b0 = 1 on packed levels, whose path
         * reads block 0 of another counter). */
        long b0 = nf >= 4 ? nf / 4 : 1;
        double grid[17], zb[24];
        oracle_normals(seed, level, tag, s, stream, (int)(4 * b0 + 16), zb);
        long step = 16 / nf;
        double W = 0.0;
        grid[0] = 0.0;
        for (long k = 0; k < nf; ++k) {
            W += sqrt_h * z[k];
            grid[(k + 1) * step] = W;
        }
        long next = 4 * b0;
        for (long width = step; width > 1; width /= 2) {
            double dt_half = T / 16.0 * (double)(width / 2);
            for (long left = 0; left < 16; left += width) {
                long mid = left + width / 2;
                grid[mid] = 0.5 * (grid[left] + grid[left + width]) +
                            sqrt(dt_half / 2.0) * zb[next++];
            }
        }
        for (int k = 0; k < 16; ++k)
            W16[k] = grid[k + 1];
    }
    free(z);
}

/* Y for each sample s in [first, first + N): P_l - P_{l-1} (or P_l alone at level 0 or in
 * fine-only mode). */
int oracle_level_samples(int level, int M, uint64_t N, uint64_t first, int tag, int mode,
                         const oracle_problem *p, uint64_t seed, int stream, double *Y)
{
    if (level < 0 || level > 15 || (M != 2 && M != 4 && M != 8) || !p || !Y)
        return 1;
    long nf = ipow(M, level);
    if (nf > (1L << 24))
        return 1;
    double *dW = (double *)malloc(sizeof(double) * (size_t)nf);
    double *fine = (double *)malloc(sizeof(double) * (size_t)(nf + 1));
    double *coarse = (double *)malloc(sizeof(double) * (size_t)(nf / M + 1));
    int coupled = (level > 0 && (mode == MODE_COUPLED || mode == MODE_ANTITHETIC));
    int anti = (level > 0 && mode == MODE_ANTITHETIC);
    double *dWa = anti ? (double *)malloc(sizeof(double) * (size_t)nf) : NULL;
    double *fine_a = anti ? (double *)malloc(sizeof(double) * (size_t)(nf + 1)) : NULL;
    for (uint64_t i = 0; i < N; ++i) {
        oracle_sample_paths(level, M, first + i, tag, p, seed, stream, dW, fine,
                            coupled ? coarse : NULL);
        double Pf = oracle_payoff(p->payoff, p->K, p->Q, p->r, p->T, fine, (int)nf);
        if (anti) {
            /* the antithetic fine path: each coarse step's M increments in reverse order */
            for (long c = 0; c < nf / M; ++c)
                for (int q = 0; q < M; ++q)
                    dWa[c * M + q] = dW[c * M + (M - 1 - q)];
            scheme_path(p, (int)nf, p->T / (double)nf, dWa, fine_a);
            double Pfa = oracle_payoff(p->payoff, p->K, p->Q, p->r, p->T, fine_a, (int)nf);
            Pf = 0.5 * (Pf + Pfa);
        }
        double Pc = coupled ? oracle_payoff(p->payoff, p->K, p->Q, p->r, p->T, coarse,
                                            (int)(nf / M))
                            : 0.0;
        Y[i] = Pf - Pc;
    }
    free(dW);
    free(fine);
    free(coarse);
    free(dWa);
    free(fine_a);
    return 0;
}

/* Neumaier-compensated running sum, so that the oracle's own summation error stays at a few
 * ulps of the result however many samples are added. */
typedef struct { double s, c; } csum;
static void csum_add(csum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

/*
 * sums[k] = sum over samples of Y^(k+1), k = 0..3, for samples [first, first + N) of level l;
 * cost = N * C_l.  Returns 0 on success, 1 on invalid arguments.
 */
int oracle_level_sums(int level, int M, uint64_t N, uint64_t first, int tag, int mode,
                      const oracle_problem *p, uint64_t seed, int stream, double sums[4],
                      double *cost)
{
    if (level < 0 || level > 15 || (M != 2 && M != 4 && M != 8) || !p || !sums || !cost)
        return 1;
    const uint64_t chunk = 4096;
    double *Y = (double *)malloc(sizeof(double) * chunk);
    csum acc[4] = { { 0, 0 }, { 0, 0 }, { 0, 0 }, { 0, 0 } };
    for (uint64_t done = 0; done < N; done += chunk) {
        uint64_t n = N - done < chunk ? N - done : chunk;
        if (oracle_level_samples(level, M, n, first + done, tag, mode, p, seed, stream, Y)) {
            free(Y);
            return 1;
        }
        for (uint64_t i = 0; i < n; ++i) {
            double y = Y[i];
            csum_add(&acc[0], y);
            csum_add(&acc[1], y * y);
            csum_add(&acc[2], y * y * y);
            csum_add(&acc[3], y * y * y * y);
        }
    }
    free(Y);
    for (int k = 0; k < 4; ++k)
        sums[k] = acc[k].s + acc[k].c;
    double Cl = level == 0 ? 1.0 : (double)(ipow(M, level) + ipow(M, level - 1));
    if (mode == MODE_FINE_ONLY)
        Cl = (double)ipow(M, level);
    if (mode == MODE_ANTITHETIC && level > 0)
        Cl = (double)(2 * ipow(M, level) + ipow(M, level - 1));
    *cost = (double)N * Cl;
    return 0;
}
