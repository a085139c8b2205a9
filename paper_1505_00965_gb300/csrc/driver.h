// driver.h -- the adaptive multilevel Monte Carlo algorithm on the host, FP64 (Sec. 5).
//
// Estimator P = sum_l mean(Y_l), the telescoping sum of Eq. (mlmc:ident), with Y_0 and Y_l from
// Eqs. (mlmc:Yzero) and (Yldef).  The sample counts follow from estimated variances (the
// remark "Constructive Upper Bound" of Sec. 5): minimising sum N_l C_l subject to
// sum V_l / N_l = eps^2 / 2 gives N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)).
// Levels are added until the bias estimate max(|m_L|, |m_{L-1}| / M^alpha) / (M^alpha - 1) is
// at most eps / sqrt(2), so that bias^2 + variance <= eps^2 (the mean-square error of the
// Theorem of Sec. 5).  alpha and beta are least-squares slopes of log_M |m_l| and log_M V_l
// over l = 1..L, floored at 1/2; a level is added when no level needs more than 1% more
// samples and the bias test fails, its variance extrapolated as V_{L-1} / M^beta; for l >= 2
// the means and variances used in these formulas are floored at half the extrapolation from
// the level below.
//
// The class holds no device state: callers run the rounds (draw next_samples() per level,
// starting at samples_taken() on each level so every round draws fresh samples) and pass the
// round's sums back to absorb().
#pragma once
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <vector>

#include "mlmc.h"

namespace mlmcgb {

class AdaptiveMLMC {
  public:
    AdaptiveMLMC(double eps, int M, int Lmin, int Lmax, uint64_t N0) : eps_(eps), M_(M), Lmax_(Lmax), L_(Lmin)
    {
        N_.assign(Lmin + 1, 0);
        S_.assign(Lmin + 1, {0.0, 0.0, 0.0, 0.0});
        for (int l = 0; l <= Lmin; ++l) C_.push_back(cost_of(l));
        dN_.assign(Lmin + 1, N0);
    }

    // Samples each level should draw this round (size finest_level() + 1; 0 = none).
    const std::vector<uint64_t> &next_samples() const { return dN_; }
    bool active() const
    {
        return std::any_of(dN_.begin(), dN_.end(), [](uint64_t v) { return v > 0; });
    }
    int finest_level() const { return L_; }
    uint64_t samples_taken(int l) const { return N_[l]; }
    int rounds() const { return rounds_; }

    // Add one round's sums: sums[4 l + k] = sum Y^(k+1) of the dN_l new samples of level l
    // (levels that drew nothing are ignored).  Then choose the next round.
    void absorb(const double *sums)
    {
        ++rounds_;
        for (int l = 0; l <= L_; ++l) {
            if (!dN_[l]) continue;
            for (int k = 0; k < 4; ++k) S_[l][k] += sums[4 * l + k];
            N_[l] += dN_[l];
        }
        mean_.assign(L_ + 1, 0.0);
        var_.assign(L_ + 1, 0.0);
        for (int l = 0; l <= L_; ++l) {
            mean_[l] = S_[l][0] / (double)N_[l];
            var_[l] = std::max(S_[l][1] / (double)N_[l] - mean_[l] * mean_[l], 0.0);
        }
        fit_rates();
        std::vector<double> mf, vf;
        floored(mf, vf);
        dN_ = extra_samples(vf);
        bool settled = true;
        for (int l = 0; l <= L_; ++l)
            if ((double)dN_[l] > 0.01 * (double)N_[l]) settled = false;
        if (settled && bias(mf) > eps_ / std::sqrt(2.0) && L_ < Lmax_) {
            L_ += 1;
            vf.push_back(vf.back() / std::pow((double)M_, beta_));
            N_.push_back(0);
            S_.push_back({0.0, 0.0, 0.0, 0.0});
            C_.push_back(cost_of(L_));
            dN_ = extra_samples(vf);
        }
    }

    bool converged() const
    {
        std::vector<double> mf, vf;
        floored(mf, vf);
        return bias(mf) <= eps_ / std::sqrt(2.0);
    }

    // Estimate and per-level statistics (timing and launch counters are the caller's).
    void fill(mlmc_result *out) const
    {
        out->eps = eps_;
        out->L = L_;
        out->converged = converged() ? 1 : 0;
        out->rounds = rounds_;
        double P = 0.0, total = 0.0, steps = 0.0;
        for (int l = 0; l <= L_; ++l) {
            out->N[l] = N_[l];
            for (int k = 0; k < 4; ++k) out->sums[l][k] = S_[l][k];
            out->mean[l] = mean_[l];
            out->var[l] = var_[l];
            out->cost[l] = (double)N_[l] * C_[l];
            P += mean_[l];
            total += out->cost[l];
            double nf = 1.0;
            for (int i = 0; i < l; ++i) nf *= M_;
            steps += (double)N_[l] * nf;
        }
        out->P = P;
        out->alpha = alpha_;
        out->beta = beta_;
        out->total_cost = total;
        out->path_steps = steps;
    }

    // C_l: Euler--Maruyama steps of one level-l sample, fine and coarse (Sec. 3 cost model),
    // times the level's cost scale (1 unless set_cost_scale changed it).
    double cost_of(int l) const
    {
        double nf = 1.0;
        for (int i = 0; i < l; ++i) nf *= M_;
        const double steps = l == 0 ? 1.0 : nf + nf / M_;
        return steps * (l < (int)scale_.size() ? scale_[l] : 1.0);
    }

    // Scale level l's cost, for a level estimator that does more work per sample than the
    // plain one (the control variate's network and its mean sample).
    void set_cost_scale(int l, double factor)
    {
        if (l < 0 || l >= (int)scale_.size() || !(factor > 0)) return;
        scale_[l] = factor;
        if (l < (int)C_.size()) C_[l] = cost_of(l);
    }

  private:
    static double lsq_slope(const std::vector<double> &x, const std::vector<double> &y)
    {
        const size_t n = x.size();
        double mx = 0, my = 0;
        for (size_t i = 0; i < n; ++i) {
            mx += x[i];
            my += y[i];
        }
        mx /= n;
        my /= n;
        double sxy = 0, sxx = 0;
        for (size_t i = 0; i < n; ++i) {
            sxy += (x[i] - mx) * (y[i] - my);
            sxx += (x[i] - mx) * (x[i] - mx);
        }
        return sxy / sxx;
    }

    void fit_rates()
    {
        const double tiny = 1e-300, lnM = std::log((double)M_);
        std::vector<double> ls, lm, lv;
        for (int l = 1; l <= L_; ++l) {
            ls.push_back(l);
            lm.push_back(std::log(std::max(std::fabs(mean_[l]), tiny)) / lnM);
            lv.push_back(std::log(std::max(var_[l], tiny)) / lnM);
        }
        alpha_ = std::max(0.5, -lsq_slope(ls, lm));
        beta_ = std::max(0.5, -lsq_slope(ls, lv));
    }

    void floored(std::vector<double> &mf, std::vector<double> &vf) const
    {
        mf = mean_;
        vf = var_;
        const double Ma = std::pow((double)M_, alpha_), Mb = std::pow((double)M_, beta_);
        for (size_t l = 2; l < mf.size(); ++l) {
            mf[l] = std::max(std::fabs(mf[l]), 0.5 * std::fabs(mf[l - 1]) / Ma);
            vf[l] = std::max(vf[l], 0.5 * vf[l - 1] / Mb);
        }
    }

    double bias(const std::vector<double> &mf) const
    {
        const int L = (int)mf.size() - 1;
        const double Ma = std::pow((double)M_, alpha_);
        return std::max(std::fabs(mf[L]), std::fabs(mf[L - 1]) / Ma) / (Ma - 1.0);
    }

    std::vector<uint64_t> extra_samples(const std::vector<double> &V) const
    {
        double tot = 0;
        for (size_t l = 0; l < V.size(); ++l) tot += std::sqrt(V[l] * C_[l]);
        std::vector<uint64_t> dN(V.size(), 0);
        for (size_t l = 0; l < V.size(); ++l) {
            const double n = std::ceil(2.0 / (eps_ * eps_) * std::sqrt(V[l] / C_[l]) * tot);
            const uint64_t want = n > 9.0e18 ? (uint64_t)9.0e18 : (uint64_t)n;
            const uint64_t done = l < N_.size() ? N_[l] : 0;
            dN[l] = want > done ? want - done : 0;
        }
        return dN;
    }

    double eps_;
    int M_, Lmax_, L_;
    int rounds_ = 0;
    double alpha_ = 0.5, beta_ = 0.5;
    std::vector<uint64_t> N_, dN_;
    std::vector<std::array<double, 4>> S_;
    std::vector<double> mean_, var_, C_;
    std::vector<double> scale_ = std::vector<double>(MLMC_MAX_LEVELS, 1.0);
};

}  // namespace mlmcgb
