"""The learned control variate on the GPU against the FP64 oracle (control-variate remark of
Sec. 5: estimate E[Y - g] and add E[g]).

Tolerances, from the arithmetic of the tensor-core network: operands x, W1, W2 and GELU(z1)
are bfloat16 (8 significant bits) on both sides; the GPU evaluates tanh with the hardware
approximation (relative error about 2^-11), so a bfloat16 rounding of GELU(z1) can land one
unit (2^-7 relative) away from the oracle's.  Propagated through layer 2 and the output dot
product, |g_gpu - g_oracle| <= 2^-6 sum_o |w3_o| (sum_i |W2_oi h1_i| + |b2_o|) + 1e-5 per
sample; gradients agree to 2e-2 in norm.  Path values Y use the FP32 per-sample bound of the
level parity tests.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp

from gpu_helpers import oracle_problem, run_level

pytestmark = pytest.mark.gpu

GBM = dict(S0=100.0, r=0.05, sigma=0.2, T=1.0, K=100.0, cash=1.0)


@pytest.fixture(scope="module")
def mlmc():
    from paper_1505_00965_gb300 import build

    build.build()
    from paper_1505_00965_gb300 import mlmc as binding

    return binding


def _params(seed):
    rng = np.random.default_rng(seed)
    theta = omlp.init_params(seed)
    W1, b1, W2, b2, w3, b3 = omlp.unpack(theta)
    theta = omlp.pack(W1, 0.3 * rng.standard_normal(64), W2, 0.3 * rng.standard_normal(64), w3, 0.2)
    return theta.astype(np.float32)


def _g_bound(theta32, X):
    """Per-sample bound on |g_gpu - g_oracle| (module docstring)."""
    theta = theta32.astype(np.float64)
    _, (_, _, h1, _, _) = omlp.forward(theta, X, quantize=True)
    _, _, W2, b2, w3, _ = omlp.unpack(theta)
    W2b = omlp.bf16(W2)
    inner = np.abs(h1) @ np.abs(W2b).T + np.abs(b2)
    return 2.0 ** -6 * (inner @ np.abs(w3)) + 1e-5


def _y_bound(level, M):
    n = M ** level
    return 8.0 * (2.0 ** -24 * math.sqrt(n + 1) + 2e-6) * 100.0 * math.exp(0.05)


def test_mlp_forward_matches_oracle(mlmc):
    import torch

    rng = np.random.default_rng(1)
    X = rng.standard_normal((4096 + 17, omlp.D)).astype(np.float32)
    theta = _params(3)
    d_X = torch.tensor(X, device="cuda")
    d_G = torch.zeros(len(X), dtype=torch.float32, device="cuda")
    mlmc.mlmc_mlp_forward(theta, d_X, len(X), d_G)
    g = d_G.cpu().numpy().astype(np.float64)
    want, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64), quantize=True)
    assert np.all(np.abs(g - want) <= _g_bound(theta, X.astype(np.float64)))
    assert np.corrcoef(g, want)[0, 1] > 0.99999


@pytest.mark.parametrize("B", [2048, 32, 96, 65536])
def test_mlp_grad_matches_oracle(mlmc, B):
    """The project's forward and backward kernels (one step of the training kernel without the
    update) against the oracle's chain rule.  B = 32 runs on a cluster of 2 CTAs with one tile
    each, 96 on a cluster of 2 with idle tiles, 2048 on 16 CTAs of 8 tiles, 65536 on 16 CTAs of
    16 chunks of 256 rows."""
    import torch

    rng = np.random.default_rng(2)
    X = rng.standard_normal((B, omlp.D)).astype(np.float32)
    Y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.1 * rng.standard_normal(B)).astype(np.float32)
    theta = _params(4)
    loss, grad = mlmc.mlmc_mlp_grad(theta, torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), B)
    want_loss, want = omlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                                         quantize=True)
    assert abs(loss - want_loss) <= 1e-2 * want_loss
    grad = grad.astype(np.float64)
    assert np.linalg.norm(grad - want) <= 2e-2 * np.linalg.norm(want)
    # every parameter block separately
    nw1 = 64 * omlp.D
    bounds = [0, nw1, nw1 + 64, nw1 + 64 + 4096, nw1 + 128 + 4096, nw1 + 192 + 4096, omlp.N_PARAMS]
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert np.linalg.norm(grad[a:b] - want[a:b]) <= 5e-2 * np.linalg.norm(want[a:b]) + 1e-7, (a, b)


@pytest.mark.parametrize("M,level", [(4, 0), (4, 1), (4, 2), (4, 3), (2, 1), (2, 2), (2, 3), (2, 4), (8, 0), (8, 1)])
def test_training_data_matches_oracle(mlmc, M, level):
    """(x, Y) pairs under the training tag: inputs from the Brownian grid (bridged below sixteen
    fine steps, from the first Philox block the path does not read: block 1 on levels of 1, 2 and 4
    steps, block 2 on levels of 8), Y = P_l - P_{l-1} on the same path."""
    import torch

    p = mlmc.Problem(payoff="asian", **GBM)
    cv = mlmc.mlmc_cv_create(M, p)
    N, first = 600, 5
    d_X = torch.zeros((N, omlp.D), dtype=torch.float32, device="cuda")
    d_Y = torch.zeros(N, dtype=torch.float32, device="cuda")
    mlmc.mlmc_cv_training_data(cv, level, N, first, 9, d_X, d_Y)
    X, Y = d_X.cpu().numpy().astype(np.float64), d_Y.cpu().numpy().astype(np.float64)
    op = oracle_problem(oracle, p)
    Yo = oracle.level_samples(level, M, N, op, seed=9, first=first, stream="fp32", tag=oracle.TAG_CV_TRAIN)
    Xo = np.array([omlp.features(level, M, first + i, 1.0, seed=9, stream="fp32", tag=oracle.TAG_CV_TRAIN)
                   for i in range(N)])
    assert np.max(np.abs(Y - Yo)) <= _y_bound(level, M)
    assert np.max(np.abs(X - Xo)) <= 1e-4


@pytest.mark.parametrize("M,level", [(4, 0), (4, 1), (4, 2), (4, 3), (2, 2), (8, 1)])
def test_cv_level_and_mean_sums_match_oracle(mlmc, M, level):
    """Levels 0-2 at M = 4 run kernels compiled for their M^l; level 3 and the other M the kernel
    with a run-time M^l."""
    import torch

    p = mlmc.Problem(payoff="asian", **GBM)
    op = oracle_problem(oracle, p)
    cv = mlmc.mlmc_cv_create(M, p)
    theta = _params(10 + level)
    mlmc.mlmc_cv_set_params(cv, level, theta, kappa=2.0)
    N, first, seed = 2048 + 33, 101, 12
    d_s = torch.zeros(8, dtype=torch.float64, device="cuda")
    d_r = torch.zeros(N, dtype=torch.float32, device="cuda")
    d_g = torch.zeros(N, dtype=torch.float32, device="cuda")
    mlmc.mlmc_cv_level_sums(cv, level, N, first, seed, d_s, d_r, d_g)
    r, g = d_r.cpu().numpy().astype(np.float64), d_g.cpu().numpy().astype(np.float64)
    Yo = oracle.level_samples(level, M, N, op, seed=seed, first=first, stream="fp32")
    Xo = np.array([omlp.features(level, M, first + i, 1.0, seed=seed, stream="fp32") for i in range(N)])
    go, _ = omlp.forward(theta.astype(np.float64), Xo, quantize=True)
    assert np.all(np.abs(g - go) <= _g_bound(theta, Xo))
    assert np.max(np.abs((r + g) - Yo)) <= _y_bound(level, M) + 1e-5 * np.max(np.abs(Yo))
    # the eight sums against the device's own per-sample values
    Yg = r + g
    own = [r.sum(), (r ** 2).sum(), (r ** 3).sum(), (r ** 4).sum(), Yg.sum(), (Yg ** 2).sum(), g.sum(), (g ** 2).sum()]
    sums = d_s.cpu().numpy()
    scales = [np.abs(r).sum(), (r ** 2).sum(), (np.abs(r) ** 3).sum(), (r ** 4).sum(), np.abs(Yg).sum(),
              (Yg ** 2).sum(), np.abs(g).sum(), (g ** 2).sum()]
    for k in range(8):
        assert abs(sums[k] - own[k]) <= 1e-6 * scales[k] + 1e-9, k
    # the independent mean sample: replicates 3 and 4 of the shifted lattice, every point
    R, n = 2, omlp.LATTICE_N
    d_m = torch.zeros(2, dtype=torch.float64, device="cuda")
    d_gm = torch.zeros(R * n, dtype=torch.float32, device="cuda")
    mlmc.mlmc_cv_mean_sums(cv, level, R, 3, seed, d_m, d_gm)
    gm = d_gm.cpu().numpy().astype(np.float64).reshape(R, n)
    for j in range(R):
        Xm = omlp.mean_sample_features(3 + j, np.arange(n), seed, level)
        gmo, _ = omlp.forward(theta.astype(np.float64), Xm, quantize=True)
        assert np.all(np.abs(gm[j] - gmo) <= _g_bound(theta, Xm)), j
    Q = gm.mean(axis=1)
    np.testing.assert_allclose(d_m.cpu().numpy(), [Q.sum(), (Q ** 2).sum()], rtol=1e-9)


def test_cv_level_sums_with_many_tiles_per_block(mlmc):
    """N = 2^21 + 77 on level 1: each block of the tensor-core level kernel runs several batches
    of tiles (folds of FP32 batch sums into FP64) and the last tile is ragged.  The eight sums
    match the device's own per-sample values; g and Y of samples at the start, the middle and
    the end match the oracle."""
    import torch

    p = mlmc.Problem(payoff="asian", **GBM)
    op = oracle_problem(oracle, p)
    cv = mlmc.mlmc_cv_create(4, p)
    theta = _params(31)
    level = 1
    mlmc.mlmc_cv_set_params(cv, level, theta, kappa=2.0)
    N, first, seed = (1 << 21) + 77, 5, 19
    d_s = torch.zeros(8, dtype=torch.float64, device="cuda")
    d_r = torch.zeros(N, dtype=torch.float32, device="cuda")
    d_g = torch.zeros(N, dtype=torch.float32, device="cuda")
    mlmc.mlmc_cv_level_sums(cv, level, N, first, seed, d_s, d_r, d_g)
    r, g = d_r.cpu().numpy().astype(np.float64), d_g.cpu().numpy().astype(np.float64)
    Yg = r + g
    own = [r.sum(), (r ** 2).sum(), (r ** 3).sum(), (r ** 4).sum(), Yg.sum(), (Yg ** 2).sum(), g.sum(), (g ** 2).sum()]
    scales = [np.abs(r).sum(), (r ** 2).sum(), (np.abs(r) ** 3).sum(), (r ** 4).sum(), np.abs(Yg).sum(),
              (Yg ** 2).sum(), np.abs(g).sum(), (g ** 2).sum()]
    sums = d_s.cpu().numpy()
    for k in range(8):
        assert abs(sums[k] - own[k]) <= 1e-6 * scales[k] + 1e-9, k
    idx = np.concatenate([np.arange(40), N // 2 + np.arange(40), N - 40 + np.arange(40)])
    Yo = np.array([oracle.level_samples(level, 4, 1, op, seed=seed, first=first + int(i), stream="fp32")[0] for i in idx])
    Xo = np.array([omlp.features(level, 4, first + int(i), 1.0, seed=seed, stream="fp32") for i in idx])
    go, _ = omlp.forward(theta.astype(np.float64), Xo, quantize=True)
    assert np.all(np.abs(g[idx] - go) <= _g_bound(theta, Xo))
    assert np.max(np.abs(Yg[idx] - Yo)) <= _y_bound(level, 4) + 1e-5 * np.max(np.abs(Yo))


def test_zero_network_reduces_to_plain(mlmc):
    """g = 0 (all parameters zero): r is the plain sample Y, sample for sample."""
    import torch

    p = mlmc.Problem(payoff="lookback", **GBM)
    cv = mlmc.mlmc_cv_create(4, p)
    mlmc.mlmc_cv_set_params(cv, 2, np.zeros(mlmc.MLMC_CV_PARAMS, dtype=np.float32))
    N = 3000
    d_s = torch.zeros(8, dtype=torch.float64, device="cuda")
    d_r = torch.zeros(N, dtype=torch.float32, device="cuda")
    d_g = torch.zeros(N, dtype=torch.float32, device="cuda")
    mlmc.mlmc_cv_level_sums(cv, 2, N, 0, 4, d_s, d_r, d_g)
    assert float(d_g.abs().max()) == 0.0
    _, y = run_level(mlmc, 2, 4, N, 0, p, 4, "fp32", launch={"lanes_per_path": 1})
    assert np.max(np.abs(d_r.cpu().numpy() - y)) <= _y_bound(2, 4)


def test_training_gains_and_estimates_stay_unbiased(mlmc):
    """Trained on the method's own samples, the network removes most of the variance on the
    coarse levels of the arithmetic-Asian call (held-out data), and the control-variate
    estimates agree with the plain ones (both unbiased, RMSE <= eps)."""
    p = mlmc.Problem(payoff="asian", **GBM)
    cv = mlmc.mlmc_cv_train(4, p, seed=77, levels=3, epochs=10, n_train=200_000, batch=4096, init_seed=1)
    info = [mlmc.mlmc_cv_info(cv, l) for l in range(3)]
    assert all(i["trained"] for i in info)
    assert info[0]["var_resid"] < 0.05 * info[0]["var_plain"]
    assert info[1]["var_resid"] < 0.5 * info[1]["var_plain"]
    assert all(i["t_cv"] > 0 and i["t_mean"] > 0 and i["t_plain"] > 0 for i in info)
    # the shifted lattice estimates E[g] with far less variance per point than plain sampling
    assert info[0]["var_lattice"] < info[0]["var_g"] / 20
    assert info[1]["var_lattice"] < info[1]["var_g"] / 20
    eps = 2e-3
    for seed in (1, 2, 3):
        a = mlmc.mlmc_estimate_cv(eps, cv, seed)
        b = mlmc.mlmc_estimate(eps, p, seed)
        assert a.converged and abs(a.P - b.P) < 3 * math.sqrt(2) * eps, (a.P, b.P)


def test_training_repeats_bit_for_bit_and_reports_its_phases(mlmc):
    """The training launch reduces every gradient in a fixed order (rank-ordered partials over
    distributed shared memory), so two trainings with the same seeds give identical networks;
    mlmc_cv_train_info accounts for the call's time."""
    p = mlmc.Problem(payoff="asian", **GBM)
    kw = dict(seed=31, levels=2, epochs=3, n_train=100_000, batch=4096, init_seed=2)
    a = mlmc.mlmc_cv_train(4, p, **kw)
    b = mlmc.mlmc_cv_train(4, p, **kw)
    for level in range(2):
        np.testing.assert_array_equal(mlmc.mlmc_cv_get_params(a, level), mlmc.mlmc_cv_get_params(b, level))
    info = mlmc.mlmc_cv_train_info(a)
    assert info["levels"] == 2 and info["cluster"] in (8, 16)
    assert info["steps"] == 3 * (90_000 // 4096)
    assert 0 < info["train_kernel_ms"] <= info["train_ms"] * 1.05 + 0.1
    assert info["total_ms"] >= info["data_ms"] + info["train_ms"] + info["eval_ms"] + info["cost_ms"] - 1.0
    c = mlmc.mlmc_cv_create(4, p)
    assert mlmc.mlmc_cv_train_info(c)["steps"] == 0
