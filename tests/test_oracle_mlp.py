"""Pins of the oracle's control-variate network: gradients against finite differences, the GELU
against the exact x Phi(x), bfloat16 rounding against PyTorch's conversion, closed-form special
cases, and the law of the network inputs."""
import math

import numpy as np
import pytest
from scipy.stats import norm

import oracle
from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + 0.1 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((40, mlp.D))
    Y = rng.standard_normal(40) * 2 + 1
    loss, grad = mlp.loss_and_grad(theta, X, Y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False).tolist() + [mlp.N_PARAMS - 1, 0, 64 * mlp.D, mlp.N_PARAMS - 65]
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        lp, _ = mlp.loss_and_grad(theta + e, X, Y)
        lm, _ = mlp.loss_and_grad(theta - e, X, Y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_gelu_is_close_to_x_phi_x_and_its_derivative_is_exact():
    z = np.linspace(-6, 6, 2001)
    assert np.max(np.abs(mlp.gelu(z) - z * norm.cdf(z))) < 1e-3
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_bf16_rounding_matches_pytorch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(5000) * 10 ** rng.uniform(-3, 3, 5000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 65504.0, 1e-30]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)
    assert mlp.bf16(np.array([1 + 2 ** -8]))[0] == 1.0               # tie to even
    assert mlp.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6   # tie to even, upwards


def test_network_special_cases():
    """With W1 = 0 and b1 = 0 the first layer outputs GELU(0) = 0, so g = w3 . GELU(b2) + b3."""
    rng = np.random.default_rng(2)
    b2 = rng.standard_normal(64)
    w3 = rng.standard_normal(64)
    theta = mlp.pack(np.zeros((64, mlp.D)), np.zeros(64), rng.standard_normal((64, 64)), b2, w3, 0.7)
    X = rng.standard_normal((10, mlp.D))
    g, _ = mlp.forward(theta, X)
    want = float(w3 @ (0.5 * b2 * (1 + np.tanh(math.sqrt(2 / math.pi) * (b2 + 0.044715 * b2 ** 3))))) + 0.7
    np.testing.assert_allclose(g, want, rtol=1e-14)
    # a network that is linear in x for small weights: g ~ b3 + w3 . GELU'(0) W2 GELU'(0) W1 x
    # (GELU(z) = z / 2 + O(z^2): with |W1 x| ~ 1e-7 the quadratic terms are ~1e-7 relative)
    small = mlp.pack(rng.standard_normal((64, mlp.D)) * 1e-7, np.zeros(64), rng.standard_normal((64, 64)) * 1e-2,
                     np.zeros(64), rng.standard_normal(64), 0.0)
    W1, _, W2, _, w3s, _ = mlp.unpack(small)
    lin = X @ (0.25 * (w3s @ W2 @ W1))
    g, _ = mlp.forward(small, X)
    np.testing.assert_allclose(g, lin, rtol=1e-4, atol=1e-15)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_features_are_iid_standard_normal(level):
    """Levels 0 and 1 refine their grid by Brownian-bridge midpoints, level 2 (16 steps) is the
    fine path itself, level 3 sums four fine increments per feature."""
    n = 20000
    F = np.array([mlp.features(level, 4, s, 1.0, seed=17) for s in range(n)])
    assert np.max(np.abs(F.mean(axis=0))) < 5 / math.sqrt(n)
    assert F.shape == (n, 16)
    assert np.max(np.abs(np.cov(F.T, bias=True) - np.eye(16))) < 5 * math.sqrt(2 / n)


@pytest.mark.parametrize("M,level", [(4, 0), (4, 1), (2, 3)])
def test_features_of_bridged_levels_are_the_path_and_bridge_normals(M, level):
    """On a level whose grid is refined by Brownian-bridge midpoints the Levy coordinates give
    back the construction's own normals: x_0 = W(T) / sqrt(T) (the path's), and the midpoints the
    bridge added (the stages finer than the path's grid), stage by stage and left to right, are
    the bridge normals in the order they were drawn, from the first Philox block the path does not
    read."""
    nf = M ** level
    b0 = max(1, nf // 4)
    for s in range(3):
        x = mlp.features(level, M, s, 1.0, seed=21)
        W = oracle.grid_brownian(level, M, s, 1.0, seed=21)
        assert x[0] == W[-1]
        zb = oracle.normals(21, level, s, 4 * b0 + 16)[4 * b0:]
        k, idx, width = 0, 1, 16
        while width > 1:
            for _ in range(0, 16, width):
                if width <= 16 // nf:
                    assert x[idx] == pytest.approx(zb[k], rel=1e-9, abs=1e-9), (s, idx)
                    k += 1
                idx += 1
            width //= 2
        assert k == 16 - nf


def test_levy_coordinates_invert_to_the_grid():
    """The Levy coordinates are an orthogonal change of the standardised increments: the grid is
    rebuilt from them by the bridge construction, and the sum of squares is kept."""
    rng = np.random.default_rng(8)
    T = 1.3
    W = np.cumsum(rng.standard_normal(16) * math.sqrt(T / 16))
    x = mlp.levy_coordinates(W, T)
    inc = np.diff(np.concatenate([[0.0], W])) / math.sqrt(T / 16)
    assert np.sum(x ** 2) == pytest.approx(np.sum(inc ** 2), rel=1e-12)
    grid = np.zeros(17)
    grid[16] = x[0] * math.sqrt(T)
    idx, width = 1, 16
    while width > 1:
        for left in range(0, 16, width):
            grid[left + width // 2] = 0.5 * (grid[left] + grid[left + width]) + math.sqrt(T / 16 * width / 4) * x[idx]
            idx += 1
        width //= 2
    np.testing.assert_allclose(grid[1:], W, rtol=1e-12, atol=1e-12)


def _lattice_offsets(r, seed, level):
    """K_k(i) = i z_k mod n recovered from the oracle's 32-bit points v = K 2^16 + D mod 2^32."""
    i = np.arange(mlp.LATTICE_N)
    v = mlp.lattice_points32(r, i, seed, level)
    D = np.array(mlp.lattice_shift(r, seed, level), dtype=np.int64)
    K = (v - D[None, :]) % (1 << 32)
    assert np.all(K % 65536 == 0)
    return K // 65536


def test_tent_transform_is_two_to_one_onto_even_fractions():
    """The tent transform of the 32-bit fractions: u -> 1 - |2u - 1| up to one unit, image the
    even fractions, each hit twice (so uniform input gives uniform top-23-bit cells), and the
    uniforms used are the centred cells of the transformed points."""
    rng = np.random.default_rng(4)
    v = rng.integers(0, 2 ** 32, 200_000, dtype=np.int64)
    w = mlp.tent32(v)
    assert np.all(w % 2 == 0) and np.all((w >= 0) & (w <= 2 ** 32 - 2))
    u = v / 2.0 ** 32
    assert np.max(np.abs(w / 2.0 ** 32 - (1 - np.abs(2 * u - 1)))) <= 2.0 ** -31
    edges = np.array([0, 1, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1], dtype=np.int64)
    assert mlp.tent32(edges).tolist() == [0, 2, 2 ** 32 - 2, 2 ** 32 - 2, 2, 0]
    # exhaustive on a 12-bit analogue of the map: two to one onto the even values
    small = np.arange(4096)
    img = np.where(small < 2048, 2 * small, 2 * (4095 - small))
    assert np.array_equal(np.bincount(img, minlength=4096)[::2], np.full(2048, 2))
    uu = mlp.lattice_uniforms(3, np.arange(50), seed=1, level=0)
    ww = mlp.tent32(mlp.lattice_points32(3, np.arange(50), seed=1, level=0))
    assert np.array_equal(uu, ((ww >> 9) + 0.5) * 2.0 ** -23)


def test_lattice_is_the_korobov_rank1_lattice():
    """Before the tent transform and with the random shift removed the points are i z / n for the
    Korobov vector z = (1, a, a^2, ...) mod n: coordinate 0 is i / n, the map i -> point is
    additive mod n (a rank-1 lattice is a group), and every coordinate runs through all n strata
    once."""
    n = mlp.LATTICE_N
    K = _lattice_offsets(5, seed=17, level=2)
    assert np.array_equal(K[:, 0], np.arange(n))
    assert K[1, 1] == mlp.LATTICE_A
    for k in range(mlp.D):
        assert np.array_equal(np.sort(K[:, k]), np.arange(n)), k
    rng = np.random.default_rng(0)
    a, b = rng.integers(0, n, 500), rng.integers(0, n, 500)
    assert np.array_equal((K[a] + K[b]) % n, K[(a + b) % n])


def test_lattice_mean_is_unbiased_with_small_variance():
    """E[exp(c . x)] = exp(|c|^2 / 2) for x ~ N(0, I_16): the replicate means of the shifted lattice
    scatter around it (independent shifts, unbiased) with a variance far below that of plain
    sampling with as many points, (exp(2|c|^2) - exp(|c|^2)) / n."""
    c = np.array([0.3, 0.25, 0.2, 0.15, 0.1, 0.08, 0.05, 0.02, 0.02, 0.015, 0.01, 0.01, 0.005, 0.005, 0.002, 0.002])
    exact = math.exp(c @ c / 2)
    var_f = math.exp(2 * (c @ c)) - math.exp(c @ c)
    i = np.arange(mlp.LATTICE_N)
    Q = np.array([np.exp(mlp.mean_sample_features(r, i, seed=3, level=1) @ c).mean() for r in range(16)])
    se = Q.std(ddof=1) / math.sqrt(len(Q))
    assert se > 0
    assert abs(Q.mean() - exact) < 5 * se
    assert Q.var(ddof=1) < var_f / mlp.LATTICE_N / 100


def test_lattice_shifts_differ_between_replicates_levels_and_seeds():
    s = mlp.lattice_shift(0, seed=1, level=0)
    assert len(s) == 16 and all(0 <= w < 2 ** 32 for w in s)
    assert s != mlp.lattice_shift(1, seed=1, level=0)
    assert s != mlp.lattice_shift(0, seed=1, level=1)
    assert s != mlp.lattice_shift(0, seed=2, level=0)


def test_quantised_gradient_uses_the_rounded_forward():
    """With bf16 rounding on, the gradient is that of the rounded network with straight-through
    rounding of the weights: finite differences of the rounded forward in directions that do
    not cross a rounding boundary (b2, b3, w3, b1 are not rounded) agree."""
    rng = np.random.default_rng(9)
    theta = mlp.init_params(3)
    X = rng.standard_normal((30, mlp.D))
    Y = rng.standard_normal(30)
    _, grad = mlp.loss_and_grad(theta, X, Y, quantize=True)
    off_b1 = 64 * mlp.D
    off_b2 = off_b1 + 64 + 64 * 64
    for i in [off_b1 + 3, off_b2 + 5, off_b2 + 64 + 7, mlp.N_PARAMS - 1]:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = 1e-6
        lp, _ = mlp.loss_and_grad(theta + e, X, Y, quantize=True)
        lm, _ = mlp.loss_and_grad(theta - e, X, Y, quantize=True)
        fd = (lp - lm) / 2e-6
        # b1 moves z1, whose GELU is rounded to bf16 before layer 2: allow the rounding step
        tol = 2e-2 if i == off_b1 + 3 else 1e-6
        assert abs(fd - grad[i]) <= tol * max(1.0, abs(fd)), (i, fd, grad[i])
