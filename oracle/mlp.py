"""FP64 oracle of the learned control variate (TEST INFRASTRUCTURE ONLY).

A control variate replaces E[Y] by E[Y - g] + E[g] (the control-variate remark of Sec. 5:
compute E[X - Y] and add E[Y]).  Here g is a small network of the sample's Brownian path:

* inputs: the Brownian-bridge (Levy) coordinates of the path on the T/16 grid, iid N(0, 1)
  whatever the level: x_0 = W(T) / sqrt(T), then stage by stage (intervals of 16, 8, 4, 2 grid
  steps) and left to right the standardised midpoint deviations
  (W(m) - (W(l) + W(r)) / 2) / sqrt((r - l) / 4), m the midpoint of [l, r] (the construction of
  Caflisch, Morokoff and Owen, J. Comput. Finance 1, 1997, which puts the directions a path
  functional depends on most first: it suits the lattice rule below, whose weights decay along
  the coordinates);
* g(x) = w3 . GELU(W2 GELU(W1 x + b1) + b2) + b3, widths 16 -> 64 -> 64 -> 1, with
  GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
* parameters packed as W1 [64][16] (row = output unit), b1 [64], W2 [64][64], b2 [64],
  w3 [64], b3 [1]: 5313 numbers;
* training loss: the mean of (g(x) - Y)^2 over a batch.

`quantize=True` rounds to bfloat16 (round to nearest, ties to even) the operands of the
tensor-core products the GPU path uses: x, W1, W2 and the layer-2 input GELU(z1).  All other
arithmetic here is FP64.
"""
from __future__ import annotations

import math

import numpy as np

from scipy.special import ndtri

from . import TAG_CV_MEAN, grid_brownian, philox

H = 64
D = 16
N_PARAMS = H * D + H + H * H + H + H + 1
SQRT_2_OVER_PI = math.sqrt(2.0 / math.pi)
GELU_C = 0.044715


def unpack(theta: np.ndarray):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    o = 0
    W1 = theta[o:o + H * D].reshape(H, D); o += H * D
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as FP64 values."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(SQRT_2_OVER_PI * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    t = np.tanh(SQRT_2_OVER_PI * (z + GELU_C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * SQRT_2_OVER_PI * (1.0 + 3.0 * GELU_C * z * z)


def forward(theta, X, quantize: bool = False):
    """g(x) for the rows of X [B, 16], and the layer values (z1, h1, z2, h2)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    if quantize:
        X, W1, W2 = bf16(X), bf16(W1), bf16(W2)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    h1_in = bf16(h1) if quantize else h1
    z2 = h1_in @ W2.T + b2
    h2 = gelu(z2)
    g = h2 @ w3 + b3
    return g, (X, z1, h1_in, z2, h2)


def loss_and_grad(theta, X, Y, quantize: bool = False):
    """Mean squared error of g against Y and its gradient with respect to theta (chain rule)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    if quantize:
        W2 = bf16(W2)
    g, (Xq, z1, h1, z2, h2) = forward(theta, X, quantize)
    B = len(Y)
    r = g - np.asarray(Y, dtype=np.float64)
    loss = float(np.mean(r * r))
    d = 2.0 * r / B                       # dL/dg
    db3 = d.sum()
    dw3 = h2.T @ d
    dz2 = np.outer(d, w3) * gelu_grad(z2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    dW1 = dz1.T @ Xq
    db1 = dz1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters: weights uniform in +-1/sqrt(fan-in), biases zero."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (H, D)) / math.sqrt(D)
    W2 = rng.uniform(-1, 1, (H, H)) / math.sqrt(H)
    w3 = rng.uniform(-1, 1, H) / math.sqrt(H)
    return pack(W1, np.zeros(H), W2, np.zeros(H), w3, 0.0)


def levy_coordinates(W, T: float) -> np.ndarray:
    """The Brownian-bridge coordinates of grid values W = (W(T/16), ..., W(T)) (module docstring)."""
    grid = np.concatenate([[0.0], np.asarray(W, dtype=np.float64)])
    x = [grid[D] / math.sqrt(T)]
    width = D
    while width > 1:
        sd = math.sqrt(T / D * width / 4.0)
        for left in range(0, D, width):
            x.append((grid[left + width // 2] - 0.5 * (grid[left] + grid[left + width])) / sd)
        width //= 2
    return np.array(x)


def features(level: int, M: int, s: int, T: float, seed: int, stream: str = "fp64", tag: int = 0) -> np.ndarray:
    """The 16 network inputs of sample s: the Levy coordinates of its T/16 Brownian grid."""
    return levy_coordinates(grid_brownian(level, M, s, T, seed, stream=stream, tag=tag), T)


# The independent sample that estimates E[g] is a randomly shifted rank-1 lattice rule
# (Sloan and Joe, "Lattice Methods for Multiple Integration", 1994; random shifts after
# Cranley and Patterson, SIAM J. Numer. Anal. 13, 1976): replicate r is the point set
# {frac(i z / n + Delta_r) : i = 0 .. n - 1} with the Korobov generating vector
# z = (1, a, a^2, ..., a^15) mod n, mapped to N(0, I_16) coordinate by coordinate with the inverse
# normal distribution function, after the baker's (tent) transform u -> 1 - |2u - 1| of every
# coordinate (Hickernell, "Obtaining O(N^-2+eps) convergence for lattice quadrature rules",
# 2002), which suits integrands that are not periodic.  Each point of a replicate is uniform on
# [0, 1)^16 whatever Delta_r, and the tent transform keeps it uniform, so the replicate's mean of
# g is an unbiased estimate of E[g]; replicates with independent shifts are independent.  The
# library fixes n, a and the shift bits:
LATTICE_N = 65536
LATTICE_A = 43833


def lattice_generator() -> list[int]:
    """z_k = a^k mod n, k = 0..15."""
    return [pow(LATTICE_A, k, LATTICE_N) for k in range(D)]


def lattice_shift(r: int, seed: int, level: int) -> list[int]:
    """The shift of replicate r as sixteen 32-bit fractions: the words of Philox blocks 0..3 of
    counter r under the control-variate-mean tag."""
    words = []
    for j in range(D // 4):
        words += list(philox((j, r & 0xFFFFFFFF, r >> 32, (TAG_CV_MEAN << 16) | level),
                             (seed & 0xFFFFFFFF, seed >> 32)))
    return words


def lattice_points32(r: int, i, seed: int, level: int) -> np.ndarray:
    """Points i (array) of replicate r as 32-bit fractions: v = (i z_k mod n) 2^16 + D_k mod 2^32,
    which is frac(i z_k / n + D_k 2^-32) exactly."""
    i = np.atleast_1d(np.asarray(i, dtype=np.int64))
    z = np.array(lattice_generator(), dtype=np.int64)
    shift = np.array(lattice_shift(r, seed, level), dtype=np.int64)
    return (((i[:, None] * z[None, :]) % LATTICE_N) * 65536 + shift[None, :]) % (1 << 32)


def tent32(v: np.ndarray) -> np.ndarray:
    """The baker's (tent) transform u -> 1 - |2u - 1| on 32-bit fractions: 2v below one half,
    2 (2^32 - 1 - v) above.  It maps the 2^32 fractions two to one onto the even ones, so a
    uniform v gives a uniform top-23-bit cell."""
    v = np.asarray(v, dtype=np.int64)
    return np.where(v < (1 << 31), 2 * v, 2 * ((1 << 32) - 1 - v))


def lattice_uniforms(r: int, i, seed: int, level: int) -> np.ndarray:
    """Points i (array) of replicate r in (0, 1)^16: the tent transform of the shifted lattice point,
    keeping its top 23 bits, centred: u = (floor(tent(v) / 2^9) + 1/2) 2^-23."""
    v = tent32(lattice_points32(r, i, seed, level))
    return ((v >> 9).astype(np.float64) + 0.5) * 2.0 ** -23


def mean_sample_features(r: int, i, seed: int, level: int) -> np.ndarray:
    """Network inputs of points i of replicate r: x_k = Phi^{-1}(u_k), shape (len(i), 16)."""
    return ndtri(lattice_uniforms(r, i, seed, level))


def lattice_replicate_means(theta: np.ndarray, replicates, seed: int, level: int,
                            quantize: bool = False) -> np.ndarray:
    """Q_r = (1/n) sum_i g(x_ri): each replicate's lattice mean of the network."""
    i = np.arange(LATTICE_N)
    return np.array([forward(theta, mean_sample_features(r, i, seed, level), quantize=quantize)[0].mean()
                     for r in replicates])
