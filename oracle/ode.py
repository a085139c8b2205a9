"""FP64 oracle of the non-globally-Lipschitz test problem of Sec. 5 (TEST INFRASTRUCTURE ONLY).

Sec. 5 (Eq. count) cites the counterexample of Hutzenthaler, Jentzen and Kloeden: the random ODE

    dX = -X^5 dt,  X(0) ~ N(0, 1),  quantity E[X(T)^2],

for which multilevel Monte Carlo with the explicit Euler--Maruyama step diverges, while a
tamed step recovers convergence.  With f(x) = -x^5 and step h the two schemes are

    explicit Euler--Maruyama (Eq. em, g = 0):  X <- X + h f(X)
    tamed Euler--Maruyama:                     X <- X + h f(X) / (1 + h |f(X)|)

The fine path takes M^l steps of h = T / M^l, the coarse path M^(l-1) steps of M h, both from the
same X(0) (the coupling of Sec. 5: one random input, two grids); Y = X_f(T)^2 - X_c(T)^2, and
Y = X_f(T)^2 on level 0 (Eq. mlmc:Yzero).  The exact solution is X(t) = X0 (1 + 4 t X0^4)^(-1/4)
(separate variables: d(X^-4)/dt = 4), so E[X(T)^2] = E[X0^2 (1 + 4 T X0^4)^(-1/2)].

Random input: X(0) of sample s is normal (s mod 4) of Philox block 0 of counter index floor(s/4)
under the level's counter word (the library's stream definition for this model).  The paper
fixes no horizon; T is a parameter (the tests use T = 1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

from . import TAG_PATHS, normals

SCHEMES = ("em", "tamed")


def initial_values(level: int, first: int, N: int, seed: int, stream: str = "fp64", tag: int = TAG_PATHS):
    """X(0) of samples [first, first + N) (any 64-bit sample indices)."""
    out = np.empty(N, dtype=np.float64)
    q0, q1 = first // 4, (first + N - 1) // 4
    for q in range(q0, q1 + 1):
        z = normals(seed, level, q, 4, stream=stream, tag=tag)
        # samples 4q .. 4q + 3 that lie in the range, as offsets i = s - first
        lo, hi = max(4 * q, first), min(4 * q + 4, first + N)
        for s in range(lo, hi):
            out[s - first] = z[s - 4 * q]
    return out


def step(x: np.ndarray, h: float, scheme: str) -> np.ndarray:
    """One step of the scheme on f(x) = -x^5 (elementwise)."""
    x2 = x * x
    f = -(x2 * x2) * x
    if scheme == "em":
        return x + h * f
    if scheme == "tamed":
        return x + h * f / (1.0 + h * np.abs(f))
    raise ValueError(scheme)


def path_end(x0: np.ndarray, h: float, n: int, scheme: str) -> np.ndarray:
    """X after n steps of h from x0 (IEEE overflow gives inf / nan as in any FP64 program)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    with np.errstate(over="ignore", invalid="ignore"):
        for _ in range(n):
            x = step(x, h, scheme)
    return x


def level_samples(level: int, M: int, N: int, T: float, seed: int, scheme: str, first: int = 0,
                  stream: str = "fp64", fine_only: bool = False) -> np.ndarray:
    """Y of samples [first, first + N) of level `level`."""
    x0 = initial_values(level, first, N, seed, stream)
    nf = M ** level
    xf = path_end(x0, T / nf, nf, scheme)
    with np.errstate(over="ignore", invalid="ignore"):
        Pf = xf * xf
        if level == 0 or fine_only:
            return Pf
        xc = path_end(x0, M * T / nf, nf // M, scheme)
        return Pf - xc * xc


def level_sums(level: int, M: int, N: int, T: float, seed: int, scheme: str, first: int = 0,
               stream: str = "fp64", fine_only: bool = False) -> np.ndarray:
    """sum Y^k, k = 1..4 (math.fsum: exactly rounded sums)."""
    Y = level_samples(level, M, N, T, seed, scheme, first, stream, fine_only)
    with np.errstate(over="ignore", invalid="ignore"):
        return np.array([math.fsum(Y ** k) for k in range(1, 5)])


def exact_solution(x0, t: float):
    return np.asarray(x0, dtype=np.float64) * (1.0 + 4.0 * t * np.asarray(x0, dtype=np.float64) ** 4) ** -0.25


def exact_second_moment(T: float) -> float:
    """E[X(T)^2] = integral of x^2 (1 + 4 T x^4)^(-1/2) phi(x) dx (adaptive quadrature)."""
    def integrand(x):
        return x * x / math.sqrt(1.0 + 4.0 * T * x ** 4) * math.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    val, _ = integrate.quad(integrand, -math.inf, math.inf, epsabs=1e-14, epsrel=1e-12)
    return val
