"""FP64 CPU oracle for one multilevel Monte Carlo level and for the adaptive driver.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
use this package.  The product library never imports, links or calls it, and it shares no
code with the CUDA path.  The arithmetic lives in ``mlmc_oracle.c`` (plain C, FP64, compiled
with ``-ffp-contract=off``); this module only loads it with ctypes and marshals arguments.

Functions and the passages they follow (D. J. Higham, "An Introduction to Multilevel Monte
Carlo for Option Valuation"):

* ``philox``, ``normals``           -- the random input dW of Eq. (em); the stream is a reading
                                        (Philox4x32-10 + Box--Muller), see ``mlmc_oracle.c``.
* ``sample_paths``, ``em_path``     -- Euler--Maruyama (Sec. 2, Eq. em) on the fine and coarse
                                        grids of one Brownian path (Sec. 5, Fig. 2); Problem.scheme
                                        "milstein" switches both grids to the Milstein step (Sec. 5).
* ``payoff``                        -- discounted payoffs (Sec. 5 and Sec. 6).
* ``level_samples``, ``level_sums`` -- the level estimators of Eqs. (mlmc:Yzero) and (Yldef).
* ``driver.estimate``               -- telescoping sum Eq. (mlmc:ident) with N_l chosen from
                                        estimated variances (Sec. 5 remarks; Theorem of Sec. 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlmc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmlmc_oracle.so")
_lock = threading.Lock()
_lib = None

PAYOFFS = {"european": 0, "asian": 1, "lookback": 2, "digital": 3, "linear": 100, "geo_asian": 101}
STREAMS = {"fp64": 0, "fp32": 1}
SCHEMES = {"em": 0, "milstein": 1}
MODE_COUPLED, MODE_FINE_ONLY, MODE_ANTITHETIC = 0, 1, 2
TAG_PATHS, TAG_CV_MEAN, TAG_CV_TRAIN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle's C source into a shared library beside it (gcc, FP64, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [("S0", ctypes.c_double), ("r", ctypes.c_double), ("sigma", ctypes.c_double),
                ("T", ctypes.c_double), ("payoff", ctypes.c_int), ("K", ctypes.c_double),
                ("Q", ctypes.c_double), ("scheme", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            dptr = ctypes.POINTER(ctypes.c_double)
            u32ptr = ctypes.POINTER(ctypes.c_uint32)
            pp = ctypes.POINTER(_Problem)
            lib.oracle_philox4x32_10.argtypes = [u32ptr, u32ptr, u32ptr]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_uniform.argtypes = [ctypes.c_uint32, i32]
            lib.oracle_uniform.restype = dbl
            lib.oracle_normals.argtypes = [u64, i32, i32, u64, i32, i32, dptr]
            lib.oracle_normals.restype = None
            lib.oracle_sample_normals.argtypes = [u64, i32, i32, i32, u64, i32, dptr]
            lib.oracle_sample_normals.restype = None
            lib.oracle_em_path.argtypes = [i32, dbl, dbl, dbl, dbl, dptr, dptr]
            lib.oracle_em_path.restype = None
            lib.oracle_milstein_path.argtypes = [i32, dbl, dbl, dbl, dbl, dptr, dptr]
            lib.oracle_milstein_path.restype = None
            lib.oracle_payoff.argtypes = [i32, dbl, dbl, dbl, dbl, dptr, i32]
            lib.oracle_payoff.restype = dbl
            lib.oracle_sample_paths.argtypes = [i32, i32, u64, i32, pp, u64, i32, dptr, dptr, dptr]
            lib.oracle_sample_paths.restype = i32
            lib.oracle_grid_brownian.argtypes = [i32, i32, u64, i32, dbl, u64, i32, dptr]
            lib.oracle_grid_brownian.restype = None
            lib.oracle_level_samples.argtypes = [i32, i32, u64, u64, i32, i32, pp, u64, i32, dptr]
            lib.oracle_level_samples.restype = i32
            lib.oracle_level_sums.argtypes = [i32, i32, u64, u64, i32, i32, pp, u64, i32, dptr, dptr]
            lib.oracle_level_sums.restype = i32
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Problem:
    """GBM dS = r S dt + sigma S dW on [0, T] with a discounted payoff (Sec. 6 model)."""

    S0: float = 100.0
    r: float = 0.05
    sigma: float = 0.2
    T: float = 1.0
    payoff: str = "european"
    K: float = 100.0
    Q: float = 1.0
    scheme: str = "em"

    def c(self) -> _Problem:
        return _Problem(self.S0, self.r, self.sigma, self.T, PAYOFFS[self.payoff], self.K, self.Q,
                        SCHEMES[self.scheme])


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox(ctr, key) -> tuple:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def uniform(x: int, stream: str = "fp64") -> float:
    return _load().oracle_uniform(int(x) & 0xFFFFFFFF, STREAMS[stream])


def sample_normals(seed: int, level: int, M: int, s: int, stream: str = "fp64", tag: int = TAG_PATHS) -> np.ndarray:
    """The M^l normals that drive sample s's fine increments."""
    z = np.empty(M ** level, dtype=np.float64)
    _load().oracle_sample_normals(seed, level, M, tag, s, STREAMS[stream], _dp(z))
    return z


def normals(seed: int, level: int, s: int, n: int, stream: str = "fp64", tag: int = TAG_PATHS) -> np.ndarray:
    n4 = (n + 3) // 4 * 4
    z = np.empty(n4, dtype=np.float64)
    _load().oracle_normals(seed, level, tag, s, STREAMS[stream], n4, _dp(z))
    return z[:n]


def em_path(S0: float, r: float, sigma: float, h: float, dW: np.ndarray) -> np.ndarray:
    dW = np.ascontiguousarray(dW, dtype=np.float64)
    out = np.empty(len(dW) + 1, dtype=np.float64)
    _load().oracle_em_path(len(dW), S0, r, sigma, h, _dp(dW), _dp(out))
    return out


def payoff(p: Problem, path: np.ndarray) -> float:
    path = np.ascontiguousarray(path, dtype=np.float64)
    return _load().oracle_payoff(PAYOFFS[p.payoff], p.K, p.Q, p.r, p.T, _dp(path), len(path) - 1)


def sample_paths(level: int, M: int, s: int, p: Problem, seed: int, stream: str = "fp64", tag: int = TAG_PATHS):
    """(fine increments, fine path, coarse path or None) of sample s of level l."""
    nf = M ** level
    dW = np.empty(nf, dtype=np.float64)
    fine = np.empty(nf + 1, dtype=np.float64)
    coarse = np.empty(nf // M + 1, dtype=np.float64)
    prob = p.c()
    _load().oracle_sample_paths(level, M, s, tag, ctypes.byref(prob), seed, STREAMS[stream],
                                _dp(dW), _dp(fine), _dp(coarse) if level > 0 else None)
    return dW, fine, (coarse if level > 0 else None)


def grid_brownian(level: int, M: int, s: int, T: float, seed: int, stream: str = "fp64", tag: int = TAG_PATHS) -> np.ndarray:
    W = np.empty(16, dtype=np.float64)
    _load().oracle_grid_brownian(level, M, s, tag, T, seed, STREAMS[stream], _dp(W))
    return W


def level_samples(level: int, M: int, N: int, p: Problem, seed: int, first: int = 0, stream: str = "fp64",
                  tag: int = TAG_PATHS, mode: int = MODE_COUPLED) -> np.ndarray:
    Y = np.empty(N, dtype=np.float64)
    prob = p.c()
    rc = _load().oracle_level_samples(level, M, N, first, tag, mode, ctypes.byref(prob), seed, STREAMS[stream], _dp(Y))
    if rc:
        raise ValueError("oracle_level_samples: invalid arguments")
    return Y


def level_sums(level: int, M: int, N: int, p: Problem, seed: int, first: int = 0, stream: str = "fp64",
               tag: int = TAG_PATHS, mode: int = MODE_COUPLED):
    """(sums[4] = sum Y^k for k = 1..4, cost = N C_l) over samples [first, first + N)."""
    sums = np.zeros(4, dtype=np.float64)
    cost = ctypes.c_double(0.0)
    prob = p.c()
    rc = _load().oracle_level_sums(level, M, N, first, tag, mode, ctypes.byref(prob), seed, STREAMS[stream],
                                   _dp(sums), ctypes.byref(cost))
    if rc:
        raise ValueError("oracle_level_sums: invalid arguments")
    return sums, cost.value
