"""Python binding of the GB300 multilevel Monte Carlo level engine (include/mlmc.h).

Argument marshalling only: every step of the path runs in the CUDA library
``libmlmc_gb300.so`` built from ``csrc/`` for sm_103a.  The functions keep the C names; they
raise ``MLMCError`` for a non-zero status and return the outputs.  Importing this package
fails loudly if the library has not been built; there is no CPU fallback.

Device buffers and streams for the ``_async`` entry point come from PyTorch (any object with
``data_ptr()``, or a raw integer address; a ``torch.cuda.Stream`` or a raw handle).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmlmc_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first (python -m paper_1505_00965_gb300.build)")

_lib = ctypes.CDLL(LIB_PATH)

MLMC_OK, MLMC_EINVAL, MLMC_ECUDA, MLMC_ENOMEM, MLMC_ENOTCONV, MLMC_ETIMEOUT, MLMC_ENOTIMPL, MLMC_ENONFINITE = range(8)
MLMC_MODEL_GBM, MLMC_MODEL_QUINTIC_ODE = 0, 1
MODELS = {"gbm": MLMC_MODEL_GBM, "quintic": MLMC_MODEL_QUINTIC_ODE}
PAYOFFS = {"european": 0, "asian": 1, "lookback": 2, "digital": 3, "second_moment": 4, "linear": 100,
           "geo_asian": 101}
MLMC_FP64, MLMC_FP32_PATH, MLMC_FP64_STREAM32 = 0, 1, 2
PRECISIONS = {"fp64": MLMC_FP64, "fp32": MLMC_FP32_PATH, "fp64_stream32": MLMC_FP64_STREAM32}
SCHEMES = {"em": 0, "milstein": 1, "tamed": 2}
ESTIMATORS = {"coupled": 0, "single": 1, "antithetic": 2}
MLMC_TAG_PATHS, MLMC_TAG_CV_MEAN, MLMC_TAG_CV_TRAIN = 0, 1, 2
MLMC_MAX_LEVELS = 16


class MLMCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mlmc status {status}: {message}")
        self.status = status


class mlmc_model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("scheme", ctypes.c_int32), ("S0", ctypes.c_double),
                ("r", ctypes.c_double), ("sigma", ctypes.c_double), ("T", ctypes.c_double)]


class mlmc_payoff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("estimator", ctypes.c_int32), ("K", ctypes.c_double),
                ("cash", ctypes.c_double)]


class mlmc_launch(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("lanes_per_path", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("samples_per_thread", ctypes.c_int32)]


class mlmc_problem(ctypes.Structure):
    _fields_ = [("model", mlmc_model), ("payoff", mlmc_payoff), ("eps", ctypes.c_double), ("seed", ctypes.c_uint64)]


class mlmc_level_task(ctypes.Structure):
    _fields_ = [("problem", mlmc_problem), ("level", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("first", ctypes.c_uint64), ("N", ctypes.c_uint64)]


class mlmc_result(ctypes.Structure):
    _fields_ = [("P", ctypes.c_double), ("eps", ctypes.c_double), ("L", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("rounds", ctypes.c_int32), ("device_rounds", ctypes.c_int32),
                ("N", ctypes.c_uint64 * MLMC_MAX_LEVELS),
                ("sums", (ctypes.c_double * 4) * MLMC_MAX_LEVELS),
                ("mean", ctypes.c_double * MLMC_MAX_LEVELS), ("var", ctypes.c_double * MLMC_MAX_LEVELS),
                ("cost", ctypes.c_double * MLMC_MAX_LEVELS), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("total_cost", ctypes.c_double), ("path_steps", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("wall_ms", ctypes.c_double), ("launches", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64)]


_u64, _i32, _dbl, _vp, _sz = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_dptr = ctypes.POINTER(ctypes.c_double)
_pm, _pp, _pl = ctypes.POINTER(mlmc_model), ctypes.POINTER(mlmc_payoff), ctypes.POINTER(mlmc_launch)

MLMC_CV_PARAMS = 5313
MLMC_CV_INPUTS = 16
MLMC_CV_LATTICE_POINTS = 65536
MLMC_CV_MAX_LEVELS = 8


class mlmc_cv_options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n_train", ctypes.c_uint64), ("lr", ctypes.c_double),
                ("init_seed", ctypes.c_uint64)]


class mlmc_cv_level_info(ctypes.Structure):
    _fields_ = [("trained", ctypes.c_int32), ("used", ctypes.c_int32), ("var_plain", ctypes.c_double),
                ("var_resid", ctypes.c_double), ("var_g", ctypes.c_double), ("kappa", ctypes.c_double),
                ("t_plain", ctypes.c_double), ("t_cv", ctypes.c_double), ("t_mean", ctypes.c_double),
                ("work_ratio", ctypes.c_double), ("train_loss", ctypes.c_double), ("var_lattice", ctypes.c_double)]


class mlmc_cv_train_stats(ctypes.Structure):
    _fields_ = [("data_ms", ctypes.c_double), ("train_ms", ctypes.c_double), ("train_kernel_ms", ctypes.c_double),
                ("eval_ms", ctypes.c_double), ("cost_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("steps", ctypes.c_int64), ("cluster", ctypes.c_int32), ("levels", ctypes.c_int32)]


_fptr = ctypes.POINTER(ctypes.c_float)
_SIGNATURES = {
    "mlmc_last_error": ([], ctypes.c_char_p),
    "mlmc_version": ([], ctypes.c_char_p),
    "mlmc_device_sm_count": ([], _i32),
    "mlmc_shutdown": ([], _i32),
    "mlmc_set_driver_mode": ([_i32, ctypes.POINTER(_i32)], _i32),
    "mlmc_level_sums": ([_i32, _i32, _u64, _pm, _pp, _u64, _dptr, _dptr], _i32),
    "mlmc_level_sums_ex": ([_i32, _i32, _u64, _u64, _pm, _pp, _u64, _i32, _i32, _pl, _vp, _dptr, _dptr], _i32),
    "mlmc_level_workspace_bytes": ([_i32, _i32, _u64, _i32, _pl], _sz),
    "mlmc_level_sums_async": ([_i32, _i32, _u64, _u64, _pm, _pp, _u64, _i32, _i32, _pl, _vp, _vp, _sz, _vp, _vp],
                              _i32),
    "mlmc_level_sums_noalloc": ([_i32, _i32, _u64, _u64, _pm, _pp, _u64, _i32, _i32, _pl, _vp, _vp, _vp], _i32),
    "mlmc_cv_create": ([_i32, _pm, _pp, ctypes.POINTER(_vp)], _i32),
    "mlmc_cv_train": ([_i32, _pm, _pp, _u64, ctypes.POINTER(mlmc_cv_options), _vp, ctypes.POINTER(_vp)], _i32),
    "mlmc_cv_free": ([_vp], _i32),
    "mlmc_cv_info": ([_vp, _i32, ctypes.POINTER(mlmc_cv_level_info)], _i32),
    "mlmc_cv_train_info": ([_vp, ctypes.POINTER(mlmc_cv_train_stats)], _i32),
    "mlmc_cv_get_params": ([_vp, _i32, _fptr], _i32),
    "mlmc_cv_set_params": ([_vp, _i32, _fptr, _dbl], _i32),
    "mlmc_cv_level_sums": ([_vp, _i32, _u64, _u64, _u64, _vp, _vp, _vp, _vp], _i32),
    "mlmc_cv_mean_sums": ([_vp, _i32, _u64, _u64, _u64, _vp, _vp, _vp], _i32),
    "mlmc_cv_training_data": ([_vp, _i32, _u64, _u64, _u64, _vp, _vp, _vp], _i32),
    "mlmc_mlp_forward": ([_fptr, _vp, _u64, _vp, _vp], _i32),
    "mlmc_mlp_grad": ([_fptr, _vp, _vp, _u64, _fptr, ctypes.POINTER(_dbl), _vp], _i32),
    "mlmc_estimate_cv": ([_dbl, _i32, _i32, _i32, _u64, _pm, _pp, _u64, _vp, _vp, ctypes.POINTER(mlmc_result)], _i32),
    "mlmc_autotune": ([_i32, _i32, _i32, _i32, _vp, ctypes.POINTER(_i32)], _i32),
    "mlmc_autotune_save": ([ctypes.c_char_p], _i32),
    "mlmc_autotune_load": ([ctypes.c_char_p, ctypes.POINTER(_i32)], _i32),
    "mlmc_autotune_clear": ([], _i32),
    "mlmc_autotune_entries": ([], _i32),
    "mlmc_autotune_lookup": ([_i32, _i32, _i32, _i32, _u64, _pl], _i32),
    "mlmc_estimate_batch": ([_i32, ctypes.c_void_p, _i32, _i32, _i32, _u64, _i32, _vp, ctypes.c_void_p], _i32),
    "mlmc_level_sums_batch": ([_i32, ctypes.c_void_p, _i32, _i32, _dptr, _vp, _vp], _i32),
    "mlmc_estimate": ([_dbl, _i32, _i32, _i32, _u64, _pm, _pp, _u64, _i32, _vp, ctypes.POINTER(mlmc_result)], _i32),
}
for _name, (_args, _res) in _SIGNATURES.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _check(status: int) -> None:
    if status != MLMC_OK:
        raise MLMCError(status, mlmc_last_error())


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "cuda_stream"):
        return x.cuda_stream
    raise TypeError(f"cannot take a device address of {type(x)!r}")


@dataclass(frozen=True)
class Problem:
    """A model and a payoff (the C structs in Python form): GBM dS = r S dt + sigma S dW with a
    discounted payoff, or (kind="quintic") the random ODE dX = -X^5 dt with X(0) ~ N(0, 1) and the
    second moment X(T)^2 (scheme "em" or "tamed")."""

    S0: float = 100.0
    r: float = 0.05
    sigma: float = 0.2
    T: float = 1.0
    payoff: str = "european"
    K: float = 100.0
    cash: float = 1.0
    scheme: str = "em"            # "em" (Euler--Maruyama) or "milstein"
    estimator: str = "coupled"    # "coupled" (P_l - P_{l-1}) or "single" (P_l, standard MC)
    kind: str = "gbm"             # "gbm" or "quintic"

    def model(self) -> mlmc_model:
        return mlmc_model(MODELS[self.kind], SCHEMES[self.scheme], self.S0, self.r, self.sigma, self.T)

    def payoff_struct(self) -> mlmc_payoff:
        return mlmc_payoff(PAYOFFS[self.payoff], ESTIMATORS[self.estimator], self.K, self.cash)


def _launch(launch) -> mlmc_launch | None:
    if launch is None:
        return None
    if isinstance(launch, mlmc_launch):
        return launch
    return mlmc_launch(int(launch.get("threads_per_block", 0)), int(launch.get("lanes_per_path", 0)),
                       int(launch.get("blocks", 0)), int(launch.get("samples_per_thread", 0)))


def _prec(precision) -> int:
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def mlmc_last_error() -> str:
    return (_lib.mlmc_last_error() or b"").decode()


def mlmc_version() -> str:
    return _lib.mlmc_version().decode()


def mlmc_device_sm_count() -> int:
    n = _lib.mlmc_device_sm_count()
    if n < 0:
        raise MLMCError(MLMC_ECUDA, mlmc_last_error())
    return n


def mlmc_shutdown() -> None:
    _check(_lib.mlmc_shutdown())


def mlmc_level_sums(level: int, M: int, N: int, problem: Problem, seed: int):
    """(sums[4], cost): FP32 paths, samples [0, N), default stream."""
    sums = (ctypes.c_double * 4)()
    cost = ctypes.c_double()
    m, p = problem.model(), problem.payoff_struct()
    _check(_lib.mlmc_level_sums(level, M, N, ctypes.byref(m), ctypes.byref(p), seed, sums, ctypes.byref(cost)))
    return list(sums), cost.value


def mlmc_level_sums_ex(level: int, M: int, N: int, first: int, problem: Problem, seed: int,
                       precision="fp32", tag: int = MLMC_TAG_PATHS, launch=None, stream=None):
    """(sums[4], cost) over samples [first, first + N); synchronises `stream`."""
    sums = (ctypes.c_double * 4)()
    cost = ctypes.c_double()
    m, p, ln = problem.model(), problem.payoff_struct(), _launch(launch)
    _check(_lib.mlmc_level_sums_ex(level, M, N, first, ctypes.byref(m), ctypes.byref(p), seed, _prec(precision),
                                   tag, ctypes.byref(ln) if ln is not None else None, _addr(stream), sums,
                                   ctypes.byref(cost)))
    return list(sums), cost.value


def mlmc_level_workspace_bytes(level: int, M: int, N: int, precision="fp32", launch=None) -> int:
    ln = _launch(launch)
    n = _lib.mlmc_level_workspace_bytes(level, M, N, _prec(precision), ctypes.byref(ln) if ln is not None else None)
    if n == 0:
        raise MLMCError(MLMC_EINVAL, mlmc_last_error())
    return n


def mlmc_level_sums_async(level: int, M: int, N: int, first: int, problem: Problem, seed: int, d_sums,
                          d_workspace, workspace_bytes: int, precision="fp32", tag: int = MLMC_TAG_PATHS,
                          launch=None, d_y=None, stream=None) -> None:
    """Queue the level on `stream`; d_sums (4 doubles), d_workspace and d_y are device buffers."""
    m, p, ln = problem.model(), problem.payoff_struct(), _launch(launch)
    _check(_lib.mlmc_level_sums_async(level, M, N, first, ctypes.byref(m), ctypes.byref(p), seed, _prec(precision),
                                      tag, ctypes.byref(ln) if ln is not None else None, _addr(d_sums),
                                      _addr(d_workspace), workspace_bytes, _addr(d_y), _addr(stream)))


def mlmc_level_sums_noalloc(level: int, M: int, N: int, first: int, problem: Problem, seed: int, d_sums,
                            precision="fp32", tag: int = MLMC_TAG_PATHS, launch=None, d_y=None, stream=None) -> None:
    """Queue the level on `stream` with the library's fixed device scratch (no allocation).
    The first call on a device looks up the scratch address; calls that overlap on the GPU race."""
    m, p, ln = problem.model(), problem.payoff_struct(), _launch(launch)
    _check(_lib.mlmc_level_sums_noalloc(level, M, N, first, ctypes.byref(m), ctypes.byref(p), seed,
                                        _prec(precision), tag, ctypes.byref(ln) if ln is not None else None,
                                        _addr(d_sums), _addr(d_y), _addr(stream)))


@dataclass
class Estimate:
    status: int
    P: float
    eps: float
    L: int
    converged: bool
    rounds: int
    N: list = field(default_factory=list)
    sums: list = field(default_factory=list)
    mean: list = field(default_factory=list)
    var: list = field(default_factory=list)
    cost: list = field(default_factory=list)
    alpha: float = 0.0
    beta: float = 0.0
    total_cost: float = 0.0
    path_steps: float = 0.0
    kernel_ms: float = 0.0
    wall_ms: float = 0.0
    launches: int = 0
    d2h_bytes: int = 0
    device_rounds: bool = False


def _estimate_from(st: int, r: mlmc_result) -> "Estimate":
    L = r.L
    return Estimate(status=st, P=r.P, eps=r.eps, L=L, converged=bool(r.converged), rounds=r.rounds,
                    N=[int(r.N[l]) for l in range(L + 1)], sums=[list(r.sums[l]) for l in range(L + 1)],
                    mean=[r.mean[l] for l in range(L + 1)], var=[r.var[l] for l in range(L + 1)],
                    cost=[r.cost[l] for l in range(L + 1)], alpha=r.alpha, beta=r.beta, total_cost=r.total_cost,
                    path_steps=r.path_steps, kernel_ms=r.kernel_ms, wall_ms=r.wall_ms, launches=int(r.launches),
                    d2h_bytes=int(r.d2h_bytes), device_rounds=bool(r.device_rounds))


def mlmc_estimate_batch(problems, M: int = 4, Lmin: int = 2, Lmax: int = 8, N0: int = 10_000, precision="fp32",
                        stream=None) -> list:
    """Adaptive estimates of many problems together.  `problems` holds (Problem, eps, seed)
    triples or dicts with the Problem fields plus eps and seed.  Returns one Estimate each
    (status MLMC_ENOTCONV on those that reached Lmax first)."""
    n = len(problems)
    arr = (mlmc_problem * n)()
    for i, q in enumerate(problems):
        if isinstance(q, dict):
            prob = Problem(**{k: q[k] for k in ("S0", "r", "sigma", "T", "payoff", "K", "cash", "scheme") if k in q})
            eps, seed = q["eps"], q["seed"]
        else:
            prob, eps, seed = q
        arr[i] = mlmc_problem(prob.model(), prob.payoff_struct(), eps, seed)
    res = (mlmc_result * n)()
    st = _lib.mlmc_estimate_batch(n, ctypes.cast(arr, ctypes.c_void_p), M, Lmin, Lmax, N0, _prec(precision),
                                  _addr(stream), ctypes.cast(res, ctypes.c_void_p))
    if st not in (MLMC_OK, MLMC_ENOTCONV):
        _check(st)
    return [_estimate_from(MLMC_OK if res[i].converged else MLMC_ENOTCONV, res[i]) for i in range(n)]


DRIVER_MODES = {"auto": 0, "host": 1, "device": 2}


def mlmc_set_driver_mode(mode) -> str:
    """Where mlmc_estimate runs its rounds ("auto", "host" or "device"); returns the previous mode."""
    prev = ctypes.c_int(0)
    _check(_lib.mlmc_set_driver_mode(DRIVER_MODES[mode] if isinstance(mode, str) else int(mode), ctypes.byref(prev)))
    return {v: k for k, v in DRIVER_MODES.items()}[prev.value]


def mlmc_level_sums_batch(tasks, M: int = 4, precision="fp32", d_y=None, stream=None):
    """Level sums of many (Problem, seed, level, first, N) ranges in one batched round.  Returns
    a list of four sums per task; d_y (device buffer or None) receives every sample's Y."""
    n = len(tasks)
    arr = (mlmc_level_task * n)()
    for i, (prob, seed, level, first, N) in enumerate(tasks):
        arr[i] = mlmc_level_task(mlmc_problem(prob.model(), prob.payoff_struct(), 1.0, seed), level, 0, first, N)
    out = (ctypes.c_double * (4 * n))()
    _check(_lib.mlmc_level_sums_batch(n, ctypes.cast(arr, ctypes.c_void_p), M, _prec(precision), out, _addr(d_y),
                                      _addr(stream)))
    return [list(out[4 * i:4 * i + 4]) for i in range(n)]


def mlmc_estimate(eps: float, problem: Problem, seed: int, M: int = 4, Lmin: int = 2, Lmax: int = 8,
                  N0: int = 10_000, precision="fp32", stream=None) -> Estimate:
    """Adaptive estimate to RMS accuracy eps.  Returns the estimate also when Lmax was reached
    before the bias test passed (status MLMC_ENOTCONV, converged False)."""
    r = mlmc_result()
    m, p = problem.model(), problem.payoff_struct()
    st = _lib.mlmc_estimate(eps, M, Lmin, Lmax, N0, ctypes.byref(m), ctypes.byref(p), seed, _prec(precision),
                            _addr(stream), ctypes.byref(r))
    if st not in (MLMC_OK, MLMC_ENOTCONV):
        _check(st)
    return _estimate_from(st, r)


# ------------------------------------------------------------------ learned control variate

def _floats(a, n=MLMC_CV_PARAMS):
    import numpy as np

    arr = np.ascontiguousarray(a, dtype=np.float32)
    if arr.shape != (n,):
        raise ValueError(f"expected {n} parameters")
    return arr, arr.ctypes.data_as(_fptr)


class ControlVariate:
    """Owner of an mlmc_cv handle (freed with the object)."""

    def __init__(self, handle: int, M: int, problem: Problem):
        self.handle = ctypes.c_void_p(handle)
        self.M = M
        self.problem = problem

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.mlmc_cv_free(h)
            self.handle = None


def mlmc_cv_create(M: int, problem: Problem) -> ControlVariate:
    h = ctypes.c_void_p()
    m, p = problem.model(), problem.payoff_struct()
    _check(_lib.mlmc_cv_create(M, ctypes.byref(m), ctypes.byref(p), ctypes.byref(h)))
    return ControlVariate(h.value, M, problem)


def mlmc_cv_train(M: int, problem: Problem, seed: int, levels: int = 4, epochs: int = 20, batch: int = 4096,
                  n_train: int = 1_000_000, lr: float = 1e-3, init_seed: int = 0, stream=None) -> ControlVariate:
    h = ctypes.c_void_p()
    m, p = problem.model(), problem.payoff_struct()
    o = mlmc_cv_options(levels, epochs, batch, 0, n_train, lr, init_seed)
    _check(_lib.mlmc_cv_train(M, ctypes.byref(m), ctypes.byref(p), seed, ctypes.byref(o), _addr(stream),
                              ctypes.byref(h)))
    return ControlVariate(h.value, M, problem)


def mlmc_cv_free(cv: ControlVariate) -> None:
    if cv.handle is not None and cv.handle.value:
        _check(_lib.mlmc_cv_free(cv.handle))
        cv.handle = None


def mlmc_cv_info(cv: ControlVariate, level: int) -> dict:
    info = mlmc_cv_level_info()
    _check(_lib.mlmc_cv_info(cv.handle, level, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in mlmc_cv_level_info._fields_}


def mlmc_cv_train_info(cv: ControlVariate) -> dict:
    st = mlmc_cv_train_stats()
    _check(_lib.mlmc_cv_train_info(cv.handle, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in mlmc_cv_train_stats._fields_}


def mlmc_cv_get_params(cv: ControlVariate, level: int):
    import numpy as np

    out = np.zeros(MLMC_CV_PARAMS, dtype=np.float32)
    _check(_lib.mlmc_cv_get_params(cv.handle, level, out.ctypes.data_as(_fptr)))
    return out


def mlmc_cv_set_params(cv: ControlVariate, level: int, params, kappa: float = 1.0) -> None:
    arr, ptr = _floats(params)
    _check(_lib.mlmc_cv_set_params(cv.handle, level, ptr, kappa))


def mlmc_cv_level_sums(cv: ControlVariate, level: int, N: int, first: int, seed: int, d_sums8, d_r=None, d_g=None,
                       stream=None) -> None:
    _check(_lib.mlmc_cv_level_sums(cv.handle, level, N, first, seed, _addr(d_sums8), _addr(d_r), _addr(d_g),
                                   _addr(stream)))


def mlmc_cv_mean_sums(cv: ControlVariate, level: int, R: int, first: int, seed: int, d_sums2, d_g=None,
                      stream=None) -> None:
    _check(_lib.mlmc_cv_mean_sums(cv.handle, level, R, first, seed, _addr(d_sums2), _addr(d_g), _addr(stream)))


def mlmc_cv_training_data(cv: ControlVariate, level: int, N: int, first: int, seed: int, d_X, d_Y,
                          stream=None) -> None:
    _check(_lib.mlmc_cv_training_data(cv.handle, level, N, first, seed, _addr(d_X), _addr(d_Y), _addr(stream)))


def mlmc_mlp_forward(params, d_X, N: int, d_G, stream=None) -> None:
    arr, ptr = _floats(params)
    _check(_lib.mlmc_mlp_forward(ptr, _addr(d_X), N, _addr(d_G), _addr(stream)))


def mlmc_mlp_grad(params, d_X, d_Y, N: int, stream=None):
    """(loss, gradient) of the mean squared error on device rows d_X [N][16], d_Y [N]."""
    import numpy as np

    arr, ptr = _floats(params)
    grad = np.zeros(MLMC_CV_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(_lib.mlmc_mlp_grad(ptr, _addr(d_X), _addr(d_Y), N, grad.ctypes.data_as(_fptr), ctypes.byref(loss),
                              _addr(stream)))
    return loss.value, grad


def mlmc_estimate_cv(eps: float, cv: ControlVariate, seed: int, Lmin: int = 2, Lmax: int = 8, N0: int = 10_000,
                     stream=None) -> Estimate:
    r = mlmc_result()
    m, p = cv.problem.model(), cv.problem.payoff_struct()
    st = _lib.mlmc_estimate_cv(eps, cv.M, Lmin, Lmax, N0, ctypes.byref(m), ctypes.byref(p), seed, cv.handle,
                               _addr(stream), ctypes.byref(r))
    if st not in (MLMC_OK, MLMC_ENOTCONV):
        _check(st)
    return _estimate_from(st, r)


# ------------------------------------------------------------------ autotuner

def mlmc_autotune(M: int = 4, max_level: int = 8, precision="fp32", payoff: str = "asian", stream=None) -> int:
    """Tune launch shapes; returns the number of table entries added."""
    n = ctypes.c_int()
    _check(_lib.mlmc_autotune(M, max_level, _prec(precision), PAYOFFS[payoff], _addr(stream), ctypes.byref(n)))
    return n.value


def mlmc_autotune_save(path: str) -> None:
    _check(_lib.mlmc_autotune_save(os.fsencode(path)))


def mlmc_autotune_load(path: str) -> int:
    n = ctypes.c_int()
    _check(_lib.mlmc_autotune_load(os.fsencode(path), ctypes.byref(n)))
    return n.value


def mlmc_autotune_clear() -> None:
    _check(_lib.mlmc_autotune_clear())


def mlmc_autotune_entries() -> int:
    return int(_lib.mlmc_autotune_entries())


def mlmc_autotune_lookup(precision, payoff: str, M: int, level: int, N: int):
    """(threads_per_block, lanes_per_path, waves, samples_per_thread) or None."""
    out = mlmc_launch()
    st = _lib.mlmc_autotune_lookup(_prec(precision), PAYOFFS[payoff], M, level, N, ctypes.byref(out))
    if st != MLMC_OK:
        return None
    return out.threads_per_block, out.lanes_per_path, out.blocks, out.samples_per_thread
