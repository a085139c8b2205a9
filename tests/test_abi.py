"""The C-ABI library: it loads, exports every function include/*.h declares, and rejects bad
arguments on the host before touching the device (these tests need no GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1505_00965_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mlmc_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["mlmc_level_sums", "mlmc_level_sums_ex", "mlmc_level_sums_async", "mlmc_estimate",
                     "mlmc_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_wraps_every_symbol():
    from paper_1505_00965_gb300 import mlmc

    for name in _declared_functions():
        assert callable(getattr(mlmc, name, None)), name


def test_version_and_error_string():
    from paper_1505_00965_gb300 import mlmc

    assert "sm_103a" in mlmc.mlmc_version()
    assert isinstance(mlmc.mlmc_last_error(), str)


@pytest.mark.parametrize("kw,msg", [
    (dict(level=-1), "level"),
    (dict(level=13), "level"),
    (dict(M=3), "M must be"),
    (dict(problem=dict(sigma=0.0)), "GBM"),
    (dict(problem=dict(S0=-1.0)), "GBM"),
    (dict(problem=dict(T=float("nan"))), "GBM"),
    (dict(problem=dict(payoff="lookback", K=float("inf"))), "finite"),
    (dict(tag=70000), "tag"),
])
def test_invalid_arguments_rejected_on_host(kw, msg):
    from paper_1505_00965_gb300 import mlmc

    args = dict(level=2, M=4, N=100, first=0, seed=1, tag=0)
    prob = dict()
    for k, v in kw.items():
        if k == "problem":
            prob.update(v)
        else:
            args[k] = v
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_level_sums_ex(args["level"], args["M"], args["N"], args["first"], mlmc.Problem(**prob),
                                args["seed"], tag=args["tag"])
    assert ei.value.status == mlmc.MLMC_EINVAL
    assert msg in str(ei.value)


def test_invalid_scheme_and_estimator(lib):
    from paper_1505_00965_gb300 import mlmc

    sums = (ctypes.c_double * 4)()
    cost = ctypes.c_double()
    p = mlmc.mlmc_payoff(0, 0, 100.0, 1.0)
    m = mlmc.mlmc_model(0, 2, 100.0, 0.05, 0.2, 1.0)
    assert lib.mlmc_level_sums(2, 4, ctypes.c_uint64(10), ctypes.byref(m), ctypes.byref(p), ctypes.c_uint64(1),
                               sums, ctypes.byref(cost)) == mlmc.MLMC_EINVAL
    m = mlmc.mlmc_model(0, 0, 100.0, 0.05, 0.2, 1.0)
    p = mlmc.mlmc_payoff(0, 5, 100.0, 1.0)
    assert lib.mlmc_level_sums(2, 4, ctypes.c_uint64(10), ctypes.byref(m), ctypes.byref(p), ctypes.c_uint64(1),
                               sums, ctypes.byref(cost)) == mlmc.MLMC_EINVAL
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_estimate(1e-2, mlmc.Problem(estimator="single"), 1)
    assert ei.value.status == mlmc.MLMC_EINVAL
    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_estimate_batch([(mlmc.Problem(scheme="milstein"), 1e-2, 1)])
    assert ei.value.status == mlmc.MLMC_EINVAL


def test_invalid_payoff_kind_and_overflow(lib):
    from paper_1505_00965_gb300 import mlmc

    m = mlmc.mlmc_model(0, 0, 100.0, 0.05, 0.2, 1.0)
    p = mlmc.mlmc_payoff(7, 0, 100.0, 1.0)
    sums = (ctypes.c_double * 4)()
    cost = ctypes.c_double()
    assert lib.mlmc_level_sums(2, 4, ctypes.c_uint64(10), ctypes.byref(m), ctypes.byref(p), ctypes.c_uint64(1),
                               sums, ctypes.byref(cost)) == mlmc.MLMC_EINVAL
    with pytest.raises(mlmc.MLMCError):
        mlmc.mlmc_level_sums_ex(2, 4, 10, 2 ** 64 - 5, mlmc.Problem(), 1)
    # NULL outputs
    p = mlmc.mlmc_payoff(0, 0, 100.0, 1.0)
    assert lib.mlmc_level_sums(2, 4, ctypes.c_uint64(10), ctypes.byref(m), ctypes.byref(p), ctypes.c_uint64(1),
                               None, None) == mlmc.MLMC_EINVAL


def test_estimate_argument_checks():
    from paper_1505_00965_gb300 import mlmc

    for kw in [dict(eps=0.0), dict(eps=-1.0), dict(M=5), dict(Lmin=0), dict(Lmin=5, Lmax=3), dict(Lmax=16),
               dict(N0=1)]:
        args = dict(eps=1e-2, M=4, Lmin=2, Lmax=8, N0=1000)
        args.update(kw)
        with pytest.raises(mlmc.MLMCError) as ei:
            mlmc.mlmc_estimate(args["eps"], mlmc.Problem(), 1, M=args["M"], Lmin=args["Lmin"], Lmax=args["Lmax"],
                               N0=args["N0"])
        assert ei.value.status == mlmc.MLMC_EINVAL


def test_no_cpu_fallback_without_gpu():
    """With no usable GPU the product reports a CUDA error; it never computes on the CPU."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1505_00965_gb300 import mlmc

    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_level_sums(2, 4, 100, mlmc.Problem(), 1)
    assert ei.value.status == mlmc.MLMC_ECUDA


def test_product_does_not_reference_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1505_00965_gb300", "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text and "mlmc_oracle" not in text, path


@pytest.mark.parametrize("kw,launch,msg", [
    (dict(kind="quintic", scheme="milstein", payoff="second_moment"), None, "tamed"),
    (dict(kind="quintic", scheme="tamed", payoff="european"), None, "second-moment"),
    (dict(kind="quintic", scheme="tamed", payoff="second_moment", T=0.0), None, "T > 0"),
    (dict(kind="gbm", scheme="tamed"), None, "Milstein"),
    (dict(payoff="second_moment"), None, "payoff kind"),
    (dict(kind="quintic", scheme="em", payoff="second_moment"), {"lanes_per_path": 4}, "one thread per sample"),
    (dict(kind="quintic", scheme="tamed", payoff="second_moment", estimator="antithetic"), None, "estimator"),
])
def test_quintic_model_arguments_rejected_on_host(kw, launch, msg):
    """The QUINTIC_ODE model (Sec. 5, Eq. count) pairs with EM or tamed EM and the second moment;
    GBM takes neither; its paths are never split over lanes."""
    from paper_1505_00965_gb300 import mlmc

    with pytest.raises(mlmc.MLMCError) as ei:
        mlmc.mlmc_level_sums_ex(2, 4, 100, 0, mlmc.Problem(**kw), 1, launch=launch)
    assert ei.value.status == mlmc.MLMC_EINVAL
    assert msg in str(ei.value)


def test_batched_level_sums_arguments_rejected_on_host():
    """mlmc_level_sums_batch checks every task before any device work."""
    from paper_1505_00965_gb300 import mlmc

    ok = mlmc.Problem(payoff="asian")
    cases = [
        ([(ok, 1, 2, 0, 10)], dict(M=3), "M must be"),
        ([(ok, 1, 2, 0, 10)], dict(precision="fp64_stream32"), "batches run"),
        ([(ok, 1, 16, 0, 10)], {}, "level 16 out of range"),
        ([(mlmc.Problem(payoff="asian", scheme="milstein"), 1, 2, 0, 10)], {}, "coupled Euler--Maruyama"),
        ([(ok, 1, 2, 2 ** 64 - 5, 10)], {}, "overflows"),
        ([(ok, 1, 2, 0, 2 ** 32)], {}, "2^32"),
    ]
    for tasks, kw, msg in cases:
        with pytest.raises(mlmc.MLMCError) as ei:
            mlmc.mlmc_level_sums_batch(tasks, **kw)
        assert ei.value.status in (mlmc.MLMC_EINVAL, mlmc.MLMC_ENOTIMPL)
        assert msg in str(ei.value), (msg, str(ei.value))


def test_driver_mode_switch_on_host():
    """mlmc_set_driver_mode validates its argument and reports the mode it replaces (no GPU)."""
    from paper_1505_00965_gb300 import mlmc

    prev = mlmc.mlmc_set_driver_mode("host")
    assert prev == "host"  # the default
    try:
        assert mlmc.mlmc_set_driver_mode("device") == "host"
        with pytest.raises(mlmc.MLMCError) as ei:
            mlmc.mlmc_set_driver_mode(3)
        assert ei.value.status == mlmc.MLMC_EINVAL
        assert mlmc.mlmc_set_driver_mode("auto") == "device"
    finally:
        mlmc.mlmc_set_driver_mode(prev)
