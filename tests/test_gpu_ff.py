"""Accuracy of the float-float exp and log the mixed-precision path uses for
its Arrhenius rates and temperature (Tang's table-driven exp; log from the
FP32 logarithm y as y + log(1 + t), t = x e^(-y) - 1, to second order in t),
against numpy's FP64 functions.

Inputs carry at most 48 significant bits, so their float-float split is
exact and the FP64 reference sees the same argument.  Float-float keeps
about 48 bits (relative 2^-48 = 3.6e-15 per operation); the exp chain has a
table entry stored to that precision and about ten float-float operations,
so its relative error bound is stated as 2e-14; log's absolute error as
2e-14 * max(1, |log x|).  Float-float has FP32's exponent range: below
2^-102 (exp of x < -70.7) the low part of a result falls into FP32's
denormals, and the error there is bounded by their spacing (absolute
1.4e-45 per part) instead."""
import numpy as np
import pytest

from paper_2108_07605_gb300 import lbm

pytestmark = pytest.mark.gpu


def _48bit(x):
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 2.0 ** 48) / 2.0 ** 48, e)


def test_ff_exp_relative_error():
    rng = np.random.default_rng(11)
    x = _48bit(np.concatenate([rng.uniform(-87.0, 88.0, 200_000),
                               rng.uniform(-1e-3, 1e-3, 20_000),
                               np.arange(-80, 81, dtype=np.float64) * np.log(2.0) / 64]))
    e, _ = lbm.lbm_ff_check(x)
    ref = np.exp(x)
    full = x > np.log(2.0 ** -102)
    rel = np.abs(e[full] - ref[full]) / ref[full]
    assert rel.max() < 2e-14, (rel.max(), x[full][np.argmax(rel)])
    low = ~full
    assert low.sum() > 1000
    assert np.all(np.abs(e[low] - ref[low]) <= 2e-14 * ref[low] + 4 * 2.0 ** -149)


def test_ff_log_error():
    rng = np.random.default_rng(12)
    x = _48bit(np.concatenate([10.0 ** rng.uniform(-30, 30, 200_000),
                               1.0 + rng.uniform(-1e-3, 1e-3, 20_000),
                               rng.uniform(250.0, 4000.0, 20_000)]))
    _, lg = lbm.lbm_ff_check(x)
    ref = np.log(x)
    err = np.abs(lg - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < 2e-14, (err.max(), x[np.argmax(err)])


def test_ff_special_values():
    e, lg = lbm.lbm_ff_check(np.array([0.0, -200.0, 100.0, 1.0, -1.0]))
    assert e[0] == 1.0
    assert e[1] == 0.0
    assert np.isinf(e[2]) and e[2] > 0
    assert lg[3] == 0.0
    assert np.isnan(lg[4])


def test_ff_check_rejects_bad_arguments():
    L = lbm.load_library()
    x = np.zeros(4)
    assert L.lbm_ff_check(None, 4, x.ctypes.data, x.ctypes.data) == 1  # LBM_ERR_INVALID
    assert L.lbm_ff_check(x.ctypes.data, -1, x.ctypes.data, x.ctypes.data) == 1  # LBM_ERR_INVALID
    assert L.lbm_ff_check(x.ctypes.data, 1 << 25, x.ctypes.data, x.ctypes.data) == 6  # LBM_ERR_RANGE


def test_fp64_table_exp_error():
    """The FP64 rates' exp (Tang's method): within 2 ulp of numpy's exp over
    the range of ln k (and well beyond), exact at 0, the library's exp past
    |x| = 700."""
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(-700.0, 700.0, 200_000), rng.uniform(-1e-3, 1e-3, 20_000),
                        np.arange(-640, 641, dtype=np.float64) * np.log(2.0) / 64,
                        [0.0, 700.0, -700.0, 705.0, -720.0]])
    e = lbm.lbm_exp64_check(x)
    ref = np.exp(x)
    ulp = np.spacing(ref)
    assert np.max(np.abs(e - ref) / ulp) <= 2.0
    assert e[x == 0.0][0] == 1.0
