"""The library's error metrics (Sec. 3.1.1: the L-inf error and
PSNR = 20 log10((max x - min x) / sqrt(MSE)), in FP64; host only): against
numpy on random data, exact values on a dyadic grid, the special cases
(identical arrays, a constant field, no values), the non-finite rules, and
the same result on every call (fixed chunked sums)."""
import math

import numpy as np
import pytest

from paper_2502_04093_gb300 import build, ipc


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 1000, (1 << 16) * 9 + 17])
def test_against_numpy(dtype, n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n).astype(dtype)
    y = (x + rng.uniform(-1e-3, 1e-3, size=n)).astype(dtype)
    m = ipc.ipc_error_metrics_host(x, y)
    d = x.astype(np.float64) - y.astype(np.float64)
    assert m["max_abs_err"] == np.abs(d).max()
    assert m["mse"] == pytest.approx(np.mean(d * d), rel=1e-12)
    r = float(x.max()) - float(x.min())
    assert m["range"] == r
    if n > 1:
        assert m["psnr"] == pytest.approx(20 * math.log10(r / math.sqrt(np.mean(d * d))), rel=1e-12)
    assert m["finite"] == n and m["nonfinite_mismatch"] == 0
    assert ipc.ipc_error_metrics_host(x, y) == m  # the same sums every time


def test_exact_on_a_dyadic_grid():
    x = (np.arange(4096, dtype=np.float64) / 8.0).reshape(64, 64)
    y = x + 0.25
    m = ipc.ipc_error_metrics_host(x, y)
    assert m["max_abs_err"] == 0.25 and m["mse"] == 0.0625 and m["range"] == 511.875
    assert m["psnr"] == 20 * math.log10(511.875 / 0.25)


def test_special_cases():
    x = np.linspace(-1, 1, 100, dtype=np.float32)
    m = ipc.ipc_error_metrics_host(x, x.copy())
    assert m["mse"] == 0 and m["max_abs_err"] == 0 and m["psnr"] == math.inf
    c = np.full(50, 3.0)
    m = ipc.ipc_error_metrics_host(c, c + 1e-3)
    assert m["range"] == 0 and m["psnr"] == -math.inf
    m = ipc.ipc_error_metrics_host(np.zeros(0, np.float32), np.zeros(0, np.float32))
    assert m["finite"] == 0 and m["mse"] == 0 and m["psnr"] == math.inf


def test_nonfinite_rules():
    x = np.array([1.0, np.nan, np.inf, -np.inf, 2.0, 5.0], dtype=np.float32)
    y = x.copy()
    m = ipc.ipc_error_metrics_host(x, y)
    assert m["finite"] == 3 and m["nonfinite_mismatch"] == 0 and m["range"] == 4.0
    y2 = np.array([1.0, 0.0, -np.inf, np.inf, 2.5, 5.0], dtype=np.float32)  # three classes differ
    m = ipc.ipc_error_metrics_host(x, y2)
    assert m["nonfinite_mismatch"] == 3 and m["max_abs_err"] == 0.5
    assert m["mse"] == pytest.approx(0.25 / 3)
    y3 = x.copy()
    y3[0] = np.nan  # a finite original read back as NaN
    m = ipc.ipc_error_metrics_host(x, y3)
    assert m["nonfinite_mismatch"] == 1 and m["max_abs_err"] == math.inf
    assert m["mse"] == 0.0  # the pair leaves the sums


def test_refused():
    with pytest.raises(ipc.IpcError):
        ipc.ipc_error_metrics_host(np.zeros(4, np.float32), np.zeros(4, np.float64))
    with pytest.raises(ipc.IpcError):
        ipc.ipc_error_metrics_host(np.zeros(4, np.int32), np.zeros(4, np.int32))
