"""The logarithm of the FP64 lubrication term (tlog.cuh, Tang's table-driven
method) against high-precision values: below one unit in the last place plus
2^-60 everywhere the lubrication term calls it (x = <d>/2h between 1/2 and
<d>/2h_min) and beyond; the host build is the same source as the device
path (the GPU test checks the two agree bit for bit)."""
import numpy as np
import pytest

from paper_1711_00336_gb300 import dps


def _points():
    rng = np.random.default_rng(1)
    j = np.arange(129)
    table = 1.0 + j / 128.0
    ties = 1.0 + (2 * np.arange(128) + 1) / 256.0  # halfway between table points
    return np.concatenate([
        np.exp(rng.uniform(np.log(0.5), np.log(2e5), 20000)),
        1.0 + rng.uniform(-1e-3, 1e-3, 2000),
        table, np.nextafter(table, 0), np.nextafter(table, 3), ties, np.nextafter(ties, 0), np.nextafter(ties, 3),
        table * 2.0 ** rng.integers(-30, 30, 129),
        2.0 ** np.arange(-1022, 1024, 37).astype(np.float64), [1.0 + 2 ** -52, 1 - 2 ** -53, np.finfo(np.float64).max, 2.0 ** -1022]])


def test_tlog_within_one_ulp_of_the_exact_logarithm():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x = _points()
    y, _ = dps.check_tlog(x)
    ref = np.array([float(mp.log(mp.mpf(float(v)))) for v in x])
    err = np.abs(y - ref)
    assert np.all(err <= np.spacing(np.abs(ref)) + 2.0 ** -60)
    assert np.mean(y == ref) > 0.99  # nearly always the correctly rounded value


def test_tlog_special_arguments_take_the_library_log():
    x = np.array([0.0, -1.0, np.inf, np.nan, 2.0 ** -1060, 1.0])
    y, yl = dps.check_tlog(x)
    assert np.array_equal(y[:5], yl[:5], equal_nan=True)
    assert y[5] == 0.0


@pytest.mark.gpu
def test_tlog_device_equals_host_and_stays_near_the_cuda_log():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = _points()
    yh, _ = dps.check_tlog(x)
    yd, yl = dps.check_tlog(x, device=True)
    assert np.array_equal(yd, yh)
    assert np.all(np.abs(yd - yl) <= 2 * np.spacing(np.abs(yl)))
