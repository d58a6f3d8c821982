"""The resolvent kernel's table-driven logarithm against the host's log (numpy,
glibc) and CUDA's log (torch.log on the device): at most 2 ulp apart over
arguments spread across the double range, around 1 (where the result is
small), at every table point and its midpoints, and at the folded top of each
binade; special arguments match the library exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00454_gb300 import api, build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _args():
    rng = np.random.default_rng(20210601)
    parts = [
        np.exp(rng.uniform(-700, 700, 200000)),                  # across the normal range
        1.0 + rng.uniform(-0.02, 0.02, 100000),                  # near 1: small results
        1.0 + np.ldexp(rng.uniform(-1, 1, 20000), -40),          # very near 1
        np.ldexp(1.0 + np.arange(257) / 256.0, 0),               # table points
        np.ldexp(1.0 + (np.arange(256) + 0.5) / 256.0, 3),       # rounding midpoints of j
        np.nextafter(2.0, 0.0) * np.ldexp(1.0, np.arange(-20, 20)),  # just below powers of two
        np.ldexp(1.0, np.arange(-1020, 1020, 7)),                # powers of two
        rng.uniform(1e-3, 20.0, 100000),                         # energy differences in fm^-1
    ]
    return np.concatenate(parts)


def _ulps(a, b):
    """|a - b| in units of the last place of b (b finite, nonzero)."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_device_log_accuracy(ctx):
    import torch
    x = _args()
    xd = torch.tensor(x, device="cuda:0")
    yd = torch.empty_like(xd)
    ctx.device_log(xd, yd)
    ctx.sync()
    y = yd.cpu().numpy()
    host = np.log(x)
    cuda = torch.log(xd).cpu().numpy()
    ok = host != 0.0
    assert np.all(y[~ok] == 0.0)
    assert float(np.max(_ulps(y[ok], host[ok]))) <= 2.0
    assert float(np.max(_ulps(y[ok], cuda[ok]))) <= 2.0


def test_device_log_special(ctx):
    import torch
    x = np.array([0.0, 5e-324, 1e-310, np.inf, np.nan, -1.0, 1.0, 2.0, 0.5])
    xd = torch.tensor(x, device="cuda:0")
    yd = torch.empty_like(xd)
    ctx.device_log(xd, yd)
    ctx.sync()
    y = yd.cpu().numpy()
    ref = torch.log(xd).cpu().numpy()
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    inf = np.isinf(ref)
    assert np.array_equal(y[inf], ref[inf])
    fin = np.isfinite(ref)
    assert np.all((y[fin] == ref[fin]) | (_ulps(y[fin], ref[fin]) <= 1.0))
    assert y[6] == 0.0 and y[7] == np.log(2.0) and y[8] == -np.log(2.0)
