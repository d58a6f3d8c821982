"""The accuracy studies (WPCD against the exact MI result, Sec. 5) through the
public API: the sigma_tot error falls as N_WP grows, and MI with linear
interpolation converges to the exact result as the interpolation energies
multiply."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

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


def _wl():
    wl = W.workload_all_channels(n_wp=16, jmax=4, n_e=70)
    return wl


def test_rmse_falls_with_nwp(ctx):
    from paper_2106_00454_gb300 import studies
    res = studies.rmse_study(ctx, _wl(), [16, 32, 64], mi_interp_list=[8, 32])
    for r in range(2):  # (0, 350] and (40, 350]
        w = [res["wpcd"][n][r][0] for n in (16, 32, 64)]
        assert w[0] > w[1] > w[2], (r, w)
        m = [res["mi"][n][r][0] for n in (8, 32)]
        assert m[0] > m[1], (r, m)
    # doubling N_WP twice cuts the 40..350 MeV RMSE by more than a third
    # (measured on GB300: 2.2 mb at N_WP = 64 for this synthetic potential)
    w = [res["wpcd"][n][1][0] for n in (16, 32, 64)]
    assert w[2] < 0.65 * w[0] and w[2] < 5.0, w


def test_error_map_shape_and_trend(ctx):
    from paper_2106_00454_gb300 import studies
    errs, ref = studies.sigma_error_map(ctx, _wl(), [16, 64])
    assert errs.shape == (2, 1, 70) and ref.shape == (1, 70)
    assert np.all(ref > 0)
    assert np.median(errs[1]) < np.median(errs[0])
