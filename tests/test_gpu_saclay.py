"""Parity of the GPU spin observables (App. A: M-matrix, Saclay amplitudes,
dsigma/dOmega) with the oracle, on phases from a GPU WPCD solve; and the
optical theorem against the GPU's own sigma_tot."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import gpu_run

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


def test_saclay_matches_oracle_and_optical_theorem(ctx, orc):
    import torch
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=3, n_e=12, nwp_choices=(40, 64))
    md = api.Model(ctx, wl)
    _, d, s = gpu_run(ctx, md, wl)
    S, nch, nE = d.shape[0], d.shape[1], d.shape[2]
    theta = np.linspace(0.0, np.pi, 19)
    dev = "cuda:0"
    dd = torch.tensor(d, device=dev)
    el = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    ab = torch.zeros((S, nE, len(theta), 5, 2), dtype=torch.float64, device=dev)
    ds = torch.zeros((S, nE, len(theta)), dtype=torch.float64, device=dev)
    ctx.saclay(wl.channels, dd, S, el, th, ab, ds)
    ab = ab.cpu().numpy().view(np.complex128).reshape(S, nE, len(theta), 5)
    ds = ds.cpu().numpy()
    chs = [c.astuple() for c in wl.channels]
    for smp in range(S):
        for e in range(nE):
            p = orc.p_of_tlab(wl.e_lab[e])[0]
            oab, ods = orc.saclay(chs, d[smp, :, e, :], p, theta)
            sc = np.max(np.abs(oab))
            assert np.max(np.abs(ab[smp, e] - oab)) <= 1e-12 * sc, (smp, e)
            np.testing.assert_allclose(ds[smp, e], ods, rtol=1e-12)
            # optical theorem against the path's own sigma_tot
            opt = 2 * np.pi / p * (ab[smp, e, 0, 0] + ab[smp, e, 0, 1]).imag * 10
            assert abs(opt - s[smp, e]) <= 1e-10 * s[smp, e], (smp, e)
