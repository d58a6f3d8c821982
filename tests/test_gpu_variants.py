"""Method variants on the GPU against the oracle: the midpoint approximation of
the projection (Sec. 3.2; the one-point rule per bin), the interpolation
point q_i = k_i + (n/m)(k_{i+1} - k_i) and its bands (Sec. 5.1.1), and the
accuracy studies of Secs. 5.2-5.3 (sigma_tot error map and RMSE) computed
element by element from the oracle's WPCD and MI on a small case."""
import dataclasses

import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import compare, compare_mixed, gpu_run, oracle_run

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


def _small(n_wp=40, jmax=3, n_e=37, n_samples=3):
    wl = W.workload_all_channels(n_wp=n_wp, jmax=jmax, n_e=n_e)
    return dataclasses.replace(wl, coeffs=W.coefficient_samples(n_samples))


@pytest.mark.parametrize("prec", [0, 1])
def test_midpoint_projection(ctx, orc, prec):
    """Projection with one point per bin (the midpoint approximation) on the
    GPU and in the oracle, then the whole path."""
    from paper_2106_00454_gb300 import api
    wl = dataclasses.replace(_small(), Q=1)
    md = api.Model(ctx, wl)
    gpu = gpu_run(ctx, md, wl, prec=prec)
    ora = oracle_run(orc, wl)
    if prec == 0:
        compare(wl, gpu, ora)
    else:
        compare_mixed(wl, gpu, ora)


@pytest.mark.parametrize("frac", [0.01, 0.3, 0.7, 0.99])
def test_interpolation_point(ctx, orc, frac):
    from paper_2106_00454_gb300 import api
    wl = _small(n_wp=48)
    md = api.Model(ctx, wl)
    ctx.set_interp_point(frac)
    try:
        gpu = gpu_run(ctx, md, wl, prec=0)
        gpu_mixed = gpu_run(ctx, md, wl, prec=1)
    finally:
        ctx.set_interp_point(0.5)
    meshes = [orc.Mesh(n) for n in wl.nwp]
    Vts = [orc.project_channel(m, ch.astuple(), wl.gen, wl.gen_params, wl.n_terms) for m, ch in
           zip(meshes, wl.channels)]
    t, d, s, rc = orc.batch([c.astuple() for c in wl.channels], meshes, Vts, wl.coeffs, wl.e_lab, frac=frac)
    assert rc == 0
    compare(wl, gpu, (t, d, s))
    compare_mixed(wl, gpu_mixed, (t, d, s))


def test_interpolation_point_reset_restores_midpoint_bit_for_bit(ctx):
    """Setting the point and back to 1/2 reproduces the default results exactly
    (the change also drops any CUDA graph that baked the old point in)."""
    import torch

    from paper_2106_00454_gb300 import api
    wl = _small(n_wp=32, jmax=2, n_e=20, n_samples=4)
    md = api.Model(ctx, wl)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device="cuda:0")
    d = torch.zeros((4, len(wl.channels), 20, 3), dtype=torch.float64, device="cuda:0")
    s = torch.zeros((4, 20), dtype=torch.float64, device="cuda:0")
    outs = []
    for f in (0.5, 0.5, 0.5, 0.2, 0.5):  # three calls: the third replays a graph; then change and back
        ctx.set_interp_point(f)
        ctx.solve(md.vset, cf, 4, e, None, d, s)
        ctx.sync()
        outs.append((d.cpu().numpy().copy(), s.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[4][0]) and np.array_equal(outs[0][1], outs[4][1])
    assert not np.array_equal(outs[0][1], outs[3][1])


def test_interpolation_point_rejects_outside_open_interval(ctx):
    from paper_2106_00454_gb300 import api
    for f in (0.0, 1.0, -0.1, 1.5, float("nan")):
        with pytest.raises(api.WpcdError):
            ctx.set_interp_point(f)


def test_bands_match_oracle(ctx, orc):
    """studies.interpolation_bands on Yamaguchi 1S0 (N_WP = 32) against the
    oracle's solves at the same points, band edges element by element."""
    from paper_2106_00454_gb300 import studies
    wl = W.workload_yamaguchi(n_wp=32, n_e=40)
    res = studies.interpolation_bands(ctx, wl)
    m = orc.Mesh(32)
    Vt = orc.project_channel(m, wl.channels[0].astuple(), wl.gen, wl.gen_params, 1)
    od = []
    for f in res["fracs"]:
        _, d, _, rc = orc.batch([wl.channels[0].astuple()], [m], [Vt], np.zeros((1, 1)), wl.e_lab, frac=f)
        assert rc == 0
        od.append(d)
    od = np.array(od)
    assert np.max(np.abs(res["delta"][..., 0] - od[..., 0])) < 1e-8
    assert np.max(np.abs(res["delta_lo"][..., 0] - od.min(axis=0)[..., 0])) < 1e-8
    assert np.max(np.abs(res["delta_hi"][..., 0] - od.max(axis=0)[..., 0])) < 1e-8


def test_studies_match_oracle(ctx, orc):
    """The sigma_tot error map and the RMSE study (Secs. 5.2-5.3) on J <= 2,
    N_WP in {12, 24}, 3 samples: every entry against the same quantity formed
    from the oracle's WPCD (batch) and MI (mi_batch at every energy, the
    exact reference; at 8 Chebyshev energies, interpolated)."""
    from paper_2106_00454_gb300 import studies
    wl = _small(n_wp=24, jmax=2, n_e=20)
    nwps = [12, 24]
    errs, ref = studies.sigma_error_map(ctx, wl, nwps)
    res = studies.rmse_study(ctx, wl, nwps, mi_interp_list=[8])
    chs = [c.astuple() for c in wl.channels]
    _, _, oref, rc = orc.mi_batch(chs, wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, wl.e_lab, wl.e_lab, NQ=96)
    assert rc == 0
    np.testing.assert_allclose(ref, oref, rtol=1e-8)
    sel = [(wl.e_lab > lo) & (wl.e_lab <= hi) for lo, hi in res["ranges"]]
    for k, nwp in enumerate(nwps):
        meshes = [orc.Mesh(nwp) for _ in wl.channels]
        Vts = [orc.project_channel(m, ch, wl.gen, wl.gen_params, wl.n_terms) for m, ch in zip(meshes, chs)]
        _, _, sw, rc = orc.batch(chs, meshes, Vts, wl.coeffs, wl.e_lab)
        assert rc == 0
        oerr = np.abs(sw - oref) / np.abs(oref)
        np.testing.assert_allclose(errs[k], oerr, rtol=1e-6, atol=1e-10)
        for r, m in enumerate(sel):
            ormse = np.sqrt(np.mean((sw[:, m] - oref[:, m])**2, axis=1))
            np.testing.assert_allclose(res["wpcd"][nwp][r], ormse, rtol=1e-6)
    _, _, smi, rc = orc.mi_batch(chs, wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, W.chebyshev_energies(8),
                                 wl.e_lab, NQ=96)
    assert rc == 0
    for r, m in enumerate(sel):
        ormse = np.sqrt(np.mean((smi[:, m] - oref[:, m])**2, axis=1))
        np.testing.assert_allclose(res["mi"][8][r], ormse, rtol=1e-6)
