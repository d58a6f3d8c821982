"""Parity of the resolvent variants with the FP64 oracle, through the C ABI.

* SWP-bin average (App. B as printed): uncoupled channels without bound
  states; a coupled channel is refused, a solve with a bound state gets NaN.
* Point resolvent: T and the phases at each requested energy, every channel.

FP64 tolerances as for the free-bin average (1e-10 of max |T| per channel,
1e-8 deg, 1e-8 relative sigma); the mixed path within 1e-3 deg and 0.01 mb.
"""
import dataclasses

import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import compare, compare_mixed, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

SWP_INDEX, POINT = 1, 2


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


def _model(ctx, wl):
    from paper_2106_00454_gb300 import api
    return api.Model(ctx, wl)


def _uncoupled_no_bound(S=12):
    """The uncoupled channels of the batched workload except the 1S0 pair
    (whose samples sometimes bind), N_WP from {24, 40, 64}."""
    wl = W.workload_batched(n_samples=S, n_e=48, nwp_choices=(24, 40, 64))
    keep = [k for k, ch in enumerate(wl.channels) if not ch.coupled and ch.l > 0]
    return dataclasses.replace(wl, name=wl.name + "_uncoupled", channels=[wl.channels[k] for k in keep],
                               nwp=[wl.nwp[k] for k in keep])


@pytest.mark.parametrize("via", ["solve", "handles"])
def test_swp_index_fp64(ctx, orc, via):
    wl = _uncoupled_no_bound()
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl, via=via, res=SWP_INDEX), oracle_run(orc, wl, mode=SWP_INDEX))


def test_swp_index_mixed(ctx, orc):
    wl = _uncoupled_no_bound()
    md = _model(ctx, wl)
    compare_mixed(wl, gpu_run(ctx, md, wl, prec=1, res=SWP_INDEX), oracle_run(orc, wl, mode=SWP_INDEX))


def test_swp_index_yamaguchi(ctx, orc):
    wl = W.workload_yamaguchi()
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl, res=SWP_INDEX), oracle_run(orc, wl, mode=SWP_INDEX))


def test_swp_index_refuses_coupled(ctx):
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=2, n_e=8, nwp_choices=(24,))
    md = _model(ctx, wl)
    with pytest.raises(api.WpcdError):
        gpu_run(ctx, md, wl, res=SWP_INDEX)


def test_swp_index_bound_state_is_nan(ctx, orc):
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=64, n_e=16, nwp_choices=(40,))
    ch = wl.channels[0]
    assert ch.name == "1S0"
    m = orc.Mesh(40)
    Vt = orc.project_channel(m, ch.astuple(), wl.gen, wl.gen_params, wl.n_terms)
    rcs = [orc.channel_solve(m, 1, Vt, wl.coeffs[k], mode=SWP_INDEX)[3] for k in range(64)]
    bad, good = rcs.index(-4), rcs.index(0)
    one = dataclasses.replace(wl, channels=[ch], nwp=[40], coeffs=wl.coeffs[[good, bad]])
    md = _model(ctx, one)
    with pytest.raises(api.WpcdError):
        gpu_run(ctx, md, one, res=SWP_INDEX)
    # the outputs of the failed call: the bound sample is NaN, the other one exact
    import torch
    e = torch.tensor(one.e_lab, dtype=torch.float64, device="cuda:0")
    cf = torch.tensor(one.coeffs, dtype=torch.float64, device="cuda:0")
    d = torch.zeros((2, 1, len(one.e_lab), 3), dtype=torch.float64, device="cuda:0")
    ctx.solve(md.vset, cf, 2, e, None, d, None, res=SWP_INDEX)
    assert ctx.sync_status() != 0
    d = d.cpu().numpy()
    assert np.all(np.isnan(d[1, 0, :, 0]))
    ref = oracle_run(orc, dataclasses.replace(one, coeffs=one.coeffs[:1]), mode=SWP_INDEX)[1]
    assert np.max(np.abs(d[0, 0, :, 0] - ref[0, 0, :, 0])) < 1e-8


@pytest.mark.parametrize("via", ["solve", "handles"])
def test_point_fp64_all_channels(ctx, orc, via):
    wl = W.workload_batched(n_samples=8, n_e=40, nwp_choices=(24, 40, 64))
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl, via=via, res=POINT), oracle_run(orc, wl, mode=POINT))


def test_point_mixed_all_channels(ctx, orc):
    wl = W.workload_batched(n_samples=8, n_e=40, nwp_choices=(24, 40, 64))
    md = _model(ctx, wl)
    compare_mixed(wl, gpu_run(ctx, md, wl, prec=1, res=POINT), oracle_run(orc, wl, mode=POINT))


def test_point_yamaguchi(ctx, orc):
    wl = W.workload_yamaguchi()
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl, res=POINT), oracle_run(orc, wl, mode=POINT))


def test_point_host_entry(ctx, orc):
    wl = W.workload_batched(n_samples=3, n_e=17, nwp_choices=(40,))
    md = _model(ctx, wl)
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    t = np.zeros((S, nch, nE, 2, 2, 2))
    d = np.zeros((S, nch, nE, 3))
    s = np.zeros((S, nE))
    ctx.solve_host(md.vset, wl.coeffs, S, wl.e_lab, t, d, s, res=POINT)
    tc = t.view(np.complex128).reshape(S, nch, nE, 2, 2)
    compare(wl, (tc, d, s), oracle_run(orc, wl, mode=POINT))
