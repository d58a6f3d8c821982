"""Parity of the GPU MI comparison method (Sec. 2.1 solves at Chebyshev
interpolation energies, Sec. 6 linear interpolation in T_lab) with the FP64
oracle, through the C ABI.

Tolerances as for the FP64 WPCD path: on-shell K within 1e-10 of the
channel's max |K|, phases within 1e-8 deg, sigma within 1e-8 relative."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import dphase

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


def _gpu(ctx, chs, gen, gp, n_terms, coeffs, e_int, e_lab, nq):
    import torch
    dev = "cuda:0"
    S = coeffs.shape[0]
    mid = ctx.mi_prepare(chs, gen, gp, n_terms, n_quad=nq)
    cf = torch.tensor(coeffs, dtype=torch.float64, device=dev) if n_terms > 1 else None
    ei = torch.tensor(e_int, dtype=torch.float64, device=dev)
    el = torch.tensor(e_lab, dtype=torch.float64, device=dev)
    k = torch.zeros((S, len(chs), len(e_int), 2, 2), dtype=torch.float64, device=dev)
    d = torch.zeros((S, len(chs), len(e_lab), 3), dtype=torch.float64, device=dev)
    s = torch.zeros((S, len(e_lab)), dtype=torch.float64, device=dev)
    ctx.mi_solve(mid, cf, S, ei, el, k, d, s)
    ctx.sync()
    ctx.release(mid)
    return k.cpu().numpy(), d.cpu().numpy(), s.cpu().numpy()


def _compare(chs, gpu, ora):
    gk, gd, gs = gpu
    ok, od, os_ = ora
    for c, ch in enumerate(chs):
        K = 2 if ch[4] else 1
        sc = np.max(np.abs(ok[:, c, :, :K, :K]))
        assert np.max(np.abs(gk[:, c, :, :K, :K] - ok[:, c, :, :K, :K])) <= 1e-10 * sc, c
        assert np.max(np.abs(dphase(gd[:, c, :, :K], od[:, c, :, :K]))) <= 1e-8, c
        if K == 2:
            assert np.max(np.abs(gd[:, c, :, 2] - od[:, c, :, 2])) <= 1e-8, c
    assert np.max(np.abs(gs - os_) / np.abs(os_)) <= 1e-8


@pytest.mark.parametrize("nq,n_I", [(48, 16), (96, 9)])
def test_mi_yamaguchi(ctx, orc, nq, n_I):
    chs = [(0, 0, 0, 0, 0, 0)]
    e_int = W.chebyshev_energies(n_I)
    e_lab = W.lab_energies(64)
    coeffs = np.zeros((1, 1))
    ora = orc.mi_batch(chs, W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1, coeffs, e_int, e_lab, NQ=nq)
    assert ora[3] == 0
    _compare(chs, _gpu(ctx, chs, W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1, coeffs, e_int, e_lab, nq), ora[:3])


def test_mi_yukawa_all_channels(ctx, orc):
    wl = W.workload_batched(n_samples=3, n_e=40)
    chs = [c.astuple() for c in wl.channels]
    e_int = W.chebyshev_energies(10)
    ora = orc.mi_batch(chs, wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, e_int, wl.e_lab, NQ=96)
    assert ora[3] == 0
    _compare(chs, _gpu(ctx, chs, wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, e_int, wl.e_lab, 96), ora[:3])


def test_mi_close_to_wpcd(ctx, orc):
    # two methods, one problem: MI (N_Q = 96, 32 interpolation energies) and
    # WPCD (N_WP = 100) on the same synthetic potential agree to the method
    # error of WPCD at this N_WP (a band, not parity)
    wl = W.workload_batched(n_samples=2, n_e=32, nwp_choices=(100,))
    chs = [c.astuple() for c in wl.channels]
    mi = _gpu(ctx, chs, wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, W.chebyshev_energies(32), wl.e_lab, 96)
    from paper_2106_00454_gb300 import api
    from parity_util import gpu_run
    md = api.Model(ctx, wl)
    _, dw, sw = gpu_run(ctx, md, wl)
    sel = wl.e_lab > 5.0
    assert np.max(np.abs(dphase(mi[1][:, :, sel, :2], dw[:, :, sel, :2]))) < 3.0
    assert np.max(np.abs(mi[2][:, sel] - sw[:, sel]) / sw[:, sel]) < 0.05


def test_mi_refuses_bad_arguments(ctx):
    from paper_2106_00454_gb300 import api
    with pytest.raises(api.WpcdError):
        ctx.mi_prepare([(0, 0, 0, 0, 0, 0)], W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1, n_quad=101)
    with pytest.raises(api.WpcdError):
        ctx.mi_prepare([(1, 1, 0, 2, 1, 0)], W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1)
