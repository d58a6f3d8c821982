"""The allocation-free entry point against the regular one.

wpcd_channel_solve_noalloc serves callers that cannot call cudaMalloc (an
application that owns all device memory through its own pool, or a loop that
cannot take cudaMalloc's implicit device synchronisation): it keeps every
intermediate in a fixed 16 MiB device array inside the library.  This test
calls it twice in a row through the C ABI -- a coupled channel, then an
uncoupled one with other samples, so the second call reuses the array the
first one left behind -- and checks each result against wpcd_solve on the same
channel, within the FP64 parity tolerances.  This file is collected last so
that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import TOL_DELTA_DEG, TOL_T, dphase

pytestmark = pytest.mark.gpu


def _one_channel(wl, c, n_samples, seed):
    ch = wl.channels[c]
    return W.Workload(f"{ch.name}", [ch], [wl.nwp[c]], wl.gen, wl.gen_params, wl.n_terms,
                      W.coefficient_samples(n_samples, seed), W.lab_energies(41, 1.0, 340.0))


def _check(ctx, lib, wl):
    import torch
    from paper_2106_00454_gb300 import _lib, api
    md = api.Model(ctx, wl)
    S, nE = wl.n_samples, len(wl.e_lab)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device="cuda:0")
    t_ref = torch.zeros((S, 1, nE, 2, 2, 2), dtype=torch.float64, device="cuda:0")
    d_ref = torch.zeros((S, 1, nE, 3), dtype=torch.float64, device="cuda:0")
    ctx.solve(md.vset, cf, S, e, t_ref, d_ref, None)
    ctx.sync()
    V = torch.tensor(ctx.vset_get(md.vset, 0), dtype=torch.float64, device="cuda:0")
    t = torch.full((S, 1, nE, 2, 2, 2), float("nan"), dtype=torch.float64, device="cuda:0")
    d = torch.full((S, 1, nE, 3), float("nan"), dtype=torch.float64, device="cuda:0")
    st = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    ch = wl.channels[0]
    stream = torch.cuda.current_stream(0)
    rc = lib.wpcd_channel_solve_noalloc(
        wl.nwp[0], wl.mesh_kind, wl.alpha, wl.t, wl.kmax, wl.Q, wl.wp_kind, _lib.wpcd_channel(*ch.astuple()),
        ctypes.c_void_p(V.data_ptr()), wl.n_terms, ctypes.c_void_p(cf.data_ptr()), S,
        ctypes.c_void_p(e.data_ptr()), nE, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(d.data_ptr()),
        ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    tr = t_ref.cpu().numpy().view(np.complex128)
    tn = t.cpu().numpy().view(np.complex128)
    scale = np.max(np.abs(tr))
    assert np.max(np.abs(tn - tr)) <= TOL_T * scale
    ncomp = 2 if ch.coupled else 1
    dr, dn = d_ref.cpu().numpy(), d.cpu().numpy()
    assert np.max(np.abs(dphase(dn[..., :ncomp], dr[..., :ncomp]))) <= TOL_DELTA_DEG
    assert np.max(np.abs(dn[..., 2] - dr[..., 2])) <= TOL_DELTA_DEG


def test_noalloc_matches_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00454_gb300 import _lib, api, build
    build.build()
    lib = _lib.load()
    ctx = api.Context(0)
    try:
        wl = W.workload_batched(n_samples=1)
        _check(ctx, lib, _one_channel(wl, 4, 6, W.SEED + 11))   # 3S1-3D1, coupled
        _check(ctx, lib, _one_channel(wl, 0, 9, W.SEED + 12))   # 1S0
    finally:
        ctx.close()


def test_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00454_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    p = ctypes.c_void_p(x.data_ptr())
    ch = _lib.wpcd_channel(1, 1, 0, 2, 1, 0)
    # 4096 samples of a 200 x 200 problem need ~1.3 GB of intermediates
    rc = lib.wpcd_channel_solve_noalloc(100, 0, W.MESH_ALPHA_FM, 2.0, 8.0, 8, 0, ch, p, 15, p, 4096, p, 8, p, p,
                                        None, None)
    assert rc == -1
