"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path tolerances: |dT| <= 1e-10 max_E |T_ch| per channel, |d delta| and
|d eps_J| <= 1e-8 deg, |d sigma| <= 1e-8 relative."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import compare, dphase, gpu_run, oracle_run

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


def _model(ctx, wl):
    from paper_2106_00454_gb300 import api
    return api.Model(ctx, wl)


# ------------------------------------------------------------------------------------- mesh
@pytest.mark.parametrize("N,kind", [(32, 0), (37, 0), (100, 0), (16, 1)])
def test_mesh_matches_oracle(ctx, orc, N, kind):
    mid = ctx.mesh(N, kind=kind)
    kb, kq, wq = ctx.mesh_get(mid, N, 8)
    m = orc.Mesh(N, kind=kind)
    assert np.allclose(kb, m.kb, rtol=1e-14, atol=0)
    assert np.allclose(kq, m.kq, rtol=1e-14, atol=0)
    assert np.allclose(wq, m.wq, rtol=1e-13, atol=0)
    ctx.release(mid)


# ------------------------------------------------------------------------------------- projection
def test_projection_yamaguchi(ctx, orc):
    wl = W.workload_yamaguchi()
    md = _model(ctx, wl)
    V = ctx.vset_get(md.vset, 0)
    Vo = orc.project_channel(orc.Mesh(32), wl.channels[0].astuple(), wl.gen, wl.gen_params, 1)
    assert np.max(np.abs(V - Vo)) <= 1e-13 * np.max(np.abs(Vo))


@pytest.mark.parametrize("N", [12, 33])
def test_projection_yukawa_all_terms(ctx, orc, N):
    wl = W.workload_all_channels(n_wp=N, jmax=6)
    md = _model(ctx, wl)
    m = orc.Mesh(N)
    for c, ch in enumerate(wl.channels):
        V = ctx.vset_get(md.vset, c)
        Vo = orc.project_channel(m, ch.astuple(), wl.gen, wl.gen_params, wl.n_terms)
        for t in range(wl.n_terms):
            sc = max(np.max(np.abs(Vo[t])), 1e-300)
            assert np.max(np.abs(V[t] - Vo[t])) <= 1e-12 * sc, (ch.name, t)
            assert np.array_equal(V[t], V[t].T)


def test_projection_fine_grid_input(ctx, orc):
    torch = pytest.importorskip("torch")
    # caller-supplied fine values: the Yamaguchi form on the fine grid of one channel
    N, Q = 10, 8
    wl = W.workload_yamaguchi(n_wp=N)
    m = orc.Mesh(N)
    lam, beta = W.YAMAGUCHI_PARAMS
    g = 1.0 / (m.kq**2 + beta**2)
    vf = torch.tensor(lam * np.outer(g, g), dtype=torch.float64, device="cuda:0")
    mid = ctx.mesh(N)
    vid = ctx.project([mid], wl.channels, -1, None, 1, vf)
    V = ctx.vset_get(vid, 0)
    Vo = orc.project_channel(m, wl.channels[0].astuple(), wl.gen, wl.gen_params, 1)
    assert np.max(np.abs(V - Vo)) <= 1e-13 * np.max(np.abs(Vo))


# ------------------------------------------------------------------------------------- eigen
@pytest.mark.parametrize("N,ci", [(24, 0), (37, 4), (64, 4), (100, 4)])
def test_eigenpairs(ctx, orc, N, ci):
    torch = pytest.importorskip("torch")
    wl = W.workload_batched(n_samples=3)
    chs = [wl.channels[ci]]
    wl2 = W.Workload("eig", chs, [N], wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, wl.e_lab)
    md = _model(ctx, wl2)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    eid = ctx.diag(md.vset, cf, 3)
    st = torch.zeros((3, 1), dtype=torch.int32, device="cuda:0")
    ctx.diag_status(eid, st)
    ctx.sync()
    assert (st.cpu().numpy() > 0).all()
    Vt = orc.project_channel(orc.Mesh(N), chs[0].astuple(), wl.gen, wl.gen_params, wl.n_terms)
    m = orc.Mesh(N)
    K = chs[0].K
    h0 = np.array([orc.h0(0, m.kb[i], m.kb[i + 1]) for i in range(N)])
    for s in range(3):
        H = Vt[0] + np.tensordot(wl.coeffs[s], Vt[1:], 1) + np.diag(np.tile(h0, K))
        n = H.shape[0]
        eps, C = ctx.eig_get(eid, s, 0, n)
        nh = np.linalg.norm(H)
        u = np.finfo(float).eps
        assert np.all(np.diff(eps) >= 0)
        assert np.max(np.abs(eps - np.linalg.eigvalsh(H))) <= 20 * n * u * nh
        assert np.linalg.norm(H @ C - C * eps) <= 20 * n * u * nh
        assert np.linalg.norm(C.T @ C - np.eye(n)) <= 20 * n * u
    ctx.release(eid)


# ------------------------------------------------------------------------------------- end to end
def test_yamaguchi_workload(ctx, orc):
    """Workload 1 in full: 1S0 Yamaguchi, N_WP = 32, 64 energies."""
    wl = W.workload_yamaguchi()
    md = _model(ctx, wl)
    gpu = gpu_run(ctx, md, wl)
    ora = oracle_run(orc, wl)
    compare(wl, gpu, ora)
    gpu2 = gpu_run(ctx, md, wl, via="handles")
    for a, b in zip(gpu, gpu2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("N", [13, 40])
def test_all_channels_small(ctx, orc, N):
    """All 20 channels J <= 6 at a reduced N_WP (odd N gives a ragged tail)."""
    wl = W.workload_all_channels(n_wp=N, jmax=6, n_e=37)
    wl.e_lab = np.linspace(2.0, 300.0, 37)
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl), oracle_run(orc, wl))


def test_all_channels_workload(ctx, orc):
    """Workload 2 in full: 20 channels J <= 6, N_WP = 100 (coupled 200x200)."""
    wl = W.workload_all_channels()
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl), oracle_run(orc, wl))


def test_batched_small(ctx, orc):
    """Workload 3's generator with 6 samples: 15 channels, N_WP in {40,64,100}."""
    wl = W.workload_batched(n_samples=6)
    md = _model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl), oracle_run(orc, wl))


def test_plain_and_batched_modes_agree(ctx):
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=3)
    md = _model(ctx, wl)
    a = gpu_run(ctx, md, wl)
    ctx.set_exec(api.EXEC_PLAIN)
    try:
        b = gpu_run(ctx, md, wl)
    finally:
        ctx.set_exec(api.EXEC_BATCHED)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_host_entry_point_matches_device(ctx):
    wl = W.workload_batched(n_samples=4)
    md = _model(ctx, wl)
    gt, gd, gs = gpu_run(ctx, md, wl)
    S, nch, nE = 4, len(wl.channels), len(wl.e_lab)
    t = np.zeros((S, nch, nE, 2, 2, 2))
    d = np.zeros((S, nch, nE, 3))
    s = np.zeros((S, nE))
    ctx.solve_host(md.vset, wl.coeffs, S, wl.e_lab, t, d, s)
    assert np.array_equal(t.view(np.complex128).reshape(gt.shape), gt)
    assert np.array_equal(d, gd) and np.array_equal(s, gs)


# ------------------------------------------------------------------------------------- edges
def test_single_energy_and_bin_edges(ctx, orc):
    wl = W.workload_yamaguchi(n_wp=16)
    m = orc.Mesh(16)
    # energies exactly on a midpoint and just inside the mesh ends
    p_mid = m.kbar[5]
    t_mid = 2 * (p_mid * 197.3269804) ** 2 / 938.918309
    for e in [np.array([t_mid]), np.array([0.01]), np.array([1.0, t_mid, 300.0])]:
        wl.e_lab = e
        md = _model(ctx, wl)
        compare(wl, gpu_run(ctx, md, wl), oracle_run(orc, wl))


def test_energy_outside_mesh_is_reported(ctx):
    torch = pytest.importorskip("torch")
    from paper_2106_00454_gb300 import api
    wl = W.workload_yamaguchi(n_wp=16)
    md = _model(ctx, wl)
    e = torch.tensor([10.0, 10000.0], dtype=torch.float64, device="cuda:0")  # p(10 GeV) = 11 fm^-1 > 8
    s = torch.zeros((1, 2), dtype=torch.float64, device="cuda:0")
    ctx.solve(md.vset, None, 1, e, None, None, s)
    assert ctx.sync_status() == -1
    assert ctx.sync_status() == 0  # the status word clears


def test_budget_refusal(ctx):
    from paper_2106_00454_gb300 import api
    small = api.Context(0, hbm_budget_bytes=4096)
    with pytest.raises(api.WpcdError) as ei:
        small.mesh(512)
    assert ei.value.code == -3
    small.close()


def test_batched_full_size_sampled(ctx, orc):
    """Workload 3 at full size (4096 samples, the launch the benchmark times):
    sampled samples checked against the oracle one by one."""
    wl = W.workload_batched()
    md = _model(ctx, wl)
    gpu = gpu_run(ctx, md, wl)
    pick = [0, 1777, 4095]
    ora = oracle_run(orc, wl, samples=pick)
    compare(wl, gpu, ora, sample_idx=pick)
    assert np.all(np.isfinite(gpu[2]))


def test_autotune_table_and_results(ctx):
    """The autotuner records a CTA size per (n, precision) and the results stay
    within the FP64 tolerances of the fixed 256-thread launch."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=40)
    md = _model(ctx, wl)
    ctx.set_autotune(False)
    a = gpu_run(ctx, md, wl)
    ctx.set_autotune(True)
    b = gpu_run(ctx, md, wl)
    table = ctx.tuning()
    ns = {2 * n if ch.coupled else n for n, ch in zip(wl.nwp, wl.channels)}
    assert {e["n"] for e in table if e["precision"] == "fp64"} >= ns
    assert all(e["threads"] in (64, 128, 256, 512) for e in table)
    for c in range(len(wl.channels)):
        sc = np.max(np.abs(a[0][:, c]))
        assert np.max(np.abs(a[0][:, c] - b[0][:, c])) <= 1e-11 * sc
    assert np.max(np.abs(dphase(a[1], b[1]))) <= 1e-9
