"""Matrices above one CTA's shared memory (the global-memory Jacobi kernel):
FP64 path against the oracle at the FP64 tolerances, mixed path at 1e-3 deg /
0.01 mb, for coupled channels at N_WP = 150 (300 x 300) and N_WP = 256
(512 x 512), odd sizes (phantom row), one solve per launch, and the CUDA-graph
replay of a batch that holds such a bucket."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import compare, compare_mixed, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
FP64, MIXED = 0, 1


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


def _wl(n_wp, chans, n_samples, n_e=48):
    """The synthetic Yukawa/contact generator on the given channels, n_samples samples."""
    return W.Workload(f"large_nwp{n_wp}", list(chans), [n_wp] * len(chans), W.GEN_YUKAWA, W.YUKAWA_PARAMS.copy(),
                      W.N_TERMS_YUKAWA, W.coefficient_samples(n_samples), W.lab_energies(n_e))


J6 = W.np_channels(6)
COUPLED = [ch for ch in J6 if ch.coupled]


def test_fp64_nwp150_coupled(ctx, orc):
    """The 6 coupled channels J <= 6 plus 1S0 at N_WP = 150: 300 x 300 blocks in FP64."""
    from paper_2106_00454_gb300 import api
    wl = _wl(150, [J6[0]] + COUPLED, 2)
    md = api.Model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl, prec=FP64), oracle_run(orc, wl))


def test_fp64_nwp256(ctx, orc):
    """N_WP = 256: 1S0 (256 x 256) and 3S1-3D1 (512 x 512, bound state) in FP64."""
    from paper_2106_00454_gb300 import api
    wl = _wl(256, [J6[0], J6[4]], 1)
    md = api.Model(ctx, wl)
    compare(wl, gpu_run(ctx, md, wl, prec=FP64), oracle_run(orc, wl))


def test_mixed_nwp256(ctx, orc):
    """N_WP = 256 on the mixed path: 3S1-3D1 and 3P2-3F2 (512 x 512, FP32 Jacobi in
    global memory + FP64 refinement), 1S0 (256 x 256, shared-memory kernel)."""
    from paper_2106_00454_gb300 import api
    wl = _wl(256, [J6[0], J6[4], J6[7]], 2)
    md = api.Model(ctx, wl)
    compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl))


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_odd_size_phantom(ctx, orc, prec):
    """Odd n above the shared-memory limit of each precision (FP64: 241, mixed:
    335): the kernel pairs the last index with a zero phantom row."""
    from paper_2106_00454_gb300 import api
    n_wp = 241 if prec == FP64 else 335
    wl = _wl(n_wp, [J6[0], J6[2]], 2, n_e=33)
    md = api.Model(ctx, wl)
    gpu = gpu_run(ctx, md, wl, prec=prec)
    ora = oracle_run(orc, wl)
    if prec == FP64:
        compare(wl, gpu, ora)
    else:
        compare_mixed(wl, gpu, ora)


def test_plain_one_solve_per_launch(ctx, orc):
    """Plain execution (one eigensolve per launch) through the large kernel."""
    from paper_2106_00454_gb300 import api
    wl = _wl(150, [J6[4]], 1, n_e=24)
    md = api.Model(ctx, wl)
    ctx.set_exec(api.EXEC_PLAIN)
    try:
        gpu = gpu_run(ctx, md, wl, prec=FP64)
    finally:
        ctx.set_exec(api.EXEC_BATCHED)
    compare(wl, gpu, oracle_run(orc, wl))


def test_batched_graph_replay_matches(ctx):
    """Repeated batched solves of a set with a 300 x 300 bucket replay a CUDA
    graph and reproduce the first call bit for bit, in both precisions."""
    import torch

    from paper_2106_00454_gb300 import api
    wl = _wl(150, [J6[0], J6[4]], 8, n_e=16)
    md = api.Model(ctx, wl)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device="cuda:0")
    # the same output buffers every call: a graph is keyed on its pointers
    d = torch.zeros((8, 2, 16, 3), dtype=torch.float64, device="cuda:0")
    s = torch.zeros((8, 16), dtype=torch.float64, device="cuda:0")
    for prec in (FP64, MIXED):
        outs = []
        g0 = ctx.graph_stats()
        for _ in range(3):
            d.zero_()
            s.zero_()
            ctx.solve(md.vset, cf, 8, e, None, d, s, prec=prec)
            ctx.sync()
            outs.append((d.cpu().numpy(), s.cpu().numpy()))
        g1 = ctx.graph_stats()
        assert g1["replays"] > g0["replays"]
        for dd, ss in outs[1:]:
            assert np.array_equal(dd, outs[0][0]) and np.array_equal(ss, outs[0][1])


def test_sweep_status(ctx):
    """Every large solve reports its sweep count (converged) in the per-solve status."""
    import torch

    from paper_2106_00454_gb300 import api
    wl = _wl(256, [J6[4]], 3, n_e=8)
    md = api.Model(ctx, wl)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    for prec in (FP64, MIXED):
        eid = ctx.diag(md.vset, cf, 3, prec=prec)
        st = torch.zeros((3, 1), dtype=torch.int32, device="cuda:0")
        ctx.diag_status(eid, st)
        ctx.sync()
        sw = st.cpu().numpy()
        ctx.release(eid)
        assert (sw > 0).all() and (sw < 40).all(), sw
