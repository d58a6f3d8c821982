"""CUDA-graph replay of wpcd_solve: bit-identical to kernel-by-kernel launches,
inputs read when the graph runs (not when it was captured), the same kernel
count, and graphs dropped when an option or a workspace changes."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00454_gb300 import api, build
    build.build()
    c = api.Context(0)
    ref = api.Context(0)
    # fixed CTA sizes on both sides, so that both launch exactly the same kernels
    c.set_autotune(False)
    ref.set_autotune(False)
    ref.set_graphs(False)
    wl = W.workload_batched(n_samples=24, n_e=40)
    yield torch, api, c, ref, wl, api.Model(c, wl), api.Model(ref, wl)
    c.close()
    ref.close()


def _bufs(torch, wl):
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    f = dict(dtype=torch.float64, device=DEV)
    return (torch.tensor(wl.coeffs, **f), torch.tensor(wl.e_lab, **f), torch.zeros((S, nch, nE, 2, 2, 2), **f),
            torch.zeros((S, nch, nE, 3), **f), torch.zeros((S, nE), **f))


def _solve(ctx, md, wl, b, prec):
    cf, e, t, d, s = b
    for x in (t, d, s):
        x.fill_(np.nan)  # every output must be written by this call
    ctx.solve(md.vset, cf, wl.n_samples, e, t, d, s, prec=prec)
    ctx.sync()


def _same(a, b):
    import torch
    return all(torch.equal(x, y) for x, y in zip(a[2:], b[2:]))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_replay_matches_eager(env, prec):
    torch, api, c, ref, wl, md, mr = env
    b, rb = _bufs(torch, wl), _bufs(torch, wl)
    base = b[0].clone()
    g0 = c.graph_stats()
    counts = []
    for it in range(4):
        # new parameters each call, written into the same buffer the graph reads
        b[0].copy_(base.roll(it, 0))
        rb[0].copy_(b[0])
        l0 = c.kernel_launches()
        _solve(c, md, wl, b, prec)
        counts.append(c.kernel_launches() - l0)
        _solve(ref, mr, wl, rb, prec)
        assert _same(b, rb), f"call {it}"
        assert torch.isfinite(b[3]).all() and torch.isfinite(b[4]).all()
    g1 = c.graph_stats()
    # call 0 one by one, call 1 captures and launches, calls 2-3 replay
    assert g1["captures"] - g0["captures"] == 1
    assert g1["replays"] - g0["replays"] == 3
    assert len(set(counts)) == 1 and counts[0] > 0, counts


def test_option_change_drops_graph(env):
    torch, api, c, ref, wl, md, mr = env
    b, rb = _bufs(torch, wl), _bufs(torch, wl)
    for _ in range(2):
        _solve(c, md, wl, b, 1)
    g0 = c.graph_stats()
    c.set_refine_engine(api.REFINE_TENSOR)  # same value: still invalidates every graph
    _solve(c, md, wl, b, 1)
    g1 = c.graph_stats()
    assert g1["replays"] == g0["replays"] and g1["captures"] == g0["captures"]
    _solve(c, md, wl, b, 1)
    g2 = c.graph_stats()
    assert g2["captures"] == g1["captures"] + 1 and g2["replays"] == g1["replays"] + 1
    _solve(ref, mr, wl, rb, 1)
    assert _same(b, rb)


def test_workspace_growth_drops_graph(env):
    torch, api, c, ref, wl, md, mr = env
    b, rb = _bufs(torch, wl), _bufs(torch, wl)
    for _ in range(3):
        _solve(c, md, wl, b, 1)
    g0 = c.graph_stats()
    # a larger batch grows the eigenpair storage and the workspaces
    big = W.workload_batched(n_samples=2 * wl.n_samples, n_e=len(wl.e_lab) + 8)
    bb = _bufs(torch, big)
    c.solve(md.vset, bb[0], big.n_samples, bb[1], bb[2], bb[3], bb[4], prec=1)
    c.sync()
    _solve(c, md, wl, b, 1)
    g1 = c.graph_stats()
    assert g1["replays"] == g0["replays"], "a graph with stale workspace pointers was launched"
    _solve(ref, mr, wl, rb, 1)
    assert _same(b, rb)


def test_solve_host_replays(env):
    torch, api, c, ref, wl, md, mr = env
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)

    def run(ctx, m):
        t = np.full((S, nch, nE, 2, 2, 2), np.nan)
        d = np.full((S, nch, nE, 3), np.nan)
        s = np.full((S, nE), np.nan)
        ctx.solve_host(m.vset, wl.coeffs, S, wl.e_lab, t, d, s, prec=1)
        return t, d, s

    g0 = c.graph_stats()
    outs = [run(c, md) for _ in range(3)]
    g1 = c.graph_stats()
    assert g1["captures"] - g0["captures"] == 1 and g1["replays"] - g0["replays"] == 2
    r = run(ref, mr)
    for o in outs:
        for x, y in zip(o, r):
            assert np.array_equal(x, y, equal_nan=False)


def test_profiling_and_plain_bypass_graphs(env):
    torch, api, c, ref, wl, md, mr = env
    b = _bufs(torch, wl)
    g0 = c.graph_stats()
    c.profile(True)
    try:
        for _ in range(3):
            _solve(c, md, wl, b, 1)
    finally:
        c.profile(False)
    assert c.graph_stats()["captures"] == g0["captures"]
    small = W.workload_batched(n_samples=2, n_e=8)
    sb = _bufs(torch, small)
    c.set_exec(api.EXEC_PLAIN)
    try:
        for _ in range(3):
            _solve(c, md, small, sb, 0)
    finally:
        c.set_exec(api.EXEC_BATCHED)
    assert c.graph_stats()["captures"] == g0["captures"]
