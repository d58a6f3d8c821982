"""Serving with continuous batching: each request's result is the same alone
and in the mix, matches the oracle, and admission / timeouts / unknown
tickets are reported as the C ABI documents."""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import TOL_DELTA_DEG, TOL_SIGMA_REL, TOL_T, dphase

pytestmark = pytest.mark.gpu
CHANNELS = W.np_channels(4, extra_1s0_tz=True)


def _ctx(**kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_00454_gb300 import api, build
    build.build()
    return api.Context(0, **kw)


@pytest.fixture(scope="module")
def server():
    c = _ctx()
    c.serve_start(CHANNELS, W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA, [32, 64], max_batch=32, n_slots=3)
    yield c
    c.serve_stop()
    c.close()


def _req(seed, n_wp):
    rng = np.random.default_rng(seed)
    n_e = int(rng.integers(16, 65))
    return rng.standard_normal(14) * W.TERM_SCALE, np.sort(rng.uniform(1.0, 350.0, n_e)), n_wp


def _same(a, b):
    assert np.array_equal(a.delta, b.delta) and np.array_equal(a.sigma, b.sigma) and np.array_equal(a.T, b.T)


@pytest.mark.parametrize("prec", [0, 1])
def test_same_alone_and_in_the_mix(server, prec):
    c0, e0, nw0 = _req(1, 64)
    t = server.submit(c0, e0, nw0, prec)
    alone = server.wait(t)
    assert alone.status == 0
    # a burst of other requests (both N_WP, both precisions) with the same request in the middle
    tickets = [server.submit(*_req(100 + k, (32, 64)[k % 2]), (0, 1)[(k // 2) % 2]) for k in range(40)]
    tm = server.submit(c0, e0, nw0, prec)
    tickets += [server.submit(*_req(200 + k, (32, 64)[k % 2]), prec) for k in range(40)]
    mixed = server.wait(tm)
    for tk in tickets:
        r = server.wait(tk)
        assert r.status == 0
        server.release_result(tk)
    _same(alone, mixed)
    st = server.serve_stats()
    assert st["completed"] >= 82 and st["batches"] < st["completed"]  # requests were batched


def test_served_request_matches_oracle(server, orc):
    coeffs, e_lab, n_wp = _req(7, 32)
    r = server.wait(server.submit(coeffs, e_lab, n_wp, 0))
    meshes = [orc.Mesh(n_wp) for _ in CHANNELS]
    Vts = [orc.project_channel(m, ch.astuple(), W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA)
           for m, ch in zip(meshes, CHANNELS)]
    ot, od, os_, rc = orc.batch([c.astuple() for c in CHANNELS], meshes, Vts, coeffs[None], e_lab)
    assert rc == 0
    for c, ch in enumerate(CHANNELS):
        scale = np.max(np.abs(ot[0, c]))
        assert np.max(np.abs(r.T[c] - ot[0, c])) <= TOL_T * scale
        k = 2 if ch.coupled else 1
        assert np.max(np.abs(dphase(r.delta[c, :, :k], od[0, c, :, :k]))) <= TOL_DELTA_DEG
    assert np.max(np.abs(r.sigma - os_[0]) / os_[0]) <= TOL_SIGMA_REL


def test_unknown_ticket_and_bad_requests(server):
    from paper_2106_00454_gb300 import api
    with pytest.raises(api.WpcdError) as ei:
        server.poll(123456789)
    assert ei.value.code == -8
    c0, e0, _ = _req(3, 32)
    assert server.submit(c0, e0, 48, 0, raise_on_error=False) == -1          # N_WP not served
    assert server.submit(c0, -e0, 32, 0, raise_on_error=False) == -1         # non-positive energies


def test_admission_refusal_and_timeout():
    c = _ctx()
    try:
        c.serve_start(CHANNELS, W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA, [64], max_batch=4, n_slots=1,
                      max_queue=2)
        refused = 0
        tickets = []
        for k in range(2000):
            out = c.submit(*_req(500 + k, 64), 0, raise_on_error=False)
            if out == -3:
                refused += 1
                if refused >= 3:
                    break
            else:
                tickets.append(out)
        assert refused >= 1
        from paper_2106_00454_gb300 import api
        with pytest.raises(api.WpcdError) as ei:
            c.wait(tickets[-1], timeout_ms=0)
        assert ei.value.code in (-5,)
        for t in tickets:
            assert c.wait(t).status == 0
    finally:
        c.serve_stop()
        c.close()
