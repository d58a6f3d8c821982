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


def test_energy_above_mesh_refused_and_mix_unaffected(server):
    """A request with an energy above the mesh's top (p(E) >= 8 fm^-1, T_lab > 5.3
    GeV) is refused at submission, so the good requests around it in the same
    burst still complete with WPCD_OK and the same results as alone."""
    c0, e0, nw0 = _req(11, 32)
    alone = server.wait(server.submit(c0, e0, nw0, 1))
    assert alone.status == 0
    bad_e = np.concatenate([e0[:-1], [6000.0]])
    tickets = [server.submit(*_req(300 + k, 32), 1) for k in range(10)]
    assert server.submit(c0, bad_e, nw0, 1, raise_on_error=False) == -1
    tm = server.submit(c0, e0, nw0, 1)
    tickets += [server.submit(*_req(320 + k, 32), 1) for k in range(10)]
    mixed = server.wait(tm)
    assert mixed.status == 0
    _same(alone, mixed)
    for tk in tickets:
        assert server.wait(tk).status == 0
        server.release_result(tk)


def test_served_nwp256_matches_oracle(orc):
    """N_WP = 256 (coupled blocks 512 x 512, the global-memory Jacobi) served on
    the mixed path and in FP64, against the oracle at each path's tolerances."""
    from parity_util import TOL_MIXED_DELTA_DEG, TOL_MIXED_SIGMA_MB
    chans = [CHANNELS[0], CHANNELS[4]]  # 1S0 (256 x 256) and 3S1-3D1 (512 x 512)
    c = _ctx()
    try:
        c.serve_start(chans, W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA, [256], max_batch=8, n_slots=2)
        coeffs, e_lab, _ = _req(21, 256)
        r64 = c.wait(c.submit(coeffs, e_lab, 256, 0), 600000)
        rmx = c.wait(c.submit(coeffs, e_lab, 256, 1), 600000)
        assert r64.status == 0 and rmx.status == 0
        meshes = [orc.Mesh(256) for _ in chans]
        Vts = [orc.project_channel(m, ch.astuple(), W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA)
               for m, ch in zip(meshes, chans)]
        ot, od, os_, rc = orc.batch([ch.astuple() for ch in chans], meshes, Vts, coeffs[None], e_lab)
        assert rc == 0
        for ci, ch in enumerate(chans):
            k = 2 if ch.coupled else 1
            scale = np.max(np.abs(ot[0, ci]))
            assert np.max(np.abs(r64.T[ci] - ot[0, ci])) <= TOL_T * scale
            assert np.max(np.abs(dphase(r64.delta[ci, :, :k], od[0, ci, :, :k]))) <= TOL_DELTA_DEG
            assert np.max(np.abs(dphase(rmx.delta[ci, :, :k], od[0, ci, :, :k]))) <= TOL_MIXED_DELTA_DEG
            if ch.coupled:
                assert np.max(np.abs(r64.delta[ci, :, 2] - od[0, ci, :, 2])) <= TOL_DELTA_DEG
                assert np.max(np.abs(rmx.delta[ci, :, 2] - od[0, ci, :, 2])) <= TOL_MIXED_DELTA_DEG
        # sigma here sums only the two served channels, on both sides
        assert np.max(np.abs(r64.sigma - os_[0]) / os_[0]) <= TOL_SIGMA_REL
        assert np.max(np.abs(rmx.sigma - os_[0])) <= TOL_MIXED_SIGMA_MB
    finally:
        c.serve_stop()
        c.close()
