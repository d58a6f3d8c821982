"""Reduced-precision projection (row a1): the Yukawa angle integrals as a
tensor-core contraction (BF16 three-term split, FP32 accumulation) against the
FP64 projection, term by term, and the mixed path run on it against the oracle."""
import dataclasses

import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import compare_mixed, gpu_run, oracle_run

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


def _report_worst(n_wp, Q, worst):
    """Append the measured difference to $WPCD_REPORT_DIR/projection_tc.jsonl when that is set."""
    import json
    import os
    out = os.environ.get("WPCD_REPORT_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "projection_tc.jsonl"), "a") as f:
            f.write(json.dumps({"n_wp": n_wp, "Q": Q, "worst_rel": worst}) + "\n")


def _terms(ctx, md, n_ch):
    out = []
    for c in range(n_ch):
        nch, nt, n = ctx.vset_info(md.vset, c)
        out.append(ctx.vset_get(md.vset, c).reshape(nt, n, n))
    return out


@pytest.mark.parametrize("n_wp,Q", [(40, 8), (23, 5), (30, 1)])
def test_tensor_core_angle_integrals_match_fp64(ctx, n_wp, Q):
    """Every channel J <= 6 and every term: the projection with the tensor-core
    angle integrals within 1e-5 of the FP64 projection, relative to the term's
    largest element.  The digit products are accumulated exactly and truncated
    at 2^-31; what remains is the FP32 evaluation of the integrand, amplified
    where the higher-L angle sums cancel (measured worst 1.2e-6, 1.6e-6 and
    6.5e-6 for the three cases).  Q = 5 puts bin pairs across 128-pair tiles,
    Q = 1 is the midpoint rule."""
    from paper_2106_00454_gb300 import api
    wl = dataclasses.replace(W.workload_all_channels(n_wp=n_wp, jmax=6, n_e=16), Q=Q)
    m64 = api.Model(ctx, wl)
    mtc = api.Model(ctx, wl, proj_prec=api.PREC_MIXED)
    ctx.sync()
    worst = 0.0
    for a, b in zip(_terms(ctx, m64, len(wl.channels)), _terms(ctx, mtc, len(wl.channels))):
        for t in range(a.shape[0]):
            sc = np.max(np.abs(a[t]))
            if sc == 0.0:
                assert np.max(np.abs(b[t])) == 0.0
                continue
            err = np.max(np.abs(a[t] - b[t])) / sc
            worst = max(worst, err)
    _report_worst(n_wp, Q, worst)
    assert 0.0 < worst < 1e-5, worst  # nonzero: the contraction really ran in reduced precision
    m64.release()
    mtc.release()


def test_mixed_path_on_tensor_core_projection(ctx, orc):
    """The N_WP = 150 workload (20 channels) with the tensor-core projection and
    the mixed eigensolve, every result within 1e-3 deg / 0.01 mb of the oracle."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_mixed(n_samples=2)
    md = api.Model(ctx, wl, proj_prec=api.PREC_MIXED)
    compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl))
