"""Mixed-precision path (FP32 Jacobi + FP64 Rayleigh refinement) against the
FP64 oracle: |d delta|, |d eps_J| <= 1e-3 deg and |d sigma| <= 0.01 mb for every
(sample, channel, energy)."""
import json
import os

import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

from parity_util import compare_mixed, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
MIXED = 1


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


def _report(name, worst):
    """Append the worst errors of a case to $WPCD_REPORT_DIR/mixed_errors.jsonl when that is set."""
    out = os.environ.get("WPCD_REPORT_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "mixed_errors.jsonl"), "a") as f:
            f.write(json.dumps({"case": name, **worst}) + "\n")


def test_mixed_yamaguchi(ctx, orc):
    from paper_2106_00454_gb300 import api
    wl = W.workload_yamaguchi()
    md = api.Model(ctx, wl)
    _report("yamaguchi", compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl)))


def test_mixed_all_channels(ctx, orc):
    """Workload 2 (20 channels, N_WP = 100) through the mixed path."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_all_channels()
    md = api.Model(ctx, wl)
    _report("all_channels_nwp100", compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl)))


def test_mixed_all_channels_fp64_refine_engine(ctx, orc):
    """Workload 2 with the refinement products on the FP64 CUDA cores."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_all_channels()
    md = api.Model(ctx, wl)
    ctx.set_refine_engine(api.REFINE_FP64)
    try:
        gpu = gpu_run(ctx, md, wl, prec=MIXED)
    finally:
        ctx.set_refine_engine(api.REFINE_TENSOR)
    _report("all_channels_nwp100_fp64_engine", compare_mixed(wl, gpu, oracle_run(orc, wl)))


def test_mixed_batched_sampled(ctx, orc):
    """Workload 3 at full size through the mixed path; sampled samples vs the oracle."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched()
    md = api.Model(ctx, wl)
    gpu = gpu_run(ctx, md, wl, prec=MIXED)
    pick = [0, 2048, 4095]
    _report("batched_4096_sampled", compare_mixed(wl, gpu, oracle_run(orc, wl, samples=pick), sample_idx=pick))


def test_mixed_nwp150_sampled(ctx, orc):
    """Workload 4's generator (20 channels, N_WP = 150, coupled 300 x 300) on a
    small batch, every sample against the oracle."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_mixed(n_samples=2)
    md = api.Model(ctx, wl)
    _report("nwp150_2samples", compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl)))


def test_mixed_eigenvalues_refined(ctx, orc):
    torch = pytest.importorskip("torch")
    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=2)
    ch = wl.channels[4]
    wl1 = W.Workload("e", [ch], [100], wl.gen, wl.gen_params, wl.n_terms, wl.coeffs, wl.e_lab)
    md = api.Model(ctx, wl1)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    e64 = ctx.diag(md.vset, cf, 2, prec=0)
    e32 = ctx.diag(md.vset, cf, 2, prec=MIXED)
    ctx.sync()
    worst, where, orth = 0.0, None, 0.0
    for s in range(2):
        a, _ = ctx.eig_get(e64, s, 0, 200)
        b, C = ctx.eig_get(e32, s, 0, 200)
        # The resolvent sees an eigenvalue error through the SWP bin width it
        # shifts, ~ (e_{s+2} - e_{s-2})/4 for the two interleaved branches;
        # checked where the requested energies reach (0.5..200 MeV c.m.).  The
        # refinement deliberately leaves clusters of near-zero eigenvalues
        # (far below 1 MeV) unrotated: T is invariant to rotations inside them.
        idx = np.arange(200)
        width = (a[np.minimum(idx + 2, 199)] - a[np.maximum(idx - 2, 0)]) / 4.0
        sel = (a > 0.5 / 197.3269804) & (a < 1.0)
        r = np.abs(a - b) / width
        k = int(np.argmax(np.where(sel, r, 0)))
        if r[k] > worst:
            worst, where = float(r[k]), (s, k, float(a[k]), float(b[k]))
        keep = np.where(a > 0.5 / 197.3269804)[0]
        Ck = C[:, keep]
        orth = max(orth, float(np.linalg.norm(Ck.T @ Ck - np.eye(len(keep)))))
    _report("eigenvalue_error_over_bin_width", {"worst": worst, "at": where, "orthogonality": orth})
    assert orth < 1e-6
    assert worst < 1e-4, where


@pytest.mark.parametrize("n_wp", [33, 57])
def test_mixed_odd_nwp(ctx, orc, n_wp):
    """Odd N_WP: the uncoupled matrices have odd n (the FP32 Jacobi pairs the
    last index with a zero phantom row), the coupled ones n = 2 N_WP."""
    import dataclasses

    from paper_2106_00454_gb300 import api
    wl = W.workload_all_channels(n_wp=n_wp, jmax=3, n_e=41)
    wl = dataclasses.replace(wl, coeffs=W.coefficient_samples(3))
    md = api.Model(ctx, wl)
    _report(f"odd_nwp{n_wp}", compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl)))


def test_mean_potential_basis_same_results_fewer_sweeps(ctx, orc):
    """The FP32 eigensolve in the eigenbasis of diag(H0) + V0 (the default) and in
    the original basis both match the oracle at the mixed tolerances on the
    N_WP = 150 workload; the rotated start takes fewer Jacobi sweeps."""
    import torch

    from paper_2106_00454_gb300 import api
    wl = W.workload_mixed(n_samples=4)
    md = api.Model(ctx, wl)
    ora = oracle_run(orc, wl)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    sweeps = {}
    for on in (True, False):
        ctx.set_rotate(on)
        try:
            _report(f"nwp150_rotate_{int(on)}", compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), ora))
            eid = ctx.diag(md.vset, cf, 4, prec=MIXED)
            st = torch.zeros((4, len(wl.channels)), dtype=torch.int32, device="cuda:0")
            ctx.diag_status(eid, st)
            ctx.sync()
            ctx.release(eid)
        finally:
            ctx.set_rotate(True)
        sweeps[on] = st.cpu().numpy()
    assert (sweeps[True] > 0).all() and (sweeps[False] > 0).all()
    assert sweeps[True].sum() < sweeps[False].sum(), (sweeps[True].sum(), sweeps[False].sum())


def test_single_refinement_iteration_phases(ctx, orc):
    """The opt-in single refinement iteration keeps the phase shifts inside
    1e-3 deg of the oracle on the N_WP = 150 workload; its cross sections are
    only within ~0.02 mb (measured 0.016 mb on 16 samples against the FP64
    path), outside the 0.01 mb bar, which is why two iterations are the default."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_mixed(n_samples=3)
    md = api.Model(ctx, wl)
    ctx.set_refine_iters(1)
    try:
        gpu = gpu_run(ctx, md, wl, prec=MIXED)
    finally:
        ctx.set_refine_iters(2)
    _report("nwp150_one_iteration", compare_mixed(wl, gpu, oracle_run(orc, wl), tol_s=0.05))


def test_refine_digits_option(ctx, orc):
    """WPCD_OPT_REFINE_DIGITS = 5 (15 digit pairs per product instead of 21): the
    N_WP = 150 workload stays within the mixed tolerances of the oracle (measured:
    1.9e-7 deg, 3.0e-6 mb with the FP64 projection); out-of-range values are refused."""
    from paper_2106_00454_gb300 import api
    wl = W.workload_mixed(n_samples=2)
    md = api.Model(ctx, wl)
    ctx.set_refine_digits(5)
    try:
        worst = compare_mixed(wl, gpu_run(ctx, md, wl, prec=MIXED), oracle_run(orc, wl))
    finally:
        ctx.set_refine_digits(6)
    _report("nwp150_refine_digits5", worst)
    assert worst["sigma_mb"] < 1e-3 and worst["delta_deg"] < 1e-4, worst
    with pytest.raises(api.WpcdError):
        ctx.set_refine_digits(3)
