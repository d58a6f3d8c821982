"""Helpers shared by the GPU parity tests: run the oracle and the CUDA path on
the same seeded workload and compare element by element."""
import numpy as np

from paper_2106_00454_gb300 import inputs as W

# FP64 path tolerances: T relative to the channel's max |T| over the energies,
# phases in degrees (modulo 180 for delta, which is only defined mod 180),
# cross section relative.
TOL_T = 1e-10
TOL_DELTA_DEG = 1e-8
TOL_SIGMA_REL = 1e-8


def oracle_run(orc, wl: W.Workload, samples=None, mode=0):
    """Oracle outputs for the workload (optionally a subset of samples; mode =
    resolvent: 0 free-bin average, 1 SWP-bin average, 2 point)."""
    meshes = [orc.Mesh(n, wl.mesh_kind, wl.alpha, wl.t, wl.kmax, wl.Q) for n in wl.nwp]
    Vts = [orc.project_channel(m, ch.astuple(), wl.gen, wl.gen_params, wl.n_terms, wl.wp_kind)
           for m, ch in zip(meshes, wl.channels)]
    coeffs = wl.coeffs if samples is None else wl.coeffs[samples]
    if wl.n_terms == 1:
        coeffs = np.zeros((coeffs.shape[0], 1))
    t, d, s, rc = orc.batch([c.astuple() for c in wl.channels], meshes, Vts, coeffs, wl.e_lab, wl.wp_kind, mode=mode)
    assert rc == 0, rc
    return t, d, s


# Mixed-precision path tolerances (against the FP64 oracle)
TOL_MIXED_DELTA_DEG = 1e-3
TOL_MIXED_SIGMA_MB = 1e-2


def gpu_run(ctx, model, wl: W.Workload, device="cuda:0", via="solve", prec=0, res=0):
    import torch
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    coeffs = None if wl.n_terms == 1 else torch.tensor(wl.coeffs, dtype=torch.float64, device=device)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=device)
    t = torch.zeros((S, nch, nE, 2, 2, 2), dtype=torch.float64, device=device)
    d = torch.zeros((S, nch, nE, 3), dtype=torch.float64, device=device)
    s = torch.zeros((S, nE), dtype=torch.float64, device=device)
    if via == "solve":
        ctx.solve(model.vset, coeffs, S, e, t, d, s, prec=prec, res=res)
    else:
        eid = ctx.diag(model.vset, coeffs, S, prec=prec)
        ctx.tmatrix(eid, e, t, res=res)
        ctx.observables(eid, e, d, s, res=res)
        ctx.release(eid)
    ctx.sync()
    tc = t.cpu().numpy().view(np.complex128).reshape(S, nch, nE, 2, 2)
    return tc, d.cpu().numpy(), s.cpu().numpy()


def dphase(a, b):
    """Difference of phase shifts modulo 180 deg."""
    return (a - b + 90.0) % 180.0 - 90.0


def compare(wl, gpu, ora, tol_t=TOL_T, tol_d=TOL_DELTA_DEG, tol_s=TOL_SIGMA_REL, sample_idx=None):
    gt, gd, gs = gpu
    ot, od, os_ = ora
    if sample_idx is not None:
        gt, gd, gs = gt[sample_idx], gd[sample_idx], gs[sample_idx]
    report = {}
    for c, ch in enumerate(wl.channels):
        scale = np.max(np.abs(ot[:, c]))
        err = np.max(np.abs(gt[:, c] - ot[:, c]))
        report[ch.name] = err / scale
        assert err <= tol_t * scale, (ch.name, err, scale)
        ncomp = 2 if ch.coupled else 1
        dd = np.max(np.abs(dphase(gd[:, c, :, :ncomp], od[:, c, :, :ncomp])))
        assert dd <= tol_d, (ch.name, "delta", dd)
        if ch.coupled:
            de = np.max(np.abs(gd[:, c, :, 2] - od[:, c, :, 2]))
            assert de <= tol_d, (ch.name, "eps", de)
    rs = np.max(np.abs(gs - os_) / np.maximum(np.abs(os_), 1e-300))
    assert rs <= tol_s, ("sigma", rs)
    return report


def compare_mixed(wl, gpu, ora, tol_d=TOL_MIXED_DELTA_DEG, tol_s=TOL_MIXED_SIGMA_MB, sample_idx=None):
    """Mixed path: every (sample, channel, energy) phase within tol_d degrees and
    every cross section within tol_s mb of the FP64 oracle.  Returns the worst
    errors for reporting."""
    gt, gd, gs = gpu
    ot, od, os_ = ora
    if sample_idx is not None:
        gt, gd, gs = gt[sample_idx], gd[sample_idx], gs[sample_idx]
    worst = {"delta_deg": 0.0, "eps_deg": 0.0, "sigma_mb": 0.0, "T_rel": 0.0}
    for c, ch in enumerate(wl.channels):
        ncomp = 2 if ch.coupled else 1
        dd = float(np.max(np.abs(dphase(gd[:, c, :, :ncomp], od[:, c, :, :ncomp]))))
        worst["delta_deg"] = max(worst["delta_deg"], dd)
        if ch.coupled:
            worst["eps_deg"] = max(worst["eps_deg"], float(np.max(np.abs(gd[:, c, :, 2] - od[:, c, :, 2]))))
        sc = np.max(np.abs(ot[:, c]))
        worst["T_rel"] = max(worst["T_rel"], float(np.max(np.abs(gt[:, c] - ot[:, c])) / sc))
    worst["sigma_mb"] = float(np.max(np.abs(gs - os_)))
    assert worst["delta_deg"] <= tol_d and worst["eps_deg"] <= tol_d, worst
    assert worst["sigma_mb"] <= tol_s, worst
    return worst
