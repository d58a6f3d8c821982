"""Accuracy studies of the method on the GPU (Sec. 5): WPCD against the MI
solution of the same LS equation, both through the public API.

* ``sigma_error_map``: |sigma_WPCD - sigma_exact| / sigma_exact as a function of
  N_WP and T_lab (the error heat map of Sec. 5), "exact" being MI solved at
  every requested energy (no interpolation);
* ``rmse_study``: the root-mean-square deviation of sigma_tot from the exact
  result over lab-energy ranges, RMSE = sqrt(sum_i (sigma_exact,i -
  sigma_method,i)^2 / n_E) (Sec. 5.2), for WPCD at several N_WP and for MI with
  linear interpolation between n_I Chebyshev energies;
* ``interpolation_bands``: the spread of the interpolated phase shifts and
  sigma_tot over the interpolation point q_i = k_i + (n/m)(k_{i+1} - k_i)
  (Sec. 5.1.1; the paper's m = 10, n in {0.1, 1, 2, ..., 9, 9.9}).

Only orchestration lives here: every number comes from wpcd_solve and
wpcd_mi_solve.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import api
from . import inputs as W


def _wpcd_sigma(ctx, wl: W.Workload, prec):
    import torch
    dev = f"cuda:{ctx.device}"
    md = api.Model(ctx, wl)
    S, nE = wl.n_samples, len(wl.e_lab)
    cf = None if wl.n_terms == 1 else torch.tensor(wl.coeffs, dtype=torch.float64, device=dev)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    s = torch.empty((S, nE), dtype=torch.float64, device=dev)
    ctx.solve(md.vset, cf, S, e, None, None, s, prec=prec)
    ctx.sync()
    md.release()
    return s.cpu().numpy()


def _mi_sigma(ctx, wl: W.Workload, e_int, n_quad):
    import torch
    dev = f"cuda:{ctx.device}"
    mid = ctx.mi_prepare(wl.channels, wl.gen, wl.gen_params, wl.n_terms, n_quad=n_quad)
    S, nE = wl.n_samples, len(wl.e_lab)
    cf = None if wl.n_terms == 1 else torch.tensor(wl.coeffs, dtype=torch.float64, device=dev)
    ei = torch.tensor(np.asarray(e_int, dtype=np.float64), dtype=torch.float64, device=dev)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    s = torch.empty((S, nE), dtype=torch.float64, device=dev)
    ctx.mi_solve(mid, cf, S, ei, e, None, None, s)
    ctx.sync()
    ctx.release(mid)
    return s.cpu().numpy()


def exact_sigma(ctx, wl: W.Workload, n_quad=96):
    """sigma_tot [S, n_E] from MI solved at every requested energy."""
    return _mi_sigma(ctx, wl, wl.e_lab, n_quad)


def sigma_error_map(ctx, wl: W.Workload, nwp_list, prec=api.PREC_FP64, n_quad=96):
    """Relative sigma_tot error of WPCD for each N_WP in nwp_list (every
    channel on that N_WP): array [len(nwp_list), S, n_E], plus the exact sigma."""
    ref = exact_sigma(ctx, wl, n_quad)
    out = []
    for nwp in nwp_list:
        w = dataclasses.replace(wl, nwp=[int(nwp)] * len(wl.channels))
        out.append(np.abs(_wpcd_sigma(ctx, w, prec) - ref) / np.abs(ref))
    return np.array(out), ref


def rmse_study(ctx, wl: W.Workload, nwp_list, mi_interp_list=(), ranges=((0.0, 350.0), (40.0, 350.0)),
               prec=api.PREC_FP64, n_quad=96):
    """RMSE of sigma_tot against the exact result over each lab-energy range
    (lo, hi], per sample: {"wpcd": {nwp: [range][S]}, "mi": {n_I: [range][S]}}."""
    ref = exact_sigma(ctx, wl, n_quad)
    sel = [(wl.e_lab > lo) & (wl.e_lab <= hi) for lo, hi in ranges]

    def rmse(sig):
        return [np.sqrt(np.mean((sig[:, m] - ref[:, m])**2, axis=1)) for m in sel]

    res = {"ranges": list(ranges), "wpcd": {}, "mi": {}}
    for nwp in nwp_list:
        w = dataclasses.replace(wl, nwp=[int(nwp)] * len(wl.channels))
        res["wpcd"][int(nwp)] = rmse(_wpcd_sigma(ctx, w, prec))
    for n_i in mi_interp_list:
        res["mi"][int(n_i)] = rmse(_mi_sigma(ctx, wl, W.chebyshev_energies(int(n_i)), n_quad))
    return res


BAND_FRACS = (0.01, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.99)


def interpolation_bands(ctx, wl: W.Workload, fracs=BAND_FRACS, prec=api.PREC_FP64):
    """Phase shifts and sigma_tot for each interpolation point of fracs:
    {"delta": [len(fracs), S, ch, n_E, 3], "sigma": [len(fracs), S, n_E],
    "delta_lo"/"delta_hi", "sigma_lo"/"sigma_hi": the band over fracs}.
    The context's interpolation point is restored to the midpoint afterwards."""
    import torch
    dev = f"cuda:{ctx.device}"
    md = api.Model(ctx, wl)
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    cf = None if wl.n_terms == 1 else torch.tensor(wl.coeffs, dtype=torch.float64, device=dev)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    ds, ss = [], []
    try:
        for f in fracs:
            ctx.set_interp_point(f)
            d = torch.empty((S, nch, nE, 3), dtype=torch.float64, device=dev)
            s = torch.empty((S, nE), dtype=torch.float64, device=dev)
            ctx.solve(md.vset, cf, S, e, None, d, s, prec=prec)
            ctx.sync()
            ds.append(d.cpu().numpy())
            ss.append(s.cpu().numpy())
    finally:
        ctx.set_interp_point(0.5)
        md.release()
    d, s = np.array(ds), np.array(ss)
    return {"fracs": list(fracs), "delta": d, "sigma": s, "delta_lo": d.min(axis=0), "delta_hi": d.max(axis=0),
            "sigma_lo": s.min(axis=0), "sigma_hi": s.max(axis=0)}
