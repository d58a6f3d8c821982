"""A small, fixed eigensolver case for profilers (ncu): two batched eigensolves
of one channel of the synthetic Yukawa + contact potential.

    python -m paper_2106_00454_gb300.probe SAMPLES N_WP PREC CHANNEL [ROTATE]

SAMPLES parameter samples, N_WP packets per l-block, PREC 0 (FP64) or 1
(mixed), CHANNEL an index into the J <= 6 channel list (4 = 3S1-3D1, coupled,
2 N_WP x 2 N_WP), ROTATE 1 (default) or 0 for the mixed path's mean-potential
basis.  The first call autotunes the eigensolver's CTA size (four trial
launches per matrix size) and sizes the workspaces; the second is the one to
capture (for ncu: skip the launches of the first).
"""
from __future__ import annotations

import sys


def main(argv):
    import torch

    from . import api, build
    from . import inputs as W
    if len(argv) < 4:
        raise SystemExit(__doc__)
    S, n_wp, prec, ci = (int(x) for x in argv[:4])
    rotate = int(argv[4]) if len(argv) > 4 else 1
    build.build()
    ctx = api.Context(0)
    ctx.set_rotate(bool(rotate))
    ch = W.np_channels(6)[ci]
    wl = W.Workload("probe", [ch], [n_wp], W.GEN_YUKAWA, W.YUKAWA_PARAMS.copy(), W.N_TERMS_YUKAWA,
                    W.coefficient_samples(S), W.lab_energies(16))
    md = api.Model(ctx, wl)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        eid = ctx.diag(md.vset, cf, S, prec=prec)
        ctx.sync()
        ctx.release(eid)
    print(f"probe: {S} samples of {ch.name}, N_WP {n_wp}, prec {prec}, rotate {rotate}; tuning {ctx.tuning()}")
    ctx.close()


if __name__ == "__main__":
    main(sys.argv[1:])
