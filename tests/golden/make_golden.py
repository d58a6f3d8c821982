"""Writes the regression fixtures in this directory from the oracle alone.

yamaguchi_1s0_nwp32.txt: the oracle's WPCD result for the 1S0 Yamaguchi
workload (N_WP = 32 capped-tan mesh, Q = 8, 64 lab energies 1..350 MeV):
the phase shift (Sec. 3.2 recipe, phases by App. A, interpolated as in
Sec. 5.1.1) and the np total cross section at every energy.  The paper prints
no worked-example values for a potential that can be rebuilt here (its
numbers are for N2LO_opt), so this file pins the oracle against its own
earlier output, a regression check beside the independent pins of
tests/test_oracle_pins.py.  Run from the repository root:
python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2106_00454_gb300 import inputs as W  # noqa: E402


def yamaguchi():
    wl = W.workload_yamaguchi()
    m = oracle.Mesh(wl.nwp[0])
    Vt = oracle.project_channel(m, wl.channels[0].astuple(), wl.gen, wl.gen_params, wl.n_terms)
    _, d, s, rc = oracle.batch([wl.channels[0].astuple()], [m], [Vt], np.zeros((1, 1)), wl.e_lab)
    assert rc == 0
    return wl.e_lab, d[0, 0, :, 0], s[0]


def main():
    e, delta, sigma = yamaguchi()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "yamaguchi_1s0_nwp32.txt")
    with open(out, "w") as f:
        f.write("# WPCD (oracle) for the 1S0 Yamaguchi workload, N_WP = 32, Q = 8: Sec. 3.2, App. A, Sec. 5.1.1\n")
        f.write("# written by tests/golden/make_golden.py; regression fixture (no paper values exist for it)\n")
        f.write("# T_lab [MeV]  delta [deg]  sigma_tot [mb]\n")
        for a, b, c in zip(e, delta, sigma):
            f.write(f"{float(a)!r} {float(b)!r} {float(c)!r}\n")


if __name__ == "__main__":
    main()
