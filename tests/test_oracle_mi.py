"""Pins of the oracle's MI comparison method at interpolation energies (Sec. 6):
the LS equation solved by matrix inversion at Chebyshev-distributed lab
energies, phase shifts interpolated linearly in T_lab.

The MI solver itself is pinned in test_oracle_pins (Yamaguchi closed form,
unitarity, optical theorem); these pins cover the batch driver and the
interpolation.
"""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W

HBARC = 197.3269804
MN = 938.918309
MU = 0.5 * MN / HBARC
LAM, BETA = W.YAMAGUCHI_PARAMS


def _d_exact(p):
    g = 1.0 / (p * p + BETA * BETA)
    t = g * g / (1.0 / LAM + np.pi * MU / (2 * BETA * (BETA - 1j * p)**2))
    return 0.5 * np.degrees(np.angle(1 - 2j * np.pi * MU * p * t))


def test_chebyshev_energies():
    e = W.chebyshev_energies(12, 350.0)
    assert np.all(np.diff(e) > 0) and e[0] > 0 and e[-1] < 350.0
    # the nodes are the images of cos((2k-1) pi / 2n): symmetric about e_max / 2
    np.testing.assert_allclose(e + e[::-1], 350.0, rtol=0, atol=1e-12)


def test_interp_tlab_linear_exact(orc):
    e_int = np.array([2.0, 10.0, 40.0, 90.0, 200.0, 330.0])
    ph = np.zeros((6, 3))
    ph[:, 0] = 20.0 + 0.1 * e_int
    ph[:, 1] = -5.0 + 0.02 * e_int
    ph[:, 2] = 1.0 - 0.003 * e_int
    for e in [1.0, 2.0, 33.3, 150.0, 330.0, 349.0]:  # incl. both extrapolated ends
        out = orc.interp_phase_tlab(e_int, ph, 2, e)
        np.testing.assert_allclose(out, [20 + 0.1 * e, -5 + 0.02 * e, 1 - 0.003 * e], rtol=0, atol=1e-12)


def test_interp_tlab_unwraps_across_90(orc):
    e_int = np.array([10.0, 20.0, 30.0])
    ph = np.zeros((3, 3))
    ph[:, 0] = [80.0, -85.0, -70.0]  # 80 -> 95 crossed +90
    out = orc.interp_phase_tlab(e_int, ph, 1, 15.0)
    assert abs(out[0] - 87.5) < 1e-12
    out = orc.interp_phase_tlab(e_int, ph, 1, 19.0)
    assert abs(out[0] - (93.5 - 180.0)) < 1e-12


def test_mi_batch_matches_single_solves(orc):
    chs = [W.Channel(0, 0, 0, 0, 0), W.Channel(1, 1, 0, 2, 1), W.Channel(1, 2, 1, 1, 0)]
    coeffs = W.coefficient_samples(2)
    e_int = W.chebyshev_energies(6)
    e_lab = np.array([5.0, 77.0, 300.0])
    Kb, d, s, rc = orc.mi_batch([c.astuple() for c in chs], W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA,
                                coeffs, e_int, e_lab, NQ=48)
    assert rc == 0
    for smp in range(2):
        acc = np.zeros(len(e_lab))
        for c, ch in enumerate(chs):
            ph = np.zeros((len(e_int), 3))
            for k, e in enumerate(e_int):
                p = orc.p_of_tlab(e)[0]
                Km = orc.mi_kmatrix(W.GEN_YUKAWA, W.YUKAWA_PARAMS, ch.astuple(), W.N_TERMS_YUKAWA, coeffs[smp], p,
                                    NQ=48)
                np.testing.assert_array_equal(Kb[smp, c, k, :ch.K, :ch.K], Km)
                ph[k] = orc.phases_from_S(orc.S_from_K(ch.K, p, Km))
            for k, e in enumerate(e_lab):
                np.testing.assert_allclose(d[smp, c, k], orc.interp_phase_tlab(e_int, ph, ch.K, e), rtol=0,
                                           atol=1e-12)
                acc[k] += orc.sigma_term(ch.J, ch.K, d[smp, c, k])
        pref = np.array([orc.sigma_prefactor_mb(orc.p_of_tlab(e)[0]) for e in e_lab])
        np.testing.assert_allclose(s[smp], pref * acc, rtol=1e-13)


def test_mi_interpolation_converges_yamaguchi(orc):
    # away from the low-energy extrapolation the interpolated MI phases approach
    # the closed form like the error of linear interpolation, ~1/n_I^2
    # (1.47, 0.45, 0.11 deg at n_I = 8, 16, 32)
    e_lab = np.linspace(20.0, 340.0, 33)
    de = np.array([_d_exact(orc.p_of_tlab(e)[0]) for e in e_lab])
    errs = []
    for n_I in (8, 16, 32):
        _, d, _, rc = orc.mi_batch([(0, 0, 0, 0, 0, 0)], W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1, np.zeros((1, 1)),
                                   W.chebyshev_energies(n_I), e_lab, NQ=48)
        assert rc == 0
        errs.append(np.max(np.abs(d[0, 0, :, 0] - de)))
    assert errs[1] < 0.35 * errs[0] and errs[2] < 0.35 * errs[1] and errs[2] < 0.15
