"""Pins of the oracle's spin observables (App. A): M-matrix partial-wave
expansion, Saclay amplitudes and dsigma/dOmega.

Checked against library routines (sympy Clebsch-Gordan, scipy spherical
harmonics), the textbook spinless amplitude, the spin-independent limit
(a = b = f(theta), c = d = e = 0 for a central force), the optical theorem
against the partial-wave sigma_tot, the integrated cross section against
sigma_tot for a unitary S, and the Saclay completeness relation.
"""
import numpy as np
import pytest

from paper_2106_00454_gb300 import inputs as W


def test_cg_against_sympy(orc):
    cgmod = pytest.importorskip("sympy.physics.quantum.cg")
    rng = np.random.default_rng(3)
    for _ in range(60):
        j1 = int(rng.integers(0, 7))
        j2 = int(rng.integers(0, 2))
        J = int(rng.integers(abs(j1 - j2), j1 + j2 + 1))
        m1 = int(rng.integers(-j1, j1 + 1))
        m2 = int(rng.integers(-j2, j2 + 1))
        ref = float(cgmod.CG(j1, m1, j2, m2, J, m1 + m2).doit())
        assert abs(orc.cg(j1, m1, j2, m2, J, m1 + m2) - ref) < 1e-13


def test_ylm_against_scipy(orc):
    special = pytest.importorskip("scipy.special")
    for l in range(0, 10):
        for m in range(-min(l, 2), min(l, 2) + 1):
            for th in (0.0, 0.37, 1.2, 2.9, np.pi):
                if hasattr(special, "sph_harm_y"):
                    ref = special.sph_harm_y(l, m, th, 0.0)
                else:  # older scipy: sph_harm(m, l, azimuth, polar)
                    ref = special.sph_harm(m, l, 0.0, th)
                assert abs(orc.ylm(l, m, th) - ref.real) < 1e-12 and abs(ref.imag) < 1e-14


def _np_channels(jmax):
    return [c.astuple() for c in W.np_channels(jmax)]


def _random_phases(chs, rng):
    ph = np.zeros((len(chs), 3))
    for c, ch in enumerate(chs):
        ph[c, 0] = rng.uniform(-80, 80)
        if ch[4]:
            ph[c, 1] = rng.uniform(-80, 80)
            ph[c, 2] = rng.uniform(-15, 15)
    return ph


def test_spinless_singlet_s_wave(orc):
    p, d = 0.7, 37.0
    ab, ds = orc.saclay([(0, 0, 0, 0, 0, 0)], [[d, 0.0, 0.0]], p, np.linspace(0, np.pi, 7))
    f = (np.exp(2j * np.radians(d)) - 1) / (2j * p)
    # singlet only: M = f |00><00|, unpolarised dsigma = |f|^2 / 4
    np.testing.assert_allclose(ds, 10 * abs(f)**2 / 4, rtol=1e-13)


def test_central_force_is_spin_independent(orc):
    # the same S_l in every (l, s, J) channel and no mixing: M = f(theta) 1 with the
    # spinless f = sum_l (2l+1)(S_l - 1) P_l(cos theta) / (2 i p).  With J <= 6 the
    # triplet l is complete (J = l - 1, l, l + 1) up to l = 5: no scattering above.
    chs = _np_channels(6)
    rng = np.random.default_rng(5)
    lmax = 5
    dl = np.zeros(9)
    dl[:lmax + 1] = rng.uniform(-60, 60, lmax + 1)
    ph = np.zeros((len(chs), 3))
    for c, ch in enumerate(chs):
        if ch[4]:
            ph[c, 0], ph[c, 1] = dl[ch[1] - 1], dl[ch[1] + 1]
        else:
            ph[c, 0] = dl[ch[2]]
    p = 1.1
    th = np.linspace(0.0, np.pi, 9)
    ab, ds, M = orc.saclay(chs, ph, p, th, want_m=True)
    from numpy.polynomial import legendre
    coef = np.array([(2 * l + 1) * (np.exp(2j * np.radians(dl[l])) - 1) for l in range(lmax + 1)]) / (2j * p)
    f = legendre.legval(np.cos(th), coef)
    for t in range(len(th)):
        np.testing.assert_allclose(M[t], f[t] * np.eye(4), rtol=0, atol=1e-12 * abs(f).max())
    np.testing.assert_allclose(ab[:, 0], f, rtol=0, atol=1e-12 * abs(f).max())
    np.testing.assert_allclose(ab[:, 1], f, rtol=0, atol=1e-12 * abs(f).max())
    assert np.max(np.abs(ab[:, 2:])) < 1e-12 * abs(f).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_optical_theorem_and_integrated_cross_section(orc, seed):
    chs = _np_channels(6)
    rng = np.random.default_rng(seed)
    ph = _random_phases(chs, rng)
    p = 0.4 + rng.uniform(0, 1.5)
    sig = orc.sigma_prefactor_mb(p) * sum(orc.sigma_term(ch[1], 2 if ch[4] else 1, ph[c])
                                          for c, ch in enumerate(chs) if ch[5] == 0)
    ab0, _ = orc.saclay(chs, ph, p, [0.0])
    assert abs(2 * np.pi / p * (ab0[0, 0] + ab0[0, 1]).imag * 10 - sig) < 1e-12 * sig
    x, w = np.polynomial.legendre.leggauss(40)
    ab, ds = orc.saclay(chs, ph, p, np.arccos(x))
    assert abs(2 * np.pi * np.sum(w * ds) - sig) < 1e-11 * sig  # elastic only: sigma_el = sigma_tot
    # completeness of the Saclay decomposition: Tr(M M^+)/4 = (|a|^2 + ... + |e|^2)/2
    np.testing.assert_allclose(ds, 10 * 0.5 * np.sum(np.abs(ab)**2, axis=1), rtol=1e-12)


def test_forward_amplitudes(orc):
    # at theta = 0 the spin-flip amplitude e vanishes and d, defined with
    # 1/sin(theta) in the helicity form, stays finite here by construction
    chs = _np_channels(4)
    ph = _random_phases(chs, np.random.default_rng(9))
    ab, _ = orc.saclay(chs, ph, 0.9, [0.0, 1e-4])
    assert abs(ab[0, 4]) < 1e-13 * np.max(np.abs(ab[0]))
    np.testing.assert_allclose(ab[1], ab[0], rtol=0, atol=1e-3 * np.max(np.abs(ab[0])))
