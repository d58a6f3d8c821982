"""Pins of the oracle's two resolvent variants (App. B).

* SWP-index averaging: the printed App. B form, where the on-shell energy is
  averaged over SWP bin i (not free bin i); defined for uncoupled channels
  without bound states.
* Point resolvent: no averaging; T and the phases at each requested energy,
  converted to the continuum at p itself.

Each is checked against brute force on N_WP = 6 (LAPACK eigenpairs and
adaptive quadrature, none of the oracle's code), a closed-form property, and
the convergence of the method towards the Yamaguchi closed form.
"""
import numpy as np
import pytest
from scipy import integrate

from paper_2106_00454_gb300 import inputs as W

HBARC = 197.3269804
MN = 938.918309
MU = 0.5 * MN / HBARC
LAM, BETA = W.YAMAGUCHI_PARAMS


def _t_yamaguchi(p):
    # closed form for V = lam g(p') g(p): see test_oracle_pins
    g = 1.0 / (p * p + BETA * BETA)
    return g * g / (1.0 / LAM + np.pi * MU / (2 * BETA * (BETA - 1j * p)**2))


def _d_exact(p):
    S = 1 - 2j * np.pi * MU * p * _t_yamaguchi(p)
    return 0.5 * np.degrees(np.angle(S))


def _brute_small(orc, N=6):
    """Yamaguchi on N_WP = 6 by quadrature + LAPACK: (mesh, V, h0, eps, C, SWP boundaries)."""
    m = orc.Mesh(N)
    kb = m.kb
    g = lambda k: 1.0 / (k * k + BETA * BETA)
    G = np.array([integrate.quad(lambda k: k * g(k), a, b, epsrel=1e-14)[0] / np.sqrt(b - a)
                  for a, b in zip(kb[:-1], kb[1:])])
    V = LAM * np.outer(G, G)
    h0 = np.array([integrate.quad(lambda k: k * k / (2 * MU), a, b)[0] / (b - a) for a, b in zip(kb[:-1], kb[1:])])
    e, C = np.linalg.eigh(np.diag(h0) + V)
    nb = int(np.sum(e < 0))
    ep = e[nb:]
    B = np.zeros(len(ep) + 1)
    B[1:-1] = 0.5 * (ep[:-1] + ep[1:])
    B[-1] = ep[-1] + 0.5 * (B[-2] - B[-3])
    return m, V, e, C, nb, B


# --------------------------------------------------------------------------- SWP-index averaging
def test_swp_index_same_bin_real_part_vanishes(orc):
    # averaging the point resolvent of SWP bin s over SWP bin s itself: the
    # principal-value logs cancel, only -i pi / dB remains
    for lo, hi in [(0.0, 0.3), (0.01, 0.011), (2.0, 7.5)]:
        g = orc.gbar_scatt(lo, hi, lo, hi)
        assert g.real == 0.0
        assert abs(g.imag + np.pi / (hi - lo)) <= 1e-15 * np.pi / (hi - lo)


def test_swp_index_brute_force_small(orc):
    m, V, e, C, nb, B = _brute_small(orc)
    assert nb == 0  # the Yamaguchi fit has a virtual state only
    N = m.N
    kb = m.kb
    Tc, ph, eps, rc = orc.channel_solve(m, 1, V[None], None, mode=orc.AVG_SWP_INDEX)
    assert rc == 0
    for i in range(N):
        Ea, Eb = B[i], B[i + 1]  # SWP bin i
        gb = np.zeros(N, dtype=complex)
        for s in range(N):
            lo, hi = B[s], B[s + 1]
            f = lambda x: np.log(abs((Eb - x) / (Ea - x))) if x not in (Ea, Eb) else 0.0
            pts = [x for x in (Ea, Eb) if lo < x < hi]
            re = integrate.quad(f, lo, hi, points=pts or None, epsrel=1e-13, limit=200)[0]
            ov = max(0.0, min(Eb, hi) - max(Ea, lo))
            gb[s] = (re - 1j * np.pi * ov) / ((Eb - Ea) * (hi - lo))
        R = V[i] @ C
        T = V[i, i] + np.sum(R * R * gb)
        kbar = 0.5 * (kb[i] + kb[i + 1])
        Tq = T / ((kb[i + 1] - kb[i]) * kbar**2)
        assert abs(Tc[i, 0, 0] - Tq) < 1e-9 * abs(Tq)


def test_swp_index_converges_yamaguchi(orc):
    errs, unit = [], []
    for N in (32, 64, 128):
        m = orc.Mesh(N)
        Vt = orc.project_channel(m, (0, 0, 0, 0, 0, 0), W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1)
        Tc, ph, eps, rc = orc.channel_solve(m, 1, Vt, None, mode=orc.AVG_SWP_INDEX)
        assert rc == 0
        sel = (m.kbar > 0.1) & (m.kbar < 2.1)
        de = np.array([_d_exact(p) for p in m.kbar])
        err = (ph[:, 0] - de + 90) % 180 - 90
        errs.append(np.max(np.abs(err[sel])))
        S = 1 - 2j * np.pi * MU * m.kbar * Tc[:, 0, 0]
        unit.append(np.max(np.abs(np.abs(S[sel]) - 1)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.4
    assert unit[0] > unit[1] > unit[2]


def test_swp_index_refuses_coupled_and_bound(orc):
    m = orc.Mesh(24)
    ch = W.Channel(1, 1, 0, 2, 1)  # 3S1-3D1: coupled, with the deuteron-like bound state
    Vt = orc.project_channel(m, ch.astuple(), W.GEN_YUKAWA, W.YUKAWA_PARAMS, 1)
    assert orc.channel_solve(m, 2, Vt, None, mode=orc.AVG_SWP_INDEX)[3] == -4
    assert orc.channel_solve(m, 2, Vt, None)[3] == 1


# --------------------------------------------------------------------------- point resolvent
def test_point_brute_force_small(orc):
    m, V, e, C, nb, B = _brute_small(orc)
    N = m.N
    kb = m.kb
    p = np.array([0.05, 0.3, 0.77, 1.5, 3.9, 7.2])
    p = p[p < kb[-1]]
    Tc, ph, rc = orc.channel_solve_point(m, 1, V[None], None, p)
    assert rc == 0
    for k, pk in enumerate(p):
        E = pk * pk / (2 * MU)
        i = int(np.searchsorted(kb, pk, side="right") - 1)
        g = np.zeros(N, dtype=complex)
        for s in range(N):
            lo, hi = B[s], B[s + 1]
            # Cauchy principal value of int_lo^hi dx / (E - x), over the SWP bin width
            g[s] = (np.log(abs((E - lo) / (E - hi))) - 1j * np.pi * (lo <= E <= hi)) / (hi - lo)
        R = V[i] @ C
        T = V[i, i] + np.sum(R * R * g)
        Tq = T / ((kb[i + 1] - kb[i]) * pk**2)
        assert abs(Tc[k, 0, 0] - Tq) < 1e-10 * abs(Tq)
        S = 1 - 2j * np.pi * MU * pk * Tq
        assert abs(ph[k, 0] - 0.5 * np.degrees(np.angle(S))) < 1e-9


def test_point_converges_yamaguchi(orc):
    p = orc.p_of_tlab(np.linspace(1.0, 350.0, 64))
    de = np.array([_d_exact(x) for x in p])
    rms = []
    for N in (32, 64, 128):
        m = orc.Mesh(N)
        Vt = orc.project_channel(m, (0, 0, 0, 0, 0, 0), W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1)
        Tc, ph, rc = orc.channel_solve_point(m, 1, Vt, None, p)
        assert rc == 0
        err = (ph[:, 0] - de + 90) % 180 - 90
        rms.append(np.sqrt(np.mean(err**2)))
    assert rms[1] < 0.6 * rms[0] and rms[2] < 0.6 * rms[1] and rms[2] < 0.5


def test_point_outside_mesh(orc):
    m = orc.Mesh(16)
    Vt = orc.project_channel(m, (0, 0, 0, 0, 0, 0), W.GEN_YAMAGUCHI, W.YAMAGUCHI_PARAMS, 1)
    assert orc.channel_solve_point(m, 1, Vt, None, [0.5, 9.0])[2] == -3


@pytest.mark.parametrize("mode", [1, 2])
def test_batch_modes_match_channel_solves(orc, mode):
    # the batch driver of each mode against its per-channel solve
    chs = [W.Channel(0, 0, 0, 0, 0), W.Channel(0, 1, 1, 1, 0)]
    meshes = [orc.Mesh(20), orc.Mesh(24)]
    Vts = [orc.project_channel(mm, ch.astuple(), W.GEN_YUKAWA, W.YUKAWA_PARAMS, 1) for mm, ch in zip(meshes, chs)]
    e_lab = np.array([5.0, 40.0, 120.0, 300.0])
    coeffs = np.zeros((1, 1))
    t, d, s, rc = orc.batch([c.astuple() for c in chs], meshes, Vts, coeffs, e_lab, mode=mode)
    assert rc == 0
    p = orc.p_of_tlab(e_lab)
    acc = np.zeros(len(e_lab))
    for c, (ch, mm, Vt) in enumerate(zip(chs, meshes, Vts)):
        if mode == 2:
            Tc, ph, rc2 = orc.channel_solve_point(mm, 1, Vt, None, p)
            assert rc2 >= 0
            np.testing.assert_allclose(t[0, c, :, 0, 0], Tc[:, 0, 0], rtol=1e-13, atol=0)
            np.testing.assert_allclose(d[0, c], ph, rtol=0, atol=1e-12)
        else:
            Tc, ph, _, rc2 = orc.channel_solve(mm, 1, Vt, None, mode=mode)
            assert rc2 == 0
            for k, pk in enumerate(p):
                i = int(np.searchsorted(mm.kb, pk, side="right") - 1)
                assert t[0, c, k, 0, 0] == Tc[i, 0, 0]
                np.testing.assert_allclose(d[0, c, k], orc.interp_phase(mm, ph, 1, pk), rtol=0, atol=1e-12)
        acc += np.array([orc.sigma_term(ch.J, 1, d[0, c, k]) for k in range(len(p))])
    np.testing.assert_allclose(s[0], [orc.sigma_prefactor_mb(pk) for pk in p] * acc, rtol=1e-13)
