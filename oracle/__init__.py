"""Plain FP64 CPU oracle for the WPCD hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it, and
it imports nothing from the product package: the two share only the seeded
input generators, which hold none of the method's arithmetic.

The arithmetic lives in ``wpcd_oracle.c`` (plain C, FP64, written from the
paper: Sec. 3.2 five-step recipe, App. A observables, App. B resolvent, Sec. 2.1
matrix inversion).  This module compiles it with gcc on first use and wraps
each function with ctypes and numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wpcd_oracle.c")
_SO = os.path.join(_HERE, "liboracle_wpcd.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d, i = ctypes.c_double, ctypes.c_int
            sig = {
                "or_mu": (d, []), "or_hbarc": (d, []), "or_mn": (d, []),
                "or_p_of_tlab": (d, [d]), "or_version": (i, []),
                "or_gauss_legendre": (i, [i, _dp, _dp]),
                "or_mesh": (i, [i, i, d, d, d, i, _dp, _dp, _dp]),
                "or_potential": (d, [i, _dp, i, i, i, i, i, i, i, i, i, d, d]),
                "or_h0": (d, [i, d, d]),
                "or_project_channel": (i, [i, _dp, i, _dp, _dp, i, i, i, i, i, i, i, i, _dp, i, _dp]),
                "or_project_fine": (i, [i, _dp, i, _dp, _dp, i, i, _dp, _dp]),
                "or_jacobi": (i, [i, _dp, _dp, _dp]),
                "or_swp_boundaries": (i, [i, i, _dp, _ip, _ip, _ip, _dp]),
                "or_gbar_scatt": (None, [d, d, d, d, _dp, _dp]),
                "or_gbar_bound": (d, [d, d, d]),
                "or_g_point": (None, [d, d, d, _dp, _dp]),
                "or_contract": (None, [i, i, _dp, _dp, _dp, _dp, _dp, _dp]),
                "or_phases_from_S": (None, [i, _dp, _dp]),
                "or_S_from_T": (None, [i, d, _dp, _dp]),
                "or_channel_solve": (i, [i, _dp, i, i, i, _dp, _dp, i, _dp, _dp, _dp, _ip]),
                "or_channel_solve_ip": (i, [i, _dp, i, i, i, _dp, _dp, i, d, _dp, _dp, _dp, _ip]),
                "or_interp_phase_ip": (None, [i, _dp, _dp, i, d, d, _dp]),
                "or_batch_ip": (i, [i, _ip, _ip, _lp, _dp, i, i, _lp, _dp, i, _dp, i, _dp, i, d, _dp, _dp, _dp, i]),
                "or_channel_solve_point": (i, [i, _dp, i, i, i, _dp, _dp, i, _dp, _dp, _dp]),
                "or_interp_phase": (None, [i, _dp, _dp, i, d, _dp]),
                "or_sigma_term": (d, [i, i, _dp]),
                "or_sigma_prefactor_mb": (d, [d]),
                "or_mi_kmatrix": (i, [i, _dp, i, i, i, i, i, i, i, _dp, i, d, d, _dp]),
                "or_S_from_K": (None, [i, d, _dp, _dp]),
                "or_interp_phase_tlab": (None, [i, _dp, _dp, i, d, _dp]),
                "or_mi_batch": (i, [i, _ip, i, _dp, i, i, _dp, i, d, i, _dp, i, _dp, _dp, _dp, _dp, i]),
                "or_cg": (d, [i, i, i, i, i, i]),
                "or_ylm": (d, [i, i, d]),
                "or_saclay": (None, [i, _ip, _dp, d, i, _dp, _dp, _dp, _dp]),
                "or_batch": (i, [i, _ip, _ip, _lp, _dp, i, i, _lp, _dp, i, _dp, i, _dp, i, _dp, _dp, _dp, i]),
                "or_max_threads": (i, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- constants
def mu() -> float:
    return lib().or_mu()


def p_of_tlab(tlab_mev):
    f = lib().or_p_of_tlab
    return np.array([f(float(t)) for t in np.atleast_1d(tlab_mev)])


# ----------------------------------------------------------------------------- quadrature / mesh
def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, _d(x), _d(w))
    return x, w


class Mesh:
    """Free-wave-packet mesh: boundaries kb[0..N], fine nodes kq/wq [N*Q]."""

    def __init__(self, N, kind=0, alpha=0.5067730717679395, t=2.0, kmax=8.0, Q=8):
        self.N, self.kind, self.alpha, self.t, self.kmax, self.Q = N, kind, alpha, t, kmax, Q
        self.kb = np.zeros(N + 1)
        self.kq = np.zeros(N * Q)
        self.wq = np.zeros(N * Q)
        rc = lib().or_mesh(N, kind, alpha, t, kmax, Q, _d(self.kb), _d(self.kq), _d(self.wq))
        if rc != 0:
            raise ValueError("bad mesh arguments")

    @property
    def kbar(self):
        return 0.5 * (self.kb[:-1] + self.kb[1:])


def potential(gen, gp, ch, lp, l, term, pp, p):
    gp = _f64(gp)
    return lib().or_potential(gen, _d(gp), *[int(v) for v in ch], lp, l, term, float(pp), float(p))


def h0(wp_kind, ka, kb):
    return lib().or_h0(wp_kind, ka, kb)


def project_channel(mesh: Mesh, ch, gen, gp, n_terms, wp_kind=0):
    """Bin-averaged potential of every term, shape (n_terms, n, n), n = K*N."""
    K = 2 if ch[4] else 1
    n = K * mesh.N
    Vt = np.zeros((n_terms, n, n))
    gp = _f64(gp)
    rc = lib().or_project_channel(mesh.N, _d(mesh.kb), mesh.Q, _d(mesh.kq), _d(mesh.wq), wp_kind,
                                  *[int(v) for v in ch], gen, _d(gp), n_terms, _d(Vt))
    if rc != 0:
        raise RuntimeError("projection failed")
    return Vt


def project_fine(mesh: Mesh, K, vfine, wp_kind=0):
    n = K * mesh.N
    vfine = _f64(vfine)
    V = np.zeros((n, n))
    lib().or_project_fine(mesh.N, _d(mesh.kb), mesh.Q, _d(mesh.kq), _d(mesh.wq), wp_kind, K, _d(vfine), _d(V))
    return V


# ----------------------------------------------------------------------------- eigen
def jacobi(H):
    H = _f64(H)
    n = H.shape[0]
    eps = np.zeros(n)
    C = np.zeros((n, n))
    sweeps = lib().or_jacobi(n, _d(H), _d(eps), _d(C))
    return eps, C, sweeps


def swp_boundaries(eps, K):
    eps = _f64(eps)
    n = eps.shape[0]
    branch = np.zeros(n, dtype=np.int32)
    pos = np.zeros(n, dtype=np.int32)
    mcount = np.zeros(2, dtype=np.int32)
    bnd = np.zeros(2 * (n + 1))
    nb = lib().or_swp_boundaries(n, K, _d(eps), _i(branch), _i(pos), _i(mcount), _d(bnd))
    return nb, branch, pos, mcount, bnd.reshape(2, n + 1)


def gbar_scatt(Ea, Eb, Bs, Bs1) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_gbar_scatt(Ea, Eb, Bs, Bs1, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def gbar_bound(Ea, Eb, eb) -> float:
    return lib().or_gbar_bound(Ea, Eb, eb)


def g_point(E, Bs, Bs1) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_g_point(E, Bs, Bs1, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def contract(Vd, R, g):
    """T_ab = Vd_ab + sum_s R_as g_s R_bs (K x K complex)."""
    Vd = _f64(Vd)
    R = _f64(R)
    K, n = R.shape
    g = np.asarray(g, dtype=np.complex128)
    gre = _f64(g.real)
    gim = _f64(g.imag)
    Tr = np.zeros((K, K))
    Ti = np.zeros((K, K))
    lib().or_contract(n, K, _d(Vd), _d(R), _d(gre), _d(gim), _d(Tr), _d(Ti))
    return Tr + 1j * Ti


# ----------------------------------------------------------------------------- observables
def S_from_T(K, p, T):
    T = np.ascontiguousarray(T, dtype=np.complex128).reshape(K * K)
    S = np.zeros(K * K, dtype=np.complex128)
    lib().or_S_from_T(K, p, T.ctypes.data_as(_dp), S.ctypes.data_as(_dp))
    return S.reshape(K, K)


def phases_from_S(S):
    S = np.ascontiguousarray(S, dtype=np.complex128)
    K = S.shape[0]
    out = np.zeros(3)
    lib().or_phases_from_S(K, S.reshape(-1).ctypes.data_as(_dp), _d(out))
    return out


def S_from_K(K, p, Km):
    Km = _f64(Km).reshape(K * K)
    S = np.zeros(K * K, dtype=np.complex128)
    lib().or_S_from_K(K, p, _d(Km), S.ctypes.data_as(_dp))
    return S.reshape(K, K)


def interp_phase(mesh: Mesh, ph, K, p, frac=0.5):
    """Phases interpolated linearly in p between the interpolation points of
    consecutive bins, (1 - frac) k_i + frac k_{i+1} (Sec. 5.1.1; frac = 0.5:
    the midpoints)."""
    ph = _f64(ph)
    out = np.zeros(3)
    if frac == 0.5:
        lib().or_interp_phase(mesh.N, _d(mesh.kb), _d(ph), K, float(p), _d(out))
    else:
        lib().or_interp_phase_ip(mesh.N, _d(mesh.kb), _d(ph), K, float(p), float(frac), _d(out))
    return out


def sigma_term(J, K, ph):
    ph = _f64(ph)
    return lib().or_sigma_term(J, K, _d(ph))


def sigma_prefactor_mb(p):
    return lib().or_sigma_prefactor_mb(p)


# ----------------------------------------------------------------------------- solves
AVG_FREE_BIN, AVG_SWP_INDEX, POINT = 0, 1, 2  # resolvent modes


def channel_solve(mesh: Mesh, K, Vt, c, wp_kind=0, mode=AVG_FREE_BIN, frac=0.5):
    """One channel-solve at every free bin.

    mode: AVG_FREE_BIN (resolvent averaged over the free bin) or AVG_SWP_INDEX
    (over SWP bin i; uncoupled channels without bound states, else rc = -4).
    Returns (Tc [N,K,K] complex continuum T at the bin midpoints in fm^2,
    ph [N,3] degrees, eps [n], rc) where rc = number of bound states or a
    negative error code."""
    Vt = _f64(Vt)
    n_terms = Vt.shape[0]
    n = Vt.shape[1]
    c = _f64(np.zeros(max(n_terms - 1, 1)) if c is None else c)
    N = mesh.N
    Tc = np.zeros((N, K, K), dtype=np.complex128)
    ph = np.zeros((N, 3))
    eps = np.zeros(n)
    sweeps = ctypes.c_int()
    rc = lib().or_channel_solve_ip(N, _d(mesh.kb), wp_kind, K, n_terms, _d(Vt), _d(c), int(mode), float(frac),
                                   Tc.ctypes.data_as(_dp), _d(ph), _d(eps), ctypes.byref(sweeps))
    return Tc, ph, eps, rc


def channel_solve_point(mesh: Mesh, K, Vt, c, p_list, wp_kind=0):
    """Point-resolvent channel-solve at each momentum of p_list (fm^-1, inside
    the mesh): (Tc [nE,K,K] complex fm^2, ph [nE,3] degrees, rc)."""
    Vt = _f64(Vt)
    n_terms = Vt.shape[0]
    c = _f64(np.zeros(max(n_terms - 1, 1)) if c is None else c)
    p_list = _f64(np.atleast_1d(p_list))
    nE = p_list.shape[0]
    Tc = np.zeros((nE, K, K), dtype=np.complex128)
    ph = np.zeros((nE, 3))
    rc = lib().or_channel_solve_point(mesh.N, _d(mesh.kb), wp_kind, K, n_terms, _d(Vt), _d(c), nE, _d(p_list),
                                      Tc.ctypes.data_as(_dp), _d(ph))
    return Tc, ph, rc


def mi_kmatrix(gen, gp, ch, n_terms, c, p, NQ=96, cmap=1.0):
    K = 2 if ch[4] else 1
    gp = _f64(gp)
    c = _f64(np.zeros(max(n_terms - 1, 1)) if c is None else c)
    Km = np.zeros(K * K)
    rc = lib().or_mi_kmatrix(gen, _d(gp), *[int(v) for v in ch], n_terms, _d(c), NQ, cmap, float(p), _d(Km))
    if rc != 0:
        raise RuntimeError("singular MI system")
    return Km.reshape(K, K)


def batch(channels, meshes, Vts, coeffs, e_lab, wp_kind=0, n_threads=0, mode=AVG_FREE_BIN, frac=0.5):
    """Every (sample, channel) solve plus interpolation and sigma_tot.

    channels: list of 6-tuples (s, J, l, lp, coupled, tz); meshes: one Mesh per
    channel; Vts: one (n_terms, n, n) array per channel; coeffs: (S, n_terms-1).
    mode: AVG_FREE_BIN, AVG_SWP_INDEX or POINT (T and phases at each energy).
    Returns (t_out [S,ch,E,2,2] complex, delta [S,ch,E,3] deg, sigma [S,E] mb, rc)."""
    n_ch = len(channels)
    chdesc = np.ascontiguousarray(np.array(channels, dtype=np.int32).reshape(n_ch, 6))
    nwp = np.array([m.N for m in meshes], dtype=np.int32)
    kb_all = np.concatenate([m.kb for m in meshes])
    kb_off = np.cumsum([0] + [m.N + 1 for m in meshes[:-1]]).astype(np.int64)
    n_terms = Vts[0].shape[0]
    vt_all = np.concatenate([_f64(v).reshape(-1) for v in Vts])
    vt_off = np.cumsum([0] + [v.size for v in Vts[:-1]]).astype(np.int64)
    coeffs = _f64(np.asarray(coeffs).reshape(-1, max(n_terms - 1, 1)))
    S = coeffs.shape[0]
    e_lab = _f64(e_lab)
    nE = e_lab.shape[0]
    t_out = np.zeros((S, n_ch, nE, 2, 2), dtype=np.complex128)
    delta = np.zeros((S, n_ch, nE, 3))
    sigma = np.zeros((S, nE))
    args = (n_ch, _i(chdesc), _i(nwp), kb_off.ctypes.data_as(_lp), _d(kb_all), wp_kind, n_terms,
            vt_off.ctypes.data_as(_lp), _d(vt_all), S, _d(coeffs), nE, _d(e_lab), int(mode))
    outs = (t_out.ctypes.data_as(_dp), _d(delta), _d(sigma), int(n_threads))
    if frac == 0.5:
        rc = lib().or_batch(*args, *outs)
    else:  # interpolation point at fraction frac of each bin (Sec. 5.1.1)
        rc = lib().or_batch_ip(*args, float(frac), *outs)
    return t_out, delta, sigma, rc


def interp_phase_tlab(e_int, ph, K, e):
    e_int = _f64(e_int)
    ph = _f64(ph)
    out = np.zeros(3)
    lib().or_interp_phase_tlab(e_int.shape[0], _d(e_int), _d(ph), K, float(e), _d(out))
    return out


def mi_batch(channels, gen, gp, n_terms, coeffs, e_int, e_lab, NQ=96, cmap=1.0, n_threads=0):
    """MI at the interpolation energies e_int (MeV) for every (sample, channel),
    phases interpolated linearly in T_lab to e_lab, and sigma_tot.
    Returns (K [S,ch,n_I,2,2], delta [S,ch,E,3] deg, sigma [S,E] mb, rc)."""
    n_ch = len(channels)
    chdesc = np.ascontiguousarray(np.array(channels, dtype=np.int32).reshape(n_ch, 6))
    coeffs = _f64(np.asarray(coeffs).reshape(-1, max(n_terms - 1, 1)))
    S = coeffs.shape[0]
    e_int = _f64(e_int)
    e_lab = _f64(e_lab)
    nI, nE = e_int.shape[0], e_lab.shape[0]
    k_out = np.zeros((S, n_ch, nI, 2, 2))
    delta = np.zeros((S, n_ch, nE, 3))
    sigma = np.zeros((S, nE))
    rc = lib().or_mi_batch(n_ch, _i(chdesc), int(gen), _d(_f64(gp)), n_terms, S, _d(coeffs), NQ, float(cmap), nI,
                           _d(e_int), nE, _d(e_lab), _d(k_out), _d(delta), _d(sigma), int(n_threads))
    return k_out, delta, sigma, rc


def cg(j1, m1, j2, m2, J, M) -> float:
    return lib().or_cg(j1, m1, j2, m2, J, M)


def ylm(l, m, theta) -> float:
    return lib().or_ylm(l, m, float(theta))


def saclay(channels, ph, p, theta, want_m=False):
    """Saclay amplitudes [n_theta, 5] complex (fm), dsigma/dOmega [n_theta]
    (mb/sr) and optionally the 4 x 4 M-matrices, from the phases ph [n_ch, 3]
    (degrees) of the np channels at momentum p."""
    n_ch = len(channels)
    chdesc = np.ascontiguousarray(np.array(channels, dtype=np.int32).reshape(n_ch, 6))
    ph = _f64(ph)
    theta = _f64(np.atleast_1d(theta))
    nt = theta.shape[0]
    ab = np.zeros((nt, 5), dtype=np.complex128)
    ds = np.zeros(nt)
    M = np.zeros((nt, 4, 4), dtype=np.complex128) if want_m else None
    lib().or_saclay(n_ch, _i(chdesc), _d(ph), float(p), nt, _d(theta), ab.ctypes.data_as(_dp), _d(ds),
                    M.ctypes.data_as(_dp) if want_m else None)
    return (ab, ds, M) if want_m else (ab, ds)


def max_threads() -> int:
    return lib().or_max_threads()
