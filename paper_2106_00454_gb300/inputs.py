"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds workload descriptions only -- channel lists, mesh
parameters, potential-generator parameters, seeded coefficient samples and
energy lists.  It contains none of the method's arithmetic, so both sides of
every parity test can take their inputs from it.

Workloads (seed 20210601, numpy PCG64):
  1. Yamaguchi rank-1 potential in 1S0, N_WP = 32, 64 lab energies 1..350 MeV.
  2. Synthetic regulated Yukawa + contact potential, all 20 channels J <= 6,
     N_WP = 100 (coupled blocks 200 x 200), one sample (V0), T at every bin.
  3. Batched: 4096 samples c ~ N(0, I_14) times per-term scales, 15 channels
     (the 14 np channels J <= 4 plus a T_z = +-1 copy of 1S0), N_WP per channel
     drawn once from {40, 64, 100}, 128 lab energies 1..350 MeV.
  4. Mixed precision: the generator of workload 2 with N_WP = 150, 16384 samples.
  5. Serving: Poisson arrivals, each request c ~ N(0, I_14), 16..256 sorted
     energies in [1, 350] MeV, N_WP in {32, 64, 128, 256}, 15 channels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED = 20210601

# Mesh parameters: the tan^t map with t = 2 and alpha = 100 MeV (as a momentum,
# 100 / 197.3269804 fm^-1), capped at k_max = 8 fm^-1; 8 Gauss-Legendre points per bin.
MESH_ALPHA_FM = 100.0 / 197.3269804
MESH_T = 2.0
MESH_KMAX_FM = 8.0
MESH_Q = 8
MESH_KIND_CAPPED = 0
MESH_KIND_LITERAL = 1
WP_MOMENTUM = 0
WP_ENERGY = 1

# Potential generators.
GEN_YAMAGUCHI = 0
GEN_YUKAWA = 1
GEN_FINE = -1  # caller-supplied fine-grid values

# Yamaguchi: V(p',p) = lambda g(p') g(p), g = 1/(p^2 + beta^2), beta = 1.2 fm^-1,
# lambda fixed so that the scattering length is -20 fm (fm^2).
YAMAGUCHI_PARAMS = np.array([-0.42682555403147876, 1.2])

# Synthetic regulated Yukawa + contact generator (19 numbers):
#  [0:3]  Yukawa masses m1, m2, m3 = 0.7, 3.0, 6.0 fm^-1
#  [3]    Gaussian regulator cutoff Lambda = 4 fm^-1, R = exp(-(p^2+p'^2)/Lambda^2)
#  [4:18] strengths of the 14 unit terms in V0: central(m1), spin-spin(m1),
#         central(m2), spin-orbit(m2), tensor(m3), C~1S0, C~3S1, C1S0, C3S1,
#         C3P0, C1P1, C3P1, C3P2, Ceps1.  The two S-wave LO contacts were chosen
#         so that 1S0 has a = -20 fm and 3S1-3D1 one bound state at -2.2246 MeV.
#  [18]   extra LO contact in the T_z = +-1 copy of 1S0 (a = -18.9 fm).
YUKAWA_PARAMS = np.array([
    0.7, 3.0, 6.0, 4.0,
    -0.04, -0.005, 0.1, 0.05, -0.6, 0.14271152298364703, 0.20845583187866887,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.010128443909215662,
])
N_TERMS_YUKAWA = 15  # V0 + 14 unit terms

# Per-term sample scales s_a: each makes s_a * max_ch ||V_a||_F about 5% of
# max_ch ||V0||_F on the N_WP = 64 mesh.  Samples are c_a * s_a with c ~ N(0, 1).
TERM_SCALE = np.array([
    7.41e-3, 2.53e-3, 2.01e-2, 3.91e-3, 1.11e-1, 1.10e-2, 1.10e-2,
    3.99e-4, 3.99e-4, 9.19e-4, 9.19e-4, 9.19e-4, 9.19e-4, 5.07e-4,
])


@dataclasses.dataclass(frozen=True)
class Channel:
    """Partial-wave channel (s, J, l, l', coupled, T_z).

    Coupled channels carry l = J-1, l' = J+1 and stand for the 2x2 block
    pair; T_z = 0 is np.  Only T_z = 0 channels enter the np total cross
    section."""
    s: int
    J: int
    l: int
    lp: int
    coupled: int
    tz: int = 0

    def astuple(self):
        return (self.s, self.J, self.l, self.lp, self.coupled, self.tz)

    @property
    def K(self) -> int:
        return 2 if self.coupled else 1

    @property
    def name(self) -> str:
        L = "SPDFGHIKLMN"
        if self.coupled:
            return f"3{L[self.J - 1]}{self.J}-3{L[self.J + 1]}{self.J}"
        tag = f"{2 * self.s + 1}{L[self.l]}{self.J}"
        return tag + ("(tz)" if self.tz else "")


def np_channels(jmax: int, extra_1s0_tz: bool = False) -> list[Channel]:
    """The np partial waves with J <= jmax: 1J, 3J (uncoupled), 3(J-1)-3(J+1)."""
    out = []
    for J in range(jmax + 1):
        out.append(Channel(0, J, J, J, 0))
        if J == 0:
            out.append(Channel(1, 0, 1, 1, 0))
            continue
        out.append(Channel(1, J, J, J, 0))
        out.append(Channel(1, J, J - 1, J + 1, 1))
    if extra_1s0_tz:
        out.append(Channel(0, 0, 0, 0, 0, 1))
    return out


def lab_energies(n: int, lo: float = 1.0, hi: float = 350.0) -> np.ndarray:
    return np.linspace(lo, hi, n)


def chebyshev_energies(n: int, e_max: float = 350.0) -> np.ndarray:
    """n lab energies of a Chebyshev distribution on (0, e_max] (MeV, ascending):
    e_max (1 - cos((2k - 1) pi / (2n))) / 2, k = 1..n -- the interpolation
    energies of the MI comparison."""
    k = np.arange(1, n + 1)
    return 0.5 * e_max * (1.0 - np.cos((2 * k - 1) * np.pi / (2 * n)))


def coefficient_samples(n_samples: int, seed: int = SEED, scaled: bool = True) -> np.ndarray:
    """(n_samples, 14) coefficients c_a * s_a with c ~ N(0, I_14)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((n_samples, 14))
    return c * TERM_SCALE if scaled else c


@dataclasses.dataclass
class Workload:
    name: str
    channels: list
    nwp: list            # N_WP per channel
    gen: int
    gen_params: np.ndarray
    n_terms: int
    coeffs: np.ndarray   # (S, n_terms-1)
    e_lab: np.ndarray    # MeV, ascending
    mesh_kind: int = MESH_KIND_CAPPED
    wp_kind: int = WP_MOMENTUM
    alpha: float = MESH_ALPHA_FM
    t: float = MESH_T
    kmax: float = MESH_KMAX_FM
    Q: int = MESH_Q

    @property
    def n_samples(self) -> int:
        return self.coeffs.shape[0]


def workload_yamaguchi(n_wp: int = 32, n_e: int = 64) -> Workload:
    """Workload 1: plain WPCD, 1S0 Yamaguchi, N_WP = 32, 64 energies."""
    return Workload("yamaguchi_1s0_nwp32", [Channel(0, 0, 0, 0, 0)], [n_wp], GEN_YAMAGUCHI,
                    YAMAGUCHI_PARAMS.copy(), 1, np.zeros((1, 0)), lab_energies(n_e))


def workload_all_channels(n_wp: int = 100, jmax: int = 6, n_e: int = 0) -> Workload:
    """Workload 2: all channels J <= 6, N_WP = 100, one sample (V0).

    With n_e = 0 the energies are those of every bin midpoint that lies in
    1..350 MeV -- callers that need the exact midpoints take them from the mesh."""
    chs = np_channels(jmax)
    e = lab_energies(n_e) if n_e else lab_energies(100)
    return Workload(f"all_channels_J{jmax}_nwp{n_wp}", chs, [n_wp] * len(chs), GEN_YUKAWA,
                    YUKAWA_PARAMS.copy(), N_TERMS_YUKAWA, np.zeros((1, 14)), e)


def workload_batched(n_samples: int = 4096, n_e: int = 128, seed: int = SEED,
                     nwp_choices=(40, 64, 100), sample_seed: int | None = None) -> Workload:
    """Workload 3: 15 channels J <= 4, N_WP per channel from {40, 64, 100}.

    `seed` fixes the channel set's N_WP draw (and, by default, the parameter
    samples); `sample_seed` draws only the parameter samples, so that shards of
    one job (one per GPU) solve the same channels on different samples."""
    chs = np_channels(4, extra_1s0_tz=True)
    rng = np.random.default_rng(seed + 1)
    nwp = [int(x) for x in rng.choice(np.array(nwp_choices), size=len(chs))]
    cseed = seed if sample_seed is None else sample_seed
    return Workload(f"batched_{n_samples}x15ch", chs, nwp, GEN_YUKAWA, YUKAWA_PARAMS.copy(),
                    N_TERMS_YUKAWA, coefficient_samples(n_samples, cseed), lab_energies(n_e))


def workload_mixed(n_samples: int = 16384, n_wp: int = 150, n_e: int = 128, seed: int = SEED,
                   sample_seed: int | None = None) -> Workload:
    """Workload 4: 20 channels J <= 6, N_WP = 150, 16384 samples.

    `sample_seed` draws the parameter samples of one shard of a multi-GPU job
    (default: `seed`, the single-GPU workload)."""
    chs = np_channels(6)
    cseed = seed if sample_seed is None else sample_seed
    return Workload(f"mixed_{n_samples}x20ch_nwp{n_wp}", chs, [n_wp] * len(chs), GEN_YUKAWA,
                    YUKAWA_PARAMS.copy(), N_TERMS_YUKAWA, coefficient_samples(n_samples, cseed),
                    lab_energies(n_e))


@dataclasses.dataclass
class Request:
    arrival_s: float
    coeffs: np.ndarray
    e_lab: np.ndarray
    n_wp: int


def serving_requests(duration_s: float = 30.0, rate_hz: float = 2000.0, seed: int = SEED,
                     nwp_choices=(32, 64, 128, 256)) -> list[Request]:
    """Workload 5: Poisson arrivals of independent requests."""
    rng = np.random.default_rng(seed + 5)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        n_e = int(rng.integers(16, 257))
        e = np.sort(rng.uniform(1.0, 350.0, n_e))
        out.append(Request(t, rng.standard_normal(14) * TERM_SCALE, e, int(rng.choice(np.array(nwp_choices)))))
    return out
