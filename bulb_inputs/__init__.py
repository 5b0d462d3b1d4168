"""Seeded synthetic inputs for the neutrino bulb model (shared by the oracle and the CUDA path).

This module only *generates inputs*: random numbers, emission spectra binned into per-bin number
luminosities, and the named workloads.  It holds none of the method's arithmetic (no Hamiltonian,
no moments, no integrator): those live separately in ``oracle/`` and in the CUDA library, and
neither side imports the other.

Physics of the inputs (paper Sec. 2, the flux matrix F_alpha and its prefactors L/<E> f(E)):

* each flavour is emitted with energy luminosity ``L`` (erg/s), mean energy ``<E>`` (MeV) and a
  normalised spectrum ``f(E)``; the paper leaves ``f`` open, we use a Fermi-Dirac shape with
  degeneracy parameter ``eta = 3`` whose temperature reproduces ``<E>``;
* energies are cut into equal-width bins (paper Sec. 3.2, ``E_CNT`` equal energy intervals) and the
  spectrum is sampled at bin midpoints and renormalised so that ``sum_k f(E_k) dE = 1``;
* the per-bin number luminosity handed to both sides is ``N_k = (L / <E>) f(E_k) dE`` in 1/s.

Random draws use SplitMix64 (to seed) feeding xoshiro256** (Blackman & Vigna, 2018), both written
here from their published definitions, so any language can reproduce the same stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1
MEV_TO_ERG = 1.602176634e-6  # exact (SI 2019): 1 MeV in erg


# ----------------------------------------------------------------------------------------------
# Counter-free PRNG: SplitMix64 -> xoshiro256**
# ----------------------------------------------------------------------------------------------
class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014), used to expand one 64-bit seed into a state."""

    def __init__(self, seed: int):
        self.x = seed & MASK64

    def next(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & MASK64
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Xoshiro256ss:
    """xoshiro256** 1.0 (Blackman & Vigna 2018) seeded through SplitMix64."""

    def __init__(self, seed: int):
        sm = SplitMix64(seed)
        self.s = [sm.next() for _ in range(4)]

    def next_u64(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on {lo, ..., hi} (inclusive), by rejection to avoid modulo bias."""
        span = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            v = self.next_u64()
            if v < limit:
                return lo + v % span


# ----------------------------------------------------------------------------------------------
# Spectra
# ----------------------------------------------------------------------------------------------
def _fermi_integral(n: int, eta: float) -> float:
    """Complete Fermi-Dirac integral F_n(eta) = int_0^inf x^n / (exp(x - eta) + 1) dx."""
    from scipy.integrate import quad

    val, _ = quad(lambda x: x**n / (math.exp(x - eta) + 1.0) if x - eta < 700 else 0.0,
                  0.0, eta + 200.0, limit=400, epsabs=0.0, epsrel=1e-13)
    return val


def fermi_dirac_temperature(mean_E: float, eta: float = 3.0) -> float:
    """Temperature T (MeV) for which a Fermi-Dirac spectrum E^2/(exp(E/T-eta)+1) has mean <E>."""
    return mean_E * _fermi_integral(2, eta) / _fermi_integral(3, eta)


def energy_bins(n_energy: int, E_min: float, E_max: float):
    """Equal-width energy bins (paper Sec. 3.2): returns (midpoints, width)."""
    dE = (E_max - E_min) / n_energy
    mids = E_min + (np.arange(n_energy, dtype=np.float64) + 0.5) * dE
    return mids, dE


def binned_spectrum(n_energy: int, E_min: float, E_max: float, mean_E: float, eta: float = 3.0):
    """Fermi-Dirac spectrum sampled at bin midpoints, renormalised so sum_k f_k dE = 1."""
    E, dE = energy_bins(n_energy, E_min, E_max)
    T = fermi_dirac_temperature(mean_E, eta)
    x = np.minimum(E / T - eta, 700.0)
    f = E**2 / (np.exp(x) + 1.0)
    f = f / (f.sum() * dE)
    return f, dE


def number_luminosity_bins(n_flavor: int, n_energy: int, E_min: float, E_max: float,
                           L_erg_s, mean_E_MeV, eta: float = 3.0,
                           nue_weights: Optional[np.ndarray] = None) -> np.ndarray:
    """Per-bin number luminosities N[species, flavour, k] in 1/s.

    ``L_erg_s`` and ``mean_E_MeV`` are dicts keyed by 'nue', 'nuebar', 'nux', 'nuxbar'.  For three
    flavours the mu and tau flavours both carry the 'nux'/'nuxbar' spectra.  ``nue_weights`` (length
    n_energy) multiplies the nu_e bins (the per-energy spectral weights of the adjoint workload).
    """
    out = np.zeros((2, n_flavor, n_energy), dtype=np.float64)
    keys = {0: ("nue", "nux"), 1: ("nuebar", "nuxbar")}
    for sp in (0, 1):
        ke, kx = keys[sp]
        for fl in range(n_flavor):
            key = ke if fl == 0 else kx
            f, dE = binned_spectrum(n_energy, E_min, E_max, mean_E_MeV[key], eta)
            n_tot = L_erg_s[key] / (mean_E_MeV[key] * MEV_TO_ERG)
            out[sp, fl] = n_tot * f * dE
    if nue_weights is not None:
        out[0, 0] *= np.asarray(nue_weights, dtype=np.float64)
    return out


# ----------------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------------
@dataclass
class Workload:
    """One bulb-model problem: sizes, mixing, matter, spectra parameters, radial range."""
    name: str
    n_flavor: int = 2
    n_energy: int = 64
    n_angle: int = 32
    E_min: float = 1.0
    E_max: float = 60.0
    R_km: float = 11.0
    dm2: tuple = (-2.4e-3, 0.0)          # 2f: dm2[0]; 3f: (dm2_21, dm2_31)
    theta: tuple = (0.1, 0.0, 0.0)       # 2f: theta_v; 3f: (theta12, theta13, theta23)
    L: dict = field(default_factory=lambda: {"nue": 1e51, "nuebar": 1e51, "nux": 1e51, "nuxbar": 1e51})
    meanE: dict = field(default_factory=lambda: {"nue": 11.0, "nuebar": 16.0, "nux": 25.0, "nuxbar": 25.0})
    eta: float = 3.0
    matter: str = "none"                 # none | power_law | constant | table
    rho0_gcc: float = 1e7
    r_ref_km: float = 100.0
    power: float = 3.0
    Ye: float = 0.5
    lambda_const: float = 0.0
    matter_table_r: Optional[list] = None        # matter == "table": radii (km), increasing
    matter_table_lambda: Optional[list] = None   # and sqrt(2) G_F n_e there (1/km), > 0
    r0: float = 11.0
    r1: float = 200.0
    integrator: str = "rk4"              # rk4 | dp45 | lie_rk4
    n_steps: int = 0                     # fixed-step count (0 => adaptive)
    precision: str = "fp64"              # fp64 | mixed
    rtol: float = 1e-9
    atol: float = 1e-9
    h0: float = 1e-4
    nue_weights: Optional[list] = None

    @property
    def n_beams(self) -> int:
        return 2 * self.n_angle * self.n_energy

    def spectra(self) -> np.ndarray:
        w = None if self.nue_weights is None else np.asarray(self.nue_weights)
        return number_luminosity_bins(self.n_flavor, self.n_energy, self.E_min, self.E_max,
                                      self.L, self.meanE, self.eta, w)

    def to_dict(self):
        return asdict(self)


def workload_2f_small_fp64() -> Workload:
    """2-flavour multi-angle bulb, FP64: 64 E x 32 u x (nu, nubar) = 4096 beams, inverted
    dm2 = 2.4e-3 eV^2, theta_v = 0.1, L = 1e51 erg/s per flavour, R = 11 km, no matter, fixed-step
    RK4, r 11 -> 200 km in 2000 steps."""
    return Workload(name="bulb2f_64E_32u_fp64_rk4", n_energy=64, n_angle=32, r0=11.0, r1=200.0,
                    integrator="rk4", n_steps=2000)


def workload_3f_fp64(dm2_31: float = 2.4e-3) -> Workload:
    """3-flavour multi-angle bulb, FP64: 256 E x 512 u x (nu, nubar) = 262144 beams, matter
    n_e ~ r^-3 (Ye = 0.5, 1e7 g/cm^3 at 100 km), adaptive RK45, r 11 -> 1000 km."""
    return Workload(name=f"bulb3f_256E_512u_fp64_dp45_{'NH' if dm2_31 > 0 else 'IH'}", n_flavor=3,
                    n_energy=256, n_angle=512, dm2=(7.5e-5, dm2_31), theta=(0.59, 0.15, 0.785),
                    matter="power_law", r0=11.0, r1=1000.0, integrator="dp45", rtol=1e-9, atol=1e-9)


def workload_2f_large(precision: str = "mixed") -> Workload:
    """2-flavour large multi-angle bulb: 1000 E x 2000 u x (nu, nubar) = 4,000,000 beams, spectra
    and mixing as the small case plus the r^-3 matter profile, adaptive RK45, r 11 -> 500 km."""
    tol = 1e-6 if precision == "mixed" else 1e-9
    return Workload(name=f"bulb2f_1000E_2000u_{precision}_dp45", n_energy=1000, n_angle=2000,
                    matter="power_law", r0=11.0, r1=500.0, integrator="dp45", precision=precision,
                    rtol=tol, atol=tol)


def workload_adjoint() -> Workload:
    """Adjoint workload: 2-flavour bulb, 200 E x 400 u x (nu, nubar) = 160000 beams, FP64, fixed
    RK4, 5000 steps, r 11 -> 300 km."""
    return Workload(name="bulb2f_200E_400u_fp64_rk4_adjoint", n_energy=200, n_angle=400,
                    r0=11.0, r1=300.0, integrator="rk4", n_steps=5000)


BATCH_SEED = 0x5EED0003


def batched_workloads(n_instances: int = 64, seed: int = BATCH_SEED,
                      n_energy_range=(50, 500), n_angle_range=(100, 1500),
                      r1: float = 300.0) -> List[Workload]:
    """64 independent 2-flavour bulb instances of uneven sizes drawn from one xoshiro256** stream.

    Per instance, in this order: n_energy ~ U{50..500}, n_angle ~ U{100..1500}, one luminosity
    L ~ log-uniform[1e50, 1e52] erg/s applied to every flavour, hierarchy normal/inverted with
    probability 1/2 each, theta_v ~ U[0.01, 0.2].  Mixed precision, adaptive RK45, r 11 -> r1 km,
    r^-3 matter as the large case.
    """
    rng = Xoshiro256ss(seed)
    out = []
    for i in range(n_instances):
        ne = rng.randint(*n_energy_range)
        nu = rng.randint(*n_angle_range)
        L = 10.0 ** (50.0 + 2.0 * rng.uniform())
        inverted = rng.uniform() < 0.5
        th = 0.01 + 0.19 * rng.uniform()
        out.append(Workload(name=f"batch{i}", n_energy=ne, n_angle=nu,
                            dm2=(-2.4e-3 if inverted else 2.4e-3, 0.0), theta=(th, 0.0, 0.0),
                            L={"nue": L, "nuebar": L, "nux": L, "nuxbar": L},
                            matter="power_law", r0=11.0, r1=r1, integrator="dp45",
                            precision="mixed", rtol=1e-6, atol=1e-6))
    return out


def random_unit_states(n_flavor: int, n_beams: int, seed: int) -> np.ndarray:
    """Random pure flavour states for teacher-forced single-step checks.

    Returns complex wavefunctions psi[b, n_flavor] with unit norm, drawn from a seeded xoshiro
    stream through numpy's Generator seeded by it (reproducible on every platform).
    """
    rng = np.random.Generator(np.random.PCG64(Xoshiro256ss(seed).next_u64()))
    z = rng.standard_normal((n_beams, n_flavor)) + 1j * rng.standard_normal((n_beams, n_flavor))
    return z / np.linalg.norm(z, axis=1, keepdims=True)


def coherent_unit_states(n_flavor: int, n_beams: int, seed: int, spread: float = 0.3) -> np.ndarray:
    """Random pure states clustered around one common state (1, 0.4, [0.2]) / norm: every beam
    carries the same flavour coherence up to a random spread, so the angular moments are of
    the order of the total weight (unlike independent random states, whose moments cancel)."""
    base = np.array([1.0, 0.4, 0.2][:n_flavor], dtype=np.complex128)
    z = base[None, :] + spread * random_unit_states(n_flavor, n_beams, seed)
    return z / np.linalg.norm(z, axis=1, keepdims=True)
