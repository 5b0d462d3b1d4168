"""Observables of the bulb model at chosen radii, written as plain NumPy archives.

What the paper's validation figure shows (Sec. 3.4): the electron-flavour survival probability
P_ee = |a_e|^2 as a function of neutrino energy E and emission angle theta_R, and the energy
spectra of the number flux of each flavour, at a radius r.  Both come from the library
(xflat_pee, xflat_flux_spectra); this module only arranges them on the (theta_R, E) grid and
writes one .npz file per radius.
"""
from __future__ import annotations

import numpy as np

from . import xflat


def energy_bins(cfg) -> np.ndarray:
    """Midpoints of the equal-width energy bins of a config (MeV)."""
    dE = (cfg.E_max_MeV - cfg.E_min_MeV) / cfg.n_energy
    return cfg.E_min_MeV + (np.arange(cfg.n_energy) + 0.5) * dE


def snapshot(solver: "xflat.Solver", inst: int = 0, u_bins=None) -> dict:
    """P_ee(theta_R, E) maps of neutrinos and antineutrinos, flux spectra of every flavour and the
    radius, for instance `inst` of a solver.  u_bins: the angle-bin positions u = sin^2 theta_R the
    spectra were set with (None: the default equal bins at midpoints)."""
    cfg = solver.cfgs[inst]
    na, ne = cfg.n_angle, cfg.n_energy
    nphi = cfg.n_phi if cfg.n_phi >= 2 else 1
    u = (np.arange(na) + 0.5) / na if u_bins is None else np.asarray(u_bins, dtype=np.float64)
    pee, mean = solver.pee(inst=inst)
    shape = (na, ne) if nphi == 1 else (na, nphi, ne)      # extended bulb model: azimuthal bins too
    half = na * nphi * ne
    snap = {
        "r_km": np.float64(solver.stats(inst).r_km),
        "E_MeV": energy_bins(cfg),
        "theta_R_rad": np.arcsin(np.sqrt(u)),
        "pee_nu": pee[:half].reshape(shape),
        "pee_nubar": pee[half:].reshape(shape),
        "pee_mean_nu": np.float64(mean),
        "flux": solver.flux_spectra(inst),           # [species, flavour, energy]
    }
    if nphi > 1:
        snap["phi_rad"] = 2.0 * np.pi * (np.arange(nphi) + 0.5) / nphi
    return snap


def save(path: str, snap: dict) -> None:
    np.savez(path, **snap)


def evolve_with_snapshots(solver: "xflat.Solver", r0: float, radii, prefix: str, inst: int = 0,
                          u_bins=None) -> list:
    """Advance from r0 through the given radii (ascending), writing `{prefix}_r{r}km.npz` at each;
    returns the file names.  Every instance of the solver advances to the same radii."""
    files = []
    r = r0
    for rr in sorted(radii):
        if rr > r:
            solver.evolve(r, rr)
            r = rr
        name = f"{prefix}_r{rr:g}km.npz"
        save(name, snapshot(solver, inst, u_bins))
        files.append(name)
    return files
