"""The paper-literal state: one wavefunction per initial particle identity (test infrastructure only).

Sec. 3.2 keeps NBeam[THETA][PHI][PARTICLE] with PARTICLE in {nu_e, nu_x, nubar_e, nubar_x} (or all
three flavours each), every beam holding the complex amplitudes of Eq. psi.  Here psi has shape
[2 (nu, nubar), n_flavor (initial flavour alpha), N_u, N_E, n_flavor (components)], the flux matrix
is summed over alpha exactly as printed in Sec. 2,

    F = sum_alpha (L/<E>)_alpha f_alpha dE psi_alpha psi_alpha^dag
        - (L/<E>)_alphabar fbar_alpha dE [psibar_alpha psibar_alpha^dag]^*,

and every update is psi -> exp(-i H dl) psi with the propagator of Eq. U.  The commutator-free
Lie RK4 scheme of ``oracle.integrate.cf4_step`` is applied to these wavefunctions; it only ever
multiplies the state by propagators, so the density matrices psi psi^dag it produces must equal
those of the reduced electron-flavour form (``Bulb`` + ``cf4_step``) up to rounding.
"""
from __future__ import annotations

import numpy as np

from .expm import propagator


def initial_wavefunctions(bulb) -> np.ndarray:
    """Sec. 3.4: psi_nu_alpha(R) = psibar_nu_alpha(R) = unit vector of flavour alpha."""
    n, Nu, NE = bulb.n, len(bulb.grid.u), len(bulb.grid.E)
    psi = np.zeros((2, n, Nu, NE, n), dtype=np.complex128)
    for a in range(n):
        psi[:, a, :, :, a] = 1.0
    return psi


def flux_from_wavefunctions(bulb, psi: np.ndarray) -> np.ndarray:
    N = bulb.grid.N                                        # [2, n, N_E]
    rho = psi[..., :, None] * np.conj(psi[..., None, :])   # [2, n, N_u, N_E, n, n]
    w_nu = N[0][:, None, :, None, None]
    w_nubar = N[1][:, None, :, None, None]
    return (w_nu * rho[0]).sum(axis=0) - np.conj((w_nubar * rho[1]).sum(axis=0))


def generators(bulb, r: float, psi: np.ndarray):
    F = flux_from_wavefunctions(bulb, psi)
    H, Hbar = bulb.hamiltonians_from_flux(r, F)
    inv_c = (1.0 / bulb.cos_theta(r))[:, None, None, None]
    return H * inv_c, Hbar * inv_c                         # [N_u, N_E, n, n] each


def apply(Gnu, Gbar, psi: np.ndarray) -> np.ndarray:
    """psi -> exp(-i G) psi for every initial flavour, nu with G and nubar with Gbar."""
    Unu, Ubar = propagator(Gnu), propagator(Gbar)
    out = np.empty_like(psi)
    out[0] = (Unu[None] @ psi[0][..., None])[..., 0]
    out[1] = (Ubar[None] @ psi[1][..., None])[..., 0]
    return out


def cf4_step(bulb, r: float, psi: np.ndarray, h: float) -> np.ndarray:
    """The commutator-free Lie RK4 of ``oracle.integrate`` acting on wavefunctions."""
    G1 = generators(bulb, r, psi)
    p2 = apply(0.5 * h * G1[0], 0.5 * h * G1[1], psi)
    G2 = generators(bulb, r + 0.5 * h, p2)
    p3 = apply(0.5 * h * G2[0], 0.5 * h * G2[1], psi)
    G3 = generators(bulb, r + 0.5 * h, p3)
    p4 = apply(h * G3[0] - 0.5 * h * G1[0], h * G3[1] - 0.5 * h * G1[1], p2)
    G4 = generators(bulb, r + h, p4)
    first = apply(h * (G1[0] / 4 + G2[0] / 6 + G3[0] / 6 - G4[0] / 12),
                  h * (G1[1] / 4 + G2[1] / 6 + G3[1] / 6 - G4[1] / 12), psi)
    return apply(h * (-G1[0] / 12 + G2[0] / 6 + G3[0] / 6 + G4[0] / 4),
                 h * (-G1[1] / 12 + G2[1] / 6 + G3[1] / 6 + G4[1] / 4), first)


def electron_density_matrices(psi: np.ndarray) -> np.ndarray:
    """stack(P, Pbar) of the electron-initial wavefunctions, comparable to the reduced form."""
    e = psi[:, 0]
    return e[..., :, None] * np.conj(e[..., None, :])
