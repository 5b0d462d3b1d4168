"""The extended bulb model of Sec. 2 in the paper's matrix form (test infrastructure only).

The bulb model assumes every beam's flavour state is axially symmetric around the radial
direction.  The extended bulb model drops that symmetry: a beam is labelled by its energy, its
polar angle (u = sin^2 theta_R bins, Sec. 3.2) and its azimuthal angle phi around the radial
direction, and Eq. Hnu takes the replacements of Eq. int-v,

    1 - v.v'  ->  1 - [cos th cos th' + sin th sin th' (cos phi cos phi' + sin phi sin phi')],
    int d(cos th')  ->  (1/2 pi) int dphi' int d(cos th'),

so the nu-nu potential of beam (th, phi) needs the four weighted integrals of Eq. F:
Phi_1, Phi_c (weight cos th), Phi_sc (sin th cos phi), Phi_ss (sin th sin phi), with

    H_nunu(th, phi) = K [Phi_1 - cos th Phi_c - sin th (cos phi Phi_sc + sin phi Phi_ss)].

Readings (as for the bulb model in ``oracle.physics``): d(cos th') over the populated directions
is R^2/(2 r^2 cos th') du; the phi integral carries the 1/(2 pi) of Eq. int-v (Eq. F prints dphi
without it; the two differ by a constant that Eq. int-v fixes); n_phi equal phi bins centred at
phi_p = 2 pi (p + 1/2) / n_phi.  State shape [2, N_u, n_phi, N_E, n, n] (nu P, nubar Pbar).
"""
from __future__ import annotations

import math

import numpy as np

from .physics import (Grid, cos_theta, e_projector, matter_strength, sqrt2_GF_kmi_per_km3,
                      vacuum_hamiltonian, C_KM_S)


class ExtendedBulb:
    def __init__(self, wl, n_phi: int, grid: Grid | None = None):
        self.wl = wl
        self.grid = grid if grid is not None else Grid.from_workload(wl)
        self.n = wl.n_flavor
        self.n_phi = n_phi
        self.phi = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
        self.Hvac = vacuum_hamiltonian(self.grid.E, self.n, wl.dm2, wl.theta)   # [N_E, n, n]
        self.Pe = e_projector(self.n)
        self.K = sqrt2_GF_kmi_per_km3() / (2.0 * math.pi * wl.R_km**2 * C_KM_S)

    def cos_theta(self, r: float) -> np.ndarray:
        return cos_theta(self.grid.u, self.wl.R_km, r)

    def flux_matrices(self, P: np.ndarray, Pbar: np.ndarray) -> np.ndarray:
        """F[j, p, k] = N_e P + N_x (I - P) - (Nbar_e Pbar + Nbar_x (I - Pbar))^* (Sec. 2)."""
        N = self.grid.N
        I = np.eye(self.n, dtype=np.complex128)
        sh = (None, None, slice(None), None, None)
        Ne, Nx, Nbe, Nbx = N[0, 0][sh], N[0, 1][sh], N[1, 0][sh], N[1, 1][sh]
        return (Ne * P + Nx * (I - P)) - np.conj(Nbe * Pbar + Nbx * (I - Pbar))

    def moments(self, r: float, F: np.ndarray):
        """Phi_1, Phi_c, Phi_sc, Phi_ss of Eq. F with the measure of Eq. int-v."""
        Fsum = F.sum(axis=2)                                   # energy integral, [N_u, n_phi, n, n]
        c = self.cos_theta(r)
        s = np.sqrt(1.0 - c * c)
        w = self.grid.du * (self.wl.R_km**2) / (2.0 * r * r * c) / self.n_phi   # d(cos th') dphi'/2pi
        cp, sp = np.cos(self.phi), np.sin(self.phi)
        Phi1 = np.einsum("j,jpab->ab", w, Fsum)
        Phic = np.einsum("j,jpab->ab", w * c, Fsum)
        Phisc = np.einsum("j,p,jpab->ab", w * s, cp, Fsum)
        Phiss = np.einsum("j,p,jpab->ab", w * s, sp, Fsum)
        return Phi1, Phic, Phisc, Phiss

    def nunu(self, r: float, F: np.ndarray) -> np.ndarray:
        """H_nunu of every direction (j, p), [N_u, n_phi, n, n]."""
        Phi1, Phic, Phisc, Phiss = self.moments(r, F)
        c = self.cos_theta(r)
        s = np.sqrt(1.0 - c * c)
        cp, sp = np.cos(self.phi), np.sin(self.phi)
        return self.K * (Phi1[None, None] - c[:, None, None, None] * Phic[None, None]
                         - s[:, None, None, None] * (cp[None, :, None, None] * Phisc[None, None]
                                                     + sp[None, :, None, None] * Phiss[None, None]))

    def hamiltonians(self, r: float, P: np.ndarray, Pbar: np.ndarray):
        lam = matter_strength(r, self.wl)
        Hnn = self.nunu(r, self.flux_matrices(P, Pbar))[:, :, None]       # [N_u, n_phi, 1, n, n]
        Hv = self.Hvac[None, None]
        H = Hv + lam * self.Pe + Hnn
        Hbar = Hv - lam * self.Pe - np.conj(Hnn)
        return H, Hbar

    def rhs(self, r: float, Y: np.ndarray) -> np.ndarray:
        P, Pbar = Y[0], Y[1]
        H, Hbar = self.hamiltonians(r, P, Pbar)
        inv_c = (1.0 / self.cos_theta(r))[:, None, None, None, None]
        return np.stack([-1j * (H @ P - P @ H) * inv_c, -1j * (Hbar @ Pbar - Pbar @ Hbar) * inv_c])

    def generators(self, r: float, Y: np.ndarray):
        P, Pbar = Y[0], Y[1]
        H, Hbar = self.hamiltonians(r, P, Pbar)
        inv_c = (1.0 / self.cos_theta(r))[:, None, None, None, None]
        return np.stack([H * inv_c, Hbar * inv_c])

    def initial_state(self) -> np.ndarray:
        Nu, NE = len(self.grid.u), len(self.grid.E)
        P = np.broadcast_to(self.Pe, (Nu, self.n_phi, NE, self.n, self.n)).copy()
        return np.stack([P, P.copy()])

    def moment_matrices(self, r: float, Y: np.ndarray):
        """Traceless parts of J0, J1, Jc, Js = (2 r^2 / R^2) (Phi_1, Phi_c, Phi_sc, Phi_ss)."""
        Phis = self.moments(r, self.flux_matrices(Y[0], Y[1]))
        sc = 2.0 * r * r / self.wl.R_km**2
        I = np.eye(self.n)
        return tuple(sc * M - np.trace(sc * M) / self.n * I for M in Phis)
