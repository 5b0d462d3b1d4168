"""Bulb-model physics in the paper's matrix form (arXiv:1912.10596, Sec. 2).  FP64, numpy.

Test infrastructure only (see ``oracle/__init__``).

Units: r and R in km, E in MeV, every Hamiltonian entry in 1/km.

State.  For every beam (angle bin j, energy bin k) the oracle keeps the density matrix of the
wavefunction that started as an electron-flavour neutrino, P = psi_nue psi_nue^dagger, and of the
one that started as an electron-flavour antineutrino, Pbar = psibar_nue psibar_nue^dagger, exactly
as in the paper's flux matrix F_alpha (Sec. 2).  Wavefunctions of the other initial flavours stay
orthogonal to the electron one under unitary evolution, so the sum of their projectors is I - P
(and I - Pbar); with equal mu and tau spectra (the inputs guarantee this) the flux matrix needs no
further state.  ``oracle.four_psi`` keeps all four wavefunctions explicitly and checks this.

Readings of the paper taken here, where it is silent or ambiguous:

* Eq. Hnu integrates d(cos theta') over the directions populated at radius r, cos theta' in
  [sqrt(1 - R^2/r^2), 1]; in the equal-u bins of Sec. 3.2 (u = sin^2 theta_R) this measure is
  d(cos theta') = R^2 / (2 r^2 cos theta') du.
* The local polar angle follows from straight-line propagation, r sin theta = R sin theta_R, so
  cos theta(r) = sqrt(1 - u R^2 / r^2) (the geometry described in the caption of Fig. 1).
* The electron density is n_e = Ye rho / m_u with rho(r) = rho0 (r_ref / r)^power.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

# --- constants (CODATA 2018 / SI 2019) -------------------------------------------------------
G_F_GEV2 = 1.1663787e-5          # Fermi constant G_F/(hbar c)^3 in GeV^-2 (paper: ~1.166e-5)
HBARC_MEV_FM = 197.3269804       # hbar c in MeV fm (exact in SI 2019 units)
HBARC_GEV_KM = HBARC_MEV_FM * 1e-3 * 1e-18   # GeV km
HBARC_EV_KM = HBARC_MEV_FM * 1e6 * 1e-18     # eV km
C_KM_S = 299792.458              # speed of light, km/s
M_U_G = 1.66053906660e-24        # atomic mass unit, g
CM3_PER_KM3 = 1e15


def sqrt2_GF_kmi_per_km3() -> float:
    """sqrt(2) G_F times a number density of 1 per km^3, expressed in 1/km.

    sqrt(2) G_F n has dimension of energy in natural units; dividing by hbar c turns it into an
    inverse length: sqrt(2) G_F (hbar c)^3 n / (hbar c) = sqrt(2) G_F (hbar c)^2 n.
    """
    return math.sqrt(2.0) * G_F_GEV2 * HBARC_GEV_KM**2


# --- Hamiltonians ------------------------------------------------------------------------------
def pmns(theta12: float, theta13: float, theta23: float) -> np.ndarray:
    """Real three-flavour mixing matrix U = R23 R13 R12 (delta_CP = 0)."""
    c12, s12 = math.cos(theta12), math.sin(theta12)
    c13, s13 = math.cos(theta13), math.sin(theta13)
    c23, s23 = math.cos(theta23), math.sin(theta23)
    R12 = np.array([[c12, s12, 0], [-s12, c12, 0], [0, 0, 1]], dtype=np.float64)
    R13 = np.array([[c13, 0, s13], [0, 1, 0], [-s13, 0, c13]], dtype=np.float64)
    R23 = np.array([[1, 0, 0], [0, c23, s23], [0, -s23, c23]], dtype=np.float64)
    return R23 @ R13 @ R12


def vacuum_hamiltonian(E_MeV: np.ndarray, n_flavor: int, dm2, theta) -> np.ndarray:
    """H_vac(E) for every energy bin, shape [N_E, n, n] complex (1/km).

    Two flavours (Sec. 2): H_vac = dm2/(4E) [[-cos 2 theta_v, sin 2 theta_v],
                                             [ sin 2 theta_v, cos 2 theta_v]].
    Three flavours (the paper only says it can be done): H_vac = U diag(0, dm2_21, dm2_31) U^T / (2E).
    dm2 in eV^2, E in MeV; dm2/(2E) [1/km] = dm2 / (2 E 1e6 hbar c[eV km]).
    """
    E = np.asarray(E_MeV, dtype=np.float64)
    inv2E = 1.0 / (2.0 * E * 1e6 * HBARC_EV_KM)          # 1/(2E) in 1/(eV^2 km)
    if n_flavor == 2:
        th = theta[0]
        M = np.array([[-math.cos(2 * th), math.sin(2 * th)],
                      [math.sin(2 * th), math.cos(2 * th)]], dtype=np.float64)
        H = (dm2[0] * inv2E / 2.0)[:, None, None] * M[None]
        return H.astype(np.complex128)
    U = pmns(*theta)
    M21 = U @ np.diag([0.0, 1.0, 0.0]) @ U.T
    M31 = U @ np.diag([0.0, 0.0, 1.0]) @ U.T
    H = (dm2[0] * inv2E)[:, None, None] * M21[None] + (dm2[1] * inv2E)[:, None, None] * M31[None]
    return H.astype(np.complex128)


def electron_density_km3(r_km: float, wl) -> float:
    """n_e(r) in 1/km^3 for the power-law profile rho(r) = rho0 (r_ref/r)^power."""
    rho = wl.rho0_gcc * (wl.r_ref_km / r_km) ** wl.power
    return wl.Ye * rho / M_U_G * CM3_PER_KM3


def matter_table_strength(r_km: float, r_tab, lam_tab) -> float:
    """sqrt(2) G_F n_e(r) from a table (r_i, lambda_i), r increasing, lambda > 0: linear in
    (log r, log lambda) between neighbouring points (each interval a power law, so a table sampled
    from rho0 (r_ref/r)^p reproduces it exactly), the end values outside the table."""
    r_tab = np.asarray(r_tab, dtype=np.float64)
    lam_tab = np.asarray(lam_tab, dtype=np.float64)
    if r_km <= r_tab[0]:
        return float(lam_tab[0])
    if r_km >= r_tab[-1]:
        return float(lam_tab[-1])
    i = int(np.searchsorted(r_tab, r_km, side="right")) - 1
    t = math.log(r_km / r_tab[i]) / math.log(r_tab[i + 1] / r_tab[i])
    return float(lam_tab[i] * (lam_tab[i + 1] / lam_tab[i]) ** t)


def matter_strength(r_km: float, wl) -> float:
    """sqrt(2) G_F n_e(r) in 1/km (the coefficient of diag(1, 0[, 0]) in H_mat, Sec. 2)."""
    if wl.matter == "none":
        return 0.0
    if wl.matter == "constant":
        return float(wl.lambda_const)
    if wl.matter == "table":
        return matter_table_strength(r_km, wl.matter_table_r, wl.matter_table_lambda)
    return sqrt2_GF_kmi_per_km3() * electron_density_km3(r_km, wl)


def e_projector(n: int) -> np.ndarray:
    D = np.zeros((n, n), dtype=np.complex128)
    D[0, 0] = 1.0
    return D


# --- discretisation ------------------------------------------------------------------------------
@dataclass
class Grid:
    """Energy and angle bins of one problem (Sec. 3.2: equal-width E bins, equal-width u bins)."""
    E: np.ndarray          # [N_E] MeV, bin midpoints
    u: np.ndarray          # [N_u] u = sin^2 theta_R, bin positions
    du: np.ndarray         # [N_u] bin weights (sum 1 for a full [0,1] cover)
    N: np.ndarray          # [2, n_flavor, N_E] per-bin number luminosities (1/s), nu then nubar

    @staticmethod
    def from_workload(wl, u=None, du=None, N=None) -> "Grid":
        dE = (wl.E_max - wl.E_min) / wl.n_energy
        E = wl.E_min + (np.arange(wl.n_energy) + 0.5) * dE
        if u is None:
            du = np.full(wl.n_angle, 1.0 / wl.n_angle)
            u = (np.arange(wl.n_angle) + 0.5) / wl.n_angle
        if N is None:
            N = wl.spectra()
        return Grid(E=E, u=np.asarray(u, dtype=np.float64), du=np.asarray(du, dtype=np.float64),
                    N=np.asarray(N, dtype=np.float64))


def cos_theta(u: np.ndarray, R: float, r: float) -> np.ndarray:
    """cos theta of a beam emitted with sin^2 theta_R = u, seen at radius r (Fig. 1 geometry)."""
    return np.sqrt(1.0 - u * (R * R) / (r * r))


class Bulb:
    """Right-hand side of Eq. eom for all beams, in the paper's matrix form.

    geometry = "bulb": the stationary, spherically symmetric bulb model of Sec. 2.
    geometry = "homogeneous": a test geometry with every beam radial (cos theta = 1 in the
    derivative) and an isotropic nu-nu potential H_nunu = mu0 * sum_b F_b / S, where
    S = sum of all per-bin number luminosities; it serves the synchronisation check.
    geometry = "single_angle": the single-angle approximation of the bulb model: every beam moves
    along the radial trajectory (cos theta = 1 in the derivative) and the nu-nu potential carries
    the geometric factor of Eq. Hnu integrated over emission uniform in u = sin^2 theta_R,
    int_0^1 du (1/sqrt(1 - u x) - 1) = (1 - sqrt(1 - x))^2 / x, x = R^2/r^2, applied to the
    angle-summed flux: H_nunu = sqrt(2) G_F/(4 pi r^2 c) ((1 - sqrt(1 - x))^2 / x) sum_j du_j F_j.
    """

    def __init__(self, wl, grid: Grid | None = None, geometry: str = "bulb", mu0: float = 0.0):
        self.wl = wl
        self.grid = grid if grid is not None else Grid.from_workload(wl)
        self.n = wl.n_flavor
        self.geometry = geometry
        self.mu0 = mu0
        self.Hvac = vacuum_hamiltonian(self.grid.E, self.n, wl.dm2, wl.theta)   # [N_E, n, n]
        self.Pe = e_projector(self.n)
        N = self.grid.N
        if self.n == 3:
            assert np.array_equal(N[:, 1], N[:, 2]), "mu and tau spectra must coincide"
        self.S = float(N.sum())
        # prefactor sqrt(2) G_F / (2 pi R^2 c) of Eq. Hnu, in 1/km per (1/s) of number luminosity
        self.K = sqrt2_GF_kmi_per_km3() / (2.0 * math.pi * wl.R_km**2 * C_KM_S)

    # geometry -----------------------------------------------------------------------------------
    def cos_theta(self, r: float) -> np.ndarray:
        if self.geometry in ("homogeneous", "single_angle"):
            return np.ones_like(self.grid.u)
        return cos_theta(self.grid.u, self.wl.R_km, r)

    # flux matrices (Sec. 2) ------------------------------------------------------------------------
    def flux_matrices(self, P: np.ndarray, Pbar: np.ndarray) -> np.ndarray:
        """F[j, k] = sum_alpha (L/<E>) f dE psi psi^dag - (Lbar/<Ebar>) fbar dE [psibar psibar^dag]^*.

        With the electron-flavour projector P and the other flavours' projectors summing to I - P:
        F = N_e P + N_x (I - P) - (Nbar_e Pbar + Nbar_x (I - Pbar))^*.
        """
        N = self.grid.N
        I = np.eye(self.n, dtype=np.complex128)
        Ne, Nx = N[0, 0][None, :, None, None], N[0, 1][None, :, None, None]
        Nbe, Nbx = N[1, 0][None, :, None, None], N[1, 1][None, :, None, None]
        nu = Ne * P + Nx * (I - P)
        nubar = Nbe * Pbar + Nbx * (I - Pbar)
        return nu - np.conj(nubar)

    def angular_moments(self, r: float, P: np.ndarray, Pbar: np.ndarray):
        """Phi_1 = sum_alpha int d(cos th') int dE F and Phi_c (same with a cos th' weight), Eq. F.

        The d(cos th') measure at radius r is R^2/(2 r^2 cos th') du (reading of Eq. Hnu).
        """
        F = self.flux_matrices(P, Pbar)                      # [N_u, N_E, n, n]
        Fsum = F.sum(axis=1)                                 # energy integral
        c = self.cos_theta(r)
        w = self.grid.du * (self.wl.R_km**2) / (2.0 * r * r * c)
        Phi1 = np.einsum("j,jab->ab", w, Fsum)
        Phic = np.einsum("j,jab->ab", w * c, Fsum)
        return Phi1, Phic

    def nunu_from_flux(self, r: float, F: np.ndarray) -> np.ndarray:
        """H_nunu for every angle bin, [N_u, n, n] (Eq. Hnu with 1 - v.v' = 1 - cos th cos th'),
        from the flux matrices F[j, k] of all beams."""
        if self.geometry == "homogeneous":
            Ftot = np.einsum("j,jkab->ab", self.grid.du, F)
            H = self.mu0 * Ftot / self.S
            return np.broadcast_to(H, (len(self.grid.u), self.n, self.n))
        if self.geometry == "single_angle":
            x = (self.wl.R_km / r) ** 2
            geo = (1.0 - math.sqrt(1.0 - x)) ** 2 / x
            Ftot = np.einsum("j,jkab->ab", self.grid.du, F)
            H = self.K * self.wl.R_km**2 / (2.0 * r * r) * geo * Ftot
            return np.broadcast_to(H, (len(self.grid.u), self.n, self.n))
        Fsum = F.sum(axis=1)                                 # energy integral
        c = self.cos_theta(r)
        w = self.grid.du * (self.wl.R_km**2) / (2.0 * r * r * c)   # d(cos th') at radius r
        Phi1 = np.einsum("j,jab->ab", w, Fsum)
        Phic = np.einsum("j,jab->ab", w * c, Fsum)
        return self.K * (Phi1[None] - c[:, None, None] * Phic[None])

    def nunu_hamiltonian(self, r: float, P: np.ndarray, Pbar: np.ndarray) -> np.ndarray:
        return self.nunu_from_flux(r, self.flux_matrices(P, Pbar))

    def hamiltonians_from_flux(self, r: float, F: np.ndarray):
        """(H, Hbar) per beam [N_u, N_E, n, n]: H = H_vac + H_mat + H_nunu and
        Hbar = H_vac - H_mat - H_nunu^* (Eq. eom)."""
        lam = matter_strength(r, self.wl)
        Hnn = self.nunu_from_flux(r, F)[:, None]                            # [N_u, 1, n, n]
        Hv = self.Hvac[None]                                                # [1, N_E, n, n]
        Hm = lam * self.Pe
        H = Hv + Hm + Hnn
        Hbar = Hv - Hm - np.conj(Hnn)
        return H, Hbar

    def hamiltonians(self, r: float, P: np.ndarray, Pbar: np.ndarray):
        """(H, Hbar) per beam from the electron-flavour projectors."""
        return self.hamiltonians_from_flux(r, self.flux_matrices(P, Pbar))

    def rhs(self, r: float, Y: np.ndarray) -> np.ndarray:
        """dY/dr for Y = stack(P, Pbar): i cos theta dP/dr = [H, P] (Eq. eom, psi psi^dag form)."""
        P, Pbar = Y[0], Y[1]
        H, Hbar = self.hamiltonians(r, P, Pbar)
        inv_c = (1.0 / self.cos_theta(r))[:, None, None, None]
        dP = -1j * (H @ P - P @ H) * inv_c
        dPbar = -1j * (Hbar @ Pbar - Pbar @ Hbar) * inv_c
        return np.stack([dP, dPbar])

    def generators(self, r: float, Y: np.ndarray):
        """(H/cos theta, Hbar/cos theta) per beam: dY/dr = -i [G, Y] with G these matrices."""
        P, Pbar = Y[0], Y[1]
        H, Hbar = self.hamiltonians(r, P, Pbar)
        inv_c = (1.0 / self.cos_theta(r))[:, None, None, None]
        return np.stack([H * inv_c, Hbar * inv_c])

    # initial condition (Sec. 3.4) ---------------------------------------------------------------
    def initial_state(self) -> np.ndarray:
        """psi_nue = psibar_nue = (1, 0[, 0]) at r = R, so P = Pbar = diag(1, 0[, 0])."""
        Nu, NE, n = len(self.grid.u), len(self.grid.E), self.n
        P = np.broadcast_to(self.Pe, (Nu, NE, n, n)).copy()
        return np.stack([P, P.copy()])

    # observables ---------------------------------------------------------------------------------
    def survival_probability(self, Y: np.ndarray) -> np.ndarray:
        """P_ee = |a_e|^2 = P[0, 0] per beam, [2, N_u, N_E] (nu, nubar)."""
        return Y[..., 0, 0].real.copy()

    def mean_survival(self, Y: np.ndarray) -> float:
        """Number-flux weighted nu_e survival probability over all (j, k) nu beams."""
        W = self.grid.du[:, None] * self.grid.N[0, 0][None, :]
        return float((W * Y[0, ..., 0, 0].real).sum() / W.sum())

    def flux_spectra(self, Y: np.ndarray) -> np.ndarray:
        """Number-flux energy spectra [2, n, N_E] of every flavour (the nu_e flux of the Sec. 3.4
        validation figure): Phi_a(E_k) = sum_j du_j [N_e,k P_aa + N_x,k (1 - P_aa)], P the density
        matrix of the beam that started as electron flavour (nu: P, nubar: Pbar), the beams that
        started as the other flavours carrying 1 - P_aa into flavour a by unitarity."""
        N, du = self.grid.N, self.grid.du
        out = np.zeros((2, self.n, len(self.grid.E)))
        for s in range(2):
            diag = np.einsum("jkaa->ajk", Y[s]).real                       # [n, N_u, N_E]
            out[s] = np.einsum("j,ajk->ak", du, N[s, 0][None, None, :] * diag
                               + N[s, 1][None, None, :] * (1.0 - diag))
        return out

    def moment_matrices(self, r: float, Y: np.ndarray):
        """Traceless parts of J0 = sum_b du F_b / cos th_b and J1 = sum_b du F_b (matrix form).

        These equal (2 r^2 / R^2) Phi_1 and (2 r^2 / R^2) Phi_c minus their traces; they are the two
        beam-independent reductions that the nu-nu potential needs at every evaluation.
        """
        Phi1, Phic = self.angular_moments(r, Y[0], Y[1])
        s = 2.0 * r * r / self.wl.R_km**2
        J0, J1 = s * Phi1, s * Phic
        I = np.eye(self.n)
        J0 = J0 - np.trace(J0) / self.n * I
        J1 = J1 - np.trace(J1) / self.n * I
        return J0, J1
