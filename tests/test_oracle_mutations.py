"""The oracle's pins catch plausible mistakes: each case plants one mistake in the oracle (on the
CPU, by patching one of its functions for the duration of the case) and checks that the pins
named beside it fail.  The mistakes are the kind a transcription of the paper's equations makes:
a flipped sign, a dropped factor, a missing term, a wrong coefficient.
"""
import math
import warnings

import numpy as np
import pytest

import test_oracle_adjoint as adj_pins
import test_oracle_extended as ext_pins
import test_oracle_pins as pins
from oracle import adjoint as adj
from oracle import extended as ex
from oracle import integrate as ig
from oracle import physics as ph

Bulb = ph.Bulb
_rhs, _hff, _nff = Bulb.rhs, Bulb.hamiltonians_from_flux, Bulb.nunu_from_flux
_vac, _matter = ph.vacuum_hamiltonian, ph.matter_strength

PINS = {
    "vacuum_rk4": lambda: pins.test_vacuum_closed_form("rk4"),
    "vacuum_dp45": lambda: pins.test_vacuum_closed_form("dp45"),
    "msw_normal": lambda: pins.test_constant_matter_closed_form(1.0),
    "msw_inverted": lambda: pins.test_constant_matter_closed_form(-1.0),
    "antineutrino": pins.test_antineutrino_conjugated_convention,
    "single_angle": pins.test_single_angle_geometric_factor,
    "lepton_number": pins.test_lepton_number_invariant,
    "synchronised": pins.test_synchronised_precession,
    "four_psi": lambda: pins.test_four_wavefunctions_equal_reduced_state(2),
    "three_to_two": pins.test_three_flavours_reduce_to_two,
    "library_rk": pins.test_runge_kutta_agrees_with_library_integrator,
    "trace_purity": pins.test_runge_kutta_trace_exact_purity_to_order,
    "order_rk4": lambda: pins.test_convergence_order("rk4", 4),
    "order_dp5": lambda: pins.test_convergence_order("dp5", 5),
    "controller": pins.test_adaptive_controller_meets_tolerance,
    "vacuum_3f": pins.test_three_flavour_vacuum_closed_form,
    "power_law": pins.test_power_law_density_profile,
    "lie_richardson": pins.test_lie_richardson_estimate_is_the_local_error,
    "lie_tolerance": pins.test_lie_adaptive_meets_tolerance,
    "single_angle_bulb": pins.test_single_angle_geometry_is_the_bulb_on_the_radial_beam,
    "matter_table": pins.test_matter_table_reproduces_a_power_law,
}


# --- the planted mistakes ---------------------------------------------------------------------------
def vacuum_sign(mp):
    """H_vac with the opposite sign (Delta m^2 sign convention slip)."""
    mp.setattr(ph, "vacuum_hamiltonian", lambda *a, **k: -_vac(*a, **k))


def no_path_factor(mp):
    """d/dr instead of d/dl: the 1/cos theta of Eq. eom dropped."""
    mp.setattr(Bulb, "rhs", lambda self, r, Y: _rhs(self, r, Y) * self.cos_theta(r)[None, :, None, None, None])


def antineutrino_matter_sign(mp):
    """Antineutrinos given +H_mat instead of -H_mat."""
    def hff(self, r, F):
        H, Hbar = _hff(self, r, F)
        return H, Hbar + 2.0 * ph.matter_strength(r, self.wl) * self.Pe
    mp.setattr(Bulb, "hamiltonians_from_flux", hff)


def commutator_order(mp):
    """-i [rho, H] instead of -i [H, rho]."""
    mp.setattr(Bulb, "rhs", lambda self, r, Y: -_rhs(self, r, Y))


def antineutrino_nunu_not_conjugated(mp):
    """Antineutrinos given -H_nunu instead of -H_nunu^*."""
    def hff(self, r, F):
        H, Hbar = _hff(self, r, F)
        Hnn = self.nunu_from_flux(r, F)[:, None]
        return H, Hbar + np.conj(Hnn) - Hnn
    mp.setattr(Bulb, "hamiltonians_from_flux", hff)


def _nunu(self, r, F, measure_cos=True, beam_cos=True):
    Fsum = F.sum(axis=1)
    c = self.cos_theta(r)
    w = self.grid.du * self.wl.R_km**2 / (2.0 * r * r * (c if measure_cos else 1.0))
    Phi1 = np.einsum("j,jab->ab", w, Fsum)
    Phic = np.einsum("j,jab->ab", w * c, Fsum)
    cb = c[:, None, None] if beam_cos else np.ones((len(c), 1, 1))
    return self.K * (Phi1[None] - cb * Phic[None])


def nunu_without_beam_cosine(mp):
    """1 - v.v' with the beam's own cos theta dropped: Phi_1 - Phi_c for every beam."""
    mp.setattr(Bulb, "nunu_from_flux",
               lambda self, r, F: _nff(self, r, F) if self.geometry == "homogeneous" else _nunu(self, r, F, beam_cos=False))


def measure_without_cosine(mp):
    """d(cos theta') = R^2/(2 r^2) du, the 1/cos theta' of the u-bin measure dropped."""
    mp.setattr(Bulb, "nunu_from_flux",
               lambda self, r, F: _nff(self, r, F) if self.geometry == "homogeneous" else _nunu(self, r, F, measure_cos=False))


def flux_antineutrino_sign(mp):
    """F = rho_nu + rho_nubar^* instead of rho_nu - rho_nubar^*."""
    def flux(self, P, Pbar):
        N = self.grid.N
        I = np.eye(self.n, dtype=np.complex128)
        Ne, Nx = N[0, 0][None, :, None, None], N[0, 1][None, :, None, None]
        Nbe, Nbx = N[1, 0][None, :, None, None], N[1, 1][None, :, None, None]
        return (Ne * P + Nx * (I - P)) + np.conj(Nbe * Pbar + Nbx * (I - Pbar))
    mp.setattr(Bulb, "flux_matrices", flux)


def matter_factor_two(mp):
    """lambda(r) twice too large (a factor slip in sqrt(2) G_F n_e)."""
    mp.setattr(ph, "matter_strength", lambda r, wl: 2.0 * _matter(r, wl))


def cos_theta_unsquared(mp):
    """cos theta = sqrt(1 - u R/r): the square of R/r dropped."""
    mp.setattr(ph, "cos_theta", lambda u, R, r: np.sqrt(1.0 - u * R / r))


def rk4_equal_weights(mp):
    """RK4 with weights 1/4 instead of 1/6, 1/3, 1/3, 1/6."""
    def rk4(f, r, Y, h):
        k1 = f(r, Y)
        k2 = f(r + 0.5 * h, Y + (0.5 * h) * k1)
        k3 = f(r + 0.5 * h, Y + (0.5 * h) * k2)
        k4 = f(r + h, Y + h * k3)
        return Y + h * (k1 + k2 + k3 + k4) / 4
    mp.setattr(ig, "rk4_step", rk4)


def dormand_prince_weight(mp):
    """b_3 = 500/1112 instead of 500/1113 in the Dormand-Prince tableau."""
    b = ig.DP_B.copy()
    b[2] = 500.0 / 1112.0
    mp.setattr(ig, "DP_B", b)


def pmns_reversed_product(mp):
    """Mixing matrix U = R12 R13 R23 instead of R23 R13 R12."""
    def pmns(t12, t13, t23):
        c12, s12, c13, s13 = math.cos(t12), math.sin(t12), math.cos(t13), math.sin(t13)
        c23, s23 = math.cos(t23), math.sin(t23)
        R12 = np.array([[c12, s12, 0], [-s12, c12, 0], [0, 0, 1]])
        R13 = np.array([[c13, 0, s13], [0, 1, 0], [-s13, 0, c13]])
        R23 = np.array([[1, 0, 0], [0, c23, s23], [0, -s23, c23]])
        return R12 @ R13 @ R23
    mp.setattr(ph, "pmns", pmns)


def mass_splittings_swapped(mp):
    """dm2_21 attached to the third mass state and dm2_31 to the second."""
    def vac(E, n, dm2, theta):
        return _vac(E, n, (dm2[1], dm2[0]) if n == 3 else dm2, theta)
    mp.setattr(ph, "vacuum_hamiltonian", vac)


def power_law_inverted(mp):
    """rho0 (r / r_ref)^power instead of rho0 (r_ref / r)^power."""
    def n_e(r, wl):
        return wl.Ye * wl.rho0_gcc * (r / wl.r_ref_km) ** wl.power / ph.M_U_G * ph.CM3_PER_KM3
    mp.setattr(ph, "electron_density_km3", n_e)


def richardson_divisor(mp):
    """Richardson estimate divided by 2^5 - 1 (the order of the local error) instead of 2^4 - 1."""
    mp.setattr(ig, "RICHARDSON_DIV", 31.0)


def second_half_step_from_start(mp):
    """The second half step taken from the step's initial state instead of the first half step's."""
    def step(G, r, Y, h, G1=None):
        if G1 is None:
            G1 = G(r, Y)
        full = ig.cf4_step(G, r, Y, h, G1)
        ig.cf4_step(G, r, Y, 0.5 * h, G1)
        return ig.cf4_step(G, r + 0.5 * h, Y, 0.5 * h), full
    mp.setattr(ig, "lie_richardson_step", step)


def single_angle_factor_unsquared(mp):
    """Single-angle geometric factor (1 - sqrt(1 - x)) / x instead of (1 - sqrt(1 - x))^2 / x."""
    def nff(self, r, F):
        if self.geometry != "single_angle":
            return _nff(self, r, F)
        x = (self.wl.R_km / r) ** 2
        Ftot = np.einsum("j,jkab->ab", self.grid.du, F)
        H = self.K * self.wl.R_km**2 / (2.0 * r * r) * (1.0 - math.sqrt(1.0 - x)) / x * Ftot
        return np.broadcast_to(H, (len(self.grid.u), self.n, self.n))
    mp.setattr(Bulb, "nunu_from_flux", nff)


def matter_table_linear(mp):
    """Table interpolated linearly in (r, lambda) instead of as a power law per interval."""
    def tab(r, rt, lt):
        return float(np.interp(r, rt, lt))
    mp.setattr(ph, "matter_table_strength", tab)


CASES = [
    (vacuum_sign, ["msw_normal", "msw_inverted", "synchronised"]),
    (no_path_factor, ["vacuum_rk4", "antineutrino", "lepton_number"]),
    (antineutrino_matter_sign, ["msw_normal", "msw_inverted", "antineutrino"]),
    (commutator_order, ["antineutrino", "synchronised"]),
    (antineutrino_nunu_not_conjugated, ["antineutrino", "lepton_number", "synchronised"]),
    (nunu_without_beam_cosine, ["lepton_number"]),
    (measure_without_cosine, ["single_angle", "lepton_number"]),
    (flux_antineutrino_sign, ["synchronised", "four_psi"]),
    (matter_factor_two, ["msw_normal", "msw_inverted", "antineutrino"]),
    (cos_theta_unsquared, ["vacuum_rk4", "single_angle", "three_to_two", "trace_purity"]),
    (rk4_equal_weights, ["vacuum_rk4", "library_rk", "order_rk4", "trace_purity"]),
    (dormand_prince_weight, ["vacuum_dp45", "order_dp5", "controller"]),
    (pmns_reversed_product, ["vacuum_3f"]),
    (mass_splittings_swapped, ["vacuum_3f"]),
    (power_law_inverted, ["power_law"]),
    (richardson_divisor, ["lie_richardson"]),
    (second_half_step_from_start, ["lie_tolerance"]),
    (single_angle_factor_unsquared, ["single_angle_bulb"]),
    (matter_table_linear, ["matter_table"]),
]


@pytest.mark.parametrize("mistake,catchers", CASES, ids=[m.__name__ for m, _ in CASES])
def test_pins_catch_planted_mistake(monkeypatch, mistake, catchers):
    mistake(monkeypatch)
    missed = []
    for name in catchers:
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            try:
                PINS[name]()
            except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
                continue
        missed.append(name)
    assert not missed, f"{mistake.__name__} passed the pins {missed}"


# --- the extended bulb model (azimuthal bins, Eq. F with the measure of Eq. int-v) ---------------------
EXT_PINS = {
    "axial_symmetry": ext_pins.test_axial_symmetry_reduces_to_bulb,
    "shift_symmetry": ext_pins.test_azimuthal_shift_symmetry,
    "cos_phi_moment": ext_pins.test_cos_phi_modulation_moments,
    "sin_phi_moment": ext_pins.test_sin_phi_modulation_moments,
}


def _ext_moments(self, r, F, per_bin=True, sc_weight="cos"):
    Fsum = F.sum(axis=2)
    c = self.cos_theta(r)
    s = np.sqrt(1.0 - c * c)
    w = self.grid.du * self.wl.R_km**2 / (2.0 * r * r * c) / (self.n_phi if per_bin else 1)
    cp, sp = np.cos(self.phi), np.sin(self.phi)
    Phi1 = np.einsum("j,jpab->ab", w, Fsum)
    Phic = np.einsum("j,jpab->ab", w * c, Fsum)
    Phisc = np.einsum("j,p,jpab->ab", w * s, cp if sc_weight == "cos" else sp, Fsum)
    Phiss = np.einsum("j,p,jpab->ab", w * s, sp, Fsum)
    return Phi1, Phic, Phisc, Phiss


def azimuthal_measure_without_bins(mp):
    """The phi integral without its 1/(2 pi): weights du instead of du / n_phi."""
    mp.setattr(ex.ExtendedBulb, "moments", lambda self, r, F: _ext_moments(self, r, F, per_bin=False))


def cos_moment_with_sine_weight(mp):
    """Phi_sc weighted by sin phi' instead of cos phi'."""
    mp.setattr(ex.ExtendedBulb, "moments", lambda self, r, F: _ext_moments(self, r, F, sc_weight="sin"))


def sine_term_sign(mp):
    """sin th (cos phi Phi_sc - sin phi Phi_ss): the sign of the sin phi sin phi' term flipped."""
    def nunu(self, r, F):
        Phi1, Phic, Phisc, Phiss = self.moments(r, F)
        c = self.cos_theta(r)
        s = np.sqrt(1.0 - c * c)
        cp, sp = np.cos(self.phi), np.sin(self.phi)
        return self.K * (Phi1[None, None] - c[:, None, None, None] * Phic[None, None]
                         - s[:, None, None, None] * (cp[None, :, None, None] * Phisc[None, None]
                                                     - sp[None, :, None, None] * Phiss[None, None]))
    mp.setattr(ex.ExtendedBulb, "nunu", nunu)


EXT_CASES = [
    (azimuthal_measure_without_bins, ["axial_symmetry"]),
    (cos_moment_with_sine_weight, ["cos_phi_moment", "sin_phi_moment"]),
    (sine_term_sign, ["shift_symmetry"]),
]


@pytest.mark.parametrize("mistake,catchers", EXT_CASES, ids=[m.__name__ for m, _ in EXT_CASES])
def test_extended_pins_catch_planted_mistake(monkeypatch, mistake, catchers):
    mistake(monkeypatch)
    missed = []
    for name in catchers:
        try:
            EXT_PINS[name]()
        except AssertionError:
            continue
        missed.append(name)
    assert not missed, f"{mistake.__name__} passed the pins {missed}"


# --- the discrete adjoint ------------------------------------------------------------------------------
_vjp = adj.rhs_vjp


def adjoint_mixing_angle_sign(mp):
    """d(H_vac)/d(theta_v) with the wrong sign in the adjoint of one right-hand-side evaluation."""
    def vjp(*a, **k):
        G_Y, G_N, G_th = _vjp(*a, **k)
        return G_Y, G_N, -G_th
    mp.setattr(adj, "rhs_vjp", vjp)


def adjoint_luminosity_transposed(mp):
    """The luminosity gradient of nu and nubar swapped."""
    def vjp(*a, **k):
        G_Y, G_N, G_th = _vjp(*a, **k)
        return G_Y, G_N[::-1].copy(), G_th
    mp.setattr(adj, "rhs_vjp", vjp)


@pytest.mark.parametrize("mistake", [adjoint_mixing_angle_sign, adjoint_luminosity_transposed],
                         ids=["adjoint_mixing_angle_sign", "adjoint_luminosity_transposed"])
def test_adjoint_pin_catches_planted_mistake(monkeypatch, mistake):
    mistake(monkeypatch)
    kw, win, n = adj_pins.CASES[0]
    with pytest.raises(AssertionError):
        adj_pins.test_adjoint_matches_central_differences(kw, win, n)
