"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what it pins and the paper passage (or the mathematics) that fixes the expected
value.  A plausible mistake anywhere in the oracle (a dropped term, a wrong sign, a wrong unit, a
transposed operand, a wrong tableau entry) makes at least one of them fail.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm

from bulb_inputs import Workload, number_luminosity_bins, workload_2f_small_fp64
from oracle import physics as ph
from oracle import four_psi
from oracle.expm import two_flavor_propagator, hermitian_propagator
from oracle.integrate import (evolve_fixed, evolve_adaptive, cf4_step, rk4_step, dp45_step,
                              DP_A, DP_B, DP_BHAT, DP_C)
from oracle.physics import Bulb, Grid, cos_theta

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")
NO_L = {k: 0.0 for k in ("nue", "nuebar", "nux", "nuxbar")}


def golden(name):
    for line in open(GOLDEN):
        if line.startswith(name):
            return line.split()[1]
    raise KeyError(name)


def pee(Y):
    return Y[..., 0, 0].real


def bloch(M):
    """Bloch vector of the traceless part of 2x2 Hermitian matrices: M = (1/2) j . sigma + tr."""
    return np.stack([2 * M[..., 0, 1].real, -2 * M[..., 0, 1].imag,
                     (M[..., 0, 0] - M[..., 1, 1]).real], axis=-1)


# --- units and constants ------------------------------------------------------------------------
def test_fermi_constant_matches_paper():
    """Sec. 2 prints G_F ~ 1.166e-5 GeV^-2."""
    assert abs(ph.G_F_GEV2 - float(golden("G_F_GeV-2"))) < 0.0005e-5


def test_matter_potential_textbook_value():
    """sqrt(2) G_F n_e = 7.63e-14 eV per (Ye rho / g cm^-3): pins G_F, hbar c, m_u and km units."""
    wl = Workload(name="m", matter="constant")
    n_e = 1.0 / ph.M_U_G * ph.CM3_PER_KM3            # Ye rho = 1 g/cm^3, per km^3
    lam_kmi = ph.sqrt2_GF_kmi_per_km3() * n_e
    lam_eV = lam_kmi * ph.HBARC_EV_KM
    assert abs(lam_eV / float(golden("V_CC_eV_per_Ye_rho")) - 1) < 2e-3


def test_initial_condition_matches_paper():
    """Sec. 3.4: electron-flavour neutrinos and antineutrinos start as (1, 0)."""
    wl = Workload(name="ic", n_energy=3, n_angle=2)
    Y = Bulb(wl).initial_state()
    e = np.array([float(x) for x in golden("psi_nue_initial").split(",")])
    assert np.array_equal(Y[..., :, :].real, np.broadcast_to(np.outer(e, e), Y.shape))


# --- Eq. U -----------------------------------------------------------------------------------------
def test_eq_u_equals_matrix_exponential():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((50, 2, 2)) + 1j * rng.standard_normal((50, 2, 2))
    H = A + np.conj(np.swapaxes(A, -1, -2))
    dl = rng.uniform(0.0, 5.0, 50)
    U = two_flavor_propagator(H, dl)
    for i in range(50):
        assert np.abs(U[i] - expm(-1j * dl[i] * H[i])).max() < 1e-13
    # lambda = 0 (H proportional to the identity) is the degenerate case of Eq. U
    Hd = np.broadcast_to(np.eye(2) * 3.0, (1, 2, 2)).astype(complex)
    assert np.abs(two_flavor_propagator(Hd, 0.5)[0] - np.exp(-1.5j) * np.eye(2)).max() < 1e-15


def test_hermitian_exponential_equals_matrix_exponential():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 3, 3)) + 1j * rng.standard_normal((30, 3, 3))
    H = A + np.conj(np.swapaxes(A, -1, -2))
    U = hermitian_propagator(H, 0.3)
    for i in range(30):
        assert np.abs(U[i] - expm(-0.3j * H[i])).max() < 1e-13


# --- closed forms -----------------------------------------------------------------------------------
def _vacuum_pee(wl, grid, r, dm2, theta):
    """P_ee = 1 - sin^2 2theta sin^2(1.267 dm2 L/E) with the path length L of each beam (km),
    E in GeV; L = r cos theta(r) - R cos theta_R for straight-line propagation from R."""
    c = cos_theta(grid.u, wl.R_km, r)
    L = r * c - wl.R_km * np.sqrt(1.0 - grid.u)
    phase = float(golden("osc_phase_coeff")) * dm2 * L[:, None] / (grid.E[None, :] * 1e-3)
    return 1.0 - math.sin(2 * theta) ** 2 * np.sin(phase) ** 2


@pytest.mark.parametrize("method", ["rk4", "lie_rk4", "dp45"])
def test_vacuum_closed_form(method):
    """mu = lambda = 0: every beam oscillates as in vacuum along its own path length."""
    wl = Workload(name="vac", n_energy=7, n_angle=5, L=NO_L, dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0))
    b = Bulb(wl)
    Y0 = b.initial_state()
    if method == "dp45":
        Y, r, _ = evolve_adaptive(b, Y0, 11.0, 31.0, 1e-11, 1e-11, 1e-3)
    else:
        Y, _ = evolve_fixed(b, Y0, 11.0, 31.0, 4000, method)
    ref = _vacuum_pee(wl, b.grid, 31.0, 2.4e-3, 0.3)
    # the textbook 1.267 has four digits: the phase (up to ~30 rad) carries ~1e-4 relative error
    assert np.abs(pee(Y[0]) - ref).max() < 5e-3
    assert np.abs(pee(Y[1]) - ref).max() < 5e-3
    # with the exact coefficient 1/(4 hbar c) the agreement is at the integrator's accuracy
    exact = 1.0 / (4 * ph.HBARC_EV_KM * 1e6)       # dm2 L / (4 E) with E in MeV, L in km
    c = cos_theta(b.grid.u, wl.R_km, 31.0)
    L = 31.0 * c - wl.R_km * np.sqrt(1.0 - b.grid.u)
    ref2 = 1 - math.sin(0.6) ** 2 * np.sin(exact * 2.4e-3 * L[:, None] / b.grid.E[None, :]) ** 2
    assert np.abs(pee(Y[0]) - ref2).max() < 2e-9
    assert abs(exact / 1e3 / float(golden("osc_phase_coeff")) - 1) < 1e-3


def test_three_flavour_vacuum_closed_form():
    """mu = lambda = 0, three flavours with every mixing angle and both mass splittings non-zero:
    each beam's nu_e survival and nu_e -> nu_mu appearance follow the textbook vacuum formulas
      P_ee = 1 - 4 sum_{i<j} U_ei^2 U_ej^2 sin^2(dm2_ji L / 4E),
      P_emu = -4 sum_{i<j} U_ei U_mui U_ej U_muj sin^2(dm2_ji L / 4E)      (real U, delta_CP = 0)
    along the beam's path length L, with the e and mu rows of the mixing matrix written out from
    the standard parametrisation (PDG neutrino-mixing review): U_e = (c12 c13, s12 c13, s13),
    U_mu = (-s12 c23 - c12 s23 s13, c12 c23 - s12 s23 s13, s23 c13).  Pins the product order of
    the mixing matrix and which vacuum matrix carries which mass splitting."""
    th, dm = (0.59, 0.15, 0.785), (7.5e-5, 2.4e-3)
    wl = Workload(name="vac3", n_flavor=3, n_energy=6, n_angle=4, E_min=2.0, E_max=20.0, L=NO_L,
                  dm2=dm, theta=th)
    b = Bulb(wl)
    Y, _ = evolve_fixed(b, b.initial_state(), 11.0, 211.0, 2000, "lie_rk4")
    c12, s12 = math.cos(th[0]), math.sin(th[0])
    c13, s13 = math.cos(th[1]), math.sin(th[1])
    c23, s23 = math.cos(th[2]), math.sin(th[2])
    Ue = [c12 * c13, s12 * c13, s13]
    Um = [-s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13]
    m2 = [0.0, dm[0], dm[1]]
    g = b.grid
    L = 211.0 * cos_theta(g.u, 11.0, 211.0) - 11.0 * np.sqrt(1.0 - g.u)
    k = 1.0 / (4 * ph.HBARC_EV_KM * 1e6)             # dm2 L / (4 E): eV^2, km, MeV
    Pee, Pem = np.ones((4, 6)), np.zeros((4, 6))
    for i in range(3):
        for j in range(i + 1, 3):
            s2 = np.sin(k * (m2[j] - m2[i]) * L[:, None] / g.E[None, :]) ** 2
            Pee -= 4 * Ue[i] ** 2 * Ue[j] ** 2 * s2
            Pem -= 4 * Ue[i] * Um[i] * Ue[j] * Um[j] * s2
    assert Pee.min() < 0.5 and Pem.max() > 0.3        # strong three-flavour oscillation
    for s in range(2):                                 # antineutrinos: the same in vacuum (delta = 0)
        assert np.abs(Y[s, ..., 0, 0].real - Pee).max() < 1e-7
        assert np.abs(Y[s, ..., 1, 1].real - Pem).max() < 1e-7


def test_power_law_density_profile():
    """rho(r) = rho0 (r_ref / r)^power: at r_ref sqrt(2) G_F n_e is the textbook 7.63e-14 eV x Ye x
    rho0 (converted to 1/km with hbar c), and it falls by 2^power when r doubles."""
    for power in (3.0, 2.0):
        wl = Workload(name="pl", matter="power_law", rho0_gcc=1e7, r_ref_km=100.0, power=power, Ye=0.5)
        lam = ph.matter_strength(100.0, wl)
        want = float(golden("V_CC_eV_per_Ye_rho")) * 0.5 * 1e7 / ph.HBARC_EV_KM
        assert abs(lam / want - 1) < 2e-3
        assert abs(ph.matter_strength(200.0, wl) * 2.0**power / lam - 1) < 1e-14
        assert abs(ph.matter_strength(50.0, wl) / (lam * 2.0**power) - 1) < 1e-14


@pytest.mark.parametrize("sign", [+1.0, -1.0])
def test_constant_matter_closed_form(sign):
    """Constant lambda, mu = 0: MSW in uniform matter.  Neutrinos see +lambda, antineutrinos
    -lambda (Eq. eom), with Delta_m = sqrt((omega cos 2th - lambda)^2 + omega^2 sin^2 2th)."""
    dm2 = sign * 2.4e-3
    wl = Workload(name="msw", n_energy=6, n_angle=4, L=NO_L, dm2=(dm2, 0.0), theta=(0.15, 0, 0),
                  matter="constant", lambda_const=0.4)
    b = Bulb(wl)
    Y, _ = evolve_fixed(b, b.initial_state(), 11.0, 21.0, 1000, "lie_rk4")
    c = cos_theta(b.grid.u, wl.R_km, 21.0)
    L = 21.0 * c - wl.R_km * np.sqrt(1.0 - b.grid.u)
    omega = dm2 / (2 * b.grid.E * 1e6 * ph.HBARC_EV_KM)
    for species, lam in ((0, 0.4), (1, -0.4)):
        D = np.sqrt((omega * math.cos(0.3) - lam) ** 2 + (omega * math.sin(0.3)) ** 2)
        s2m = (omega * math.sin(0.3)) ** 2 / D**2
        ref = 1 - s2m[None, :] * np.sin(0.5 * D[None, :] * L[:, None]) ** 2
        assert np.abs(pee(Y[species]) - ref).max() < 1e-10


# --- equation structure -----------------------------------------------------------------------------
def test_antineutrino_conjugated_convention():
    """Evolving Pbar with Hbar = H_vac - H_mat - H_nunu^* is the same as evolving sigma = Pbar^*
    with -H_vac + H_mat + H_nunu (complex conjugate of Eq. eom, real H_vac and H_mat)."""
    wl = Workload(name="c", n_energy=4, n_angle=3, matter="constant", lambda_const=2.0)
    b = Bulb(wl)
    rng = np.random.default_rng(3)
    from bulb_inputs import random_unit_states
    psi = random_unit_states(2, 2 * 3 * 4, seed=11).reshape(2, 3, 4, 2)
    Y = psi[..., :, None] * np.conj(psi[..., None, :])
    r = 40.0
    dY = b.rhs(r, Y)
    Hnn = b.nunu_hamiltonian(r, Y[0], Y[1])[:, None]
    Hs = -b.Hvac[None] + 2.0 * b.Pe + Hnn
    sigma = np.conj(Y[1])
    dsigma = -1j * (Hs @ sigma - sigma @ Hs) / b.cos_theta(r)[:, None, None, None]
    assert np.abs(np.conj(dY[1]) - dsigma).max() < 1e-12 * np.abs(dsigma).max()


def test_single_angle_geometric_factor():
    """With every beam in the same state, H_nunu of a radial beam (cos th = 1) is proportional to
    int_0^1 du (1/sqrt(1 - u x) - 1) = (1 - sqrt(1 - x))^2 / x, x = R^2/r^2 (Eq. Hnu integrated
    in closed form); the midpoint u-bins converge to it at second order."""
    r = 22.0
    x = (11.0 / r) ** 2
    D_exact = (1 - math.sqrt(1 - x)) ** 2 / x
    errs = []
    for Nu in (16, 32, 64):
        wl = Workload(name="sa", n_energy=3, n_angle=Nu)
        u = np.concatenate([(np.arange(Nu) + 0.5) / Nu, [0.0]])       # add a radial probe bin
        du = np.concatenate([np.full(Nu, 1.0 / Nu), [0.0]])
        b = Bulb(wl, grid=Grid.from_workload(wl, u=u, du=du))
        Y = b.initial_state()
        Y[..., 0, 1] = 0.3
        Y[..., 1, 0] = 0.3                  # same (non-diagonal) state in every beam
        H = b.nunu_hamiltonian(r, Y[0], Y[1])[-1]           # the radial probe bin
        F = b.flux_matrices(Y[0], Y[1])[0].sum(axis=0)      # energy-integrated flux of one bin
        mu = b.K * 11.0**2 / (2 * r * r)                   # K R^2/(2 r^2)
        D_num = (H[0, 1] / (mu * F[0, 1])).real
        errs.append(abs(D_num - D_exact))
    assert errs[-1] < 2e-3 * D_exact
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_lepton_number_invariant():
    """With lambda = 0 the continuous bulb equations conserve Tr(M J1), M the unit vacuum matrix:
    sum_b g_b B.(h_b x s_b)/c_b = mu B.(j0 x j0 - j1 x j1) = 0.  Matter breaks it."""
    wl = Workload(name="ln", n_energy=6, n_angle=5)
    b = Bulb(wl)
    M = np.array([[-math.cos(0.2), math.sin(0.2)], [math.sin(0.2), math.cos(0.2)]])
    drift = {}
    for matter in ("none", "constant"):
        wl.matter, wl.lambda_const = matter, 30.0
        b = Bulb(wl)
        vals = []
        def cb(n, r, Y):
            J0, J1 = b.moment_matrices(r, Y)
            vals.append(np.trace(M @ J1).real)
        Y0 = b.initial_state()
        evolve_fixed(b, Y0, 70.0, 80.0, 400, "rk4", callback=cb)
        scale = np.abs(b.moment_matrices(70.0, Y0)[1]).max()
        drift[matter] = (max(vals) - min(vals)) / scale
    assert drift["none"] < 1e-9
    assert drift["constant"] > 1e-4


def _sync_rate(mu0, n_energy=4, span=3.0, chunks=30):
    wl = Workload(name="sync", n_energy=n_energy, n_angle=1, E_min=5.0, E_max=30.0,
                  dm2=(2.4e-3, 0.0), theta=(0.2, 0, 0))
    b = Bulb(wl, geometry="homogeneous", mu0=mu0)
    N = b.grid.N
    g_nu = N[0, 0] - N[0, 1]
    g_bar = -(N[1, 0] - N[1, 1])
    omega = 2.4e-3 / (2 * b.grid.E * 1e6 * ph.HBARC_EV_KM)
    w_sync = (np.sum(omega * g_nu) - np.sum(omega * g_bar)) / (np.sum(g_nu) + np.sum(g_bar))
    B = np.array([math.sin(0.4), 0.0, -math.cos(0.4)])
    e1 = np.array([0.0, 0.0, 1.0]) + B * math.cos(0.4)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(B, e1)
    Y, r, phases, rs = b.initial_state(), 0.0, [], []
    for _ in range(chunks):
        Y, r, _ = evolve_adaptive(b, Y, r, r + span / chunks, 1e-10, 1e-10, 1e-4)
        j = bloch(b.moment_matrices(r, Y)[1])
        phases.append(math.atan2(j @ e2, j @ e1))
        rs.append(r)
    return np.polyfit(rs, np.unwrap(phases), 1)[0], w_sync


def test_synchronised_precession():
    """Homogeneous geometry, mu0 >> omega: the collective vector J = sum_b g_b s_b precesses about
    B at omega_sync = sum_b eta_b omega_b g_b / sum_b g_b (synchronised oscillation), with a
    deviation that falls like 1/mu0."""
    dev = []
    for mu0 in (100.0, 1000.0):
        slope, w_sync = _sync_rate(mu0)
        dev.append(abs(slope / w_sync - 1))
    # |J| is ~12% of the total flux here, so the effective coupling is ~0.12 mu0
    assert dev[1] < 1.5e-2
    assert dev[0] / dev[1] > 5.0


def test_duplicated_angles_equal_single_angle():
    """A multi-angle run whose bins all sit at the same u (weights summing to 1) equals the one-bin
    run at that u, bin by bin."""
    u_star = 0.37
    wl1 = Workload(name="d1", n_energy=5, n_angle=1)
    b1 = Bulb(wl1, grid=Grid.from_workload(wl1, u=[u_star], du=[1.0]))
    wl4 = Workload(name="d4", n_energy=5, n_angle=4)
    b4 = Bulb(wl4, grid=Grid.from_workload(wl4, u=[u_star] * 4, du=[0.25] * 4))
    Y1, _ = evolve_fixed(b1, b1.initial_state(), 60.0, 70.0, 200, "rk4")
    Y4, _ = evolve_fixed(b4, b4.initial_state(), 60.0, 70.0, 200, "rk4")
    assert np.abs(pee(Y1)).min() < 0.999          # non-trivial evolution
    for j in range(4):
        assert np.abs(Y4[:, j] - Y1[:, 0]).max() < 1e-12


# --- invariants ---------------------------------------------------------------------------------------
def test_exponential_scheme_keeps_pure_states():
    """exp(-i H dl) is unitary: Tr P = 1, P^2 = P and P = P^dag hold to rounding (Sec. 3.4, Eq. U)."""
    wl = Workload(name="inv", n_energy=6, n_angle=5, matter="power_law")
    b = Bulb(wl)
    Y, _ = evolve_fixed(b, b.initial_state(), 40.0, 60.0, 100, "lie_rk4")
    tr = np.trace(Y, axis1=-2, axis2=-1)
    assert np.abs(tr - 1).max() < 1e-11
    assert np.abs(Y @ Y - Y).max() < 1e-11
    assert np.abs(Y - np.conj(np.swapaxes(Y, -1, -2))).max() < 1e-14


def test_runge_kutta_trace_exact_purity_to_order():
    wl = Workload(name="inv2", n_energy=6, n_angle=5)
    b = Bulb(wl)
    Y, _ = evolve_fixed(b, b.initial_state(), 70.0, 80.0, 400, "rk4")
    assert np.abs(np.trace(Y, axis1=-2, axis2=-1) - 1).max() < 1e-13   # commutator: trace exact
    purity = np.abs(Y @ Y - Y).max()                                      # purity only to O(h^4)
    assert 1e-12 < purity < 1e-4


# --- integrators --------------------------------------------------------------------------------------
def _nonlinear_case():
    wl = Workload(name="nl", n_energy=6, n_angle=5, r0=80, r1=82)
    b = Bulb(wl)
    return b, b.initial_state()


def test_runge_kutta_agrees_with_library_integrator():
    """The oracle's RK4 on its right-hand side matches scipy's DOP853 on the same right-hand side."""
    b, Y0 = _nonlinear_case()
    shape = Y0.shape
    def f(r, y):
        return b.rhs(r, y.reshape(shape)).ravel()
    sol = solve_ivp(f, (80.0, 82.0), Y0.ravel(), method="DOP853", rtol=1e-13, atol=1e-13)
    Yref = sol.y[:, -1].reshape(shape)
    Y, _ = evolve_fixed(b, Y0, 80.0, 82.0, 2000, "rk4")
    assert np.abs(Y - Yref).max() < 1e-10


@pytest.mark.parametrize("method,order", [("rk4", 4), ("lie_rk4", 4), ("dp5", 5)])
def test_convergence_order(method, order):
    """Richardson: halving h divides the error by 2^order (classical RK4, CF4, Dormand-Prince 5)."""
    b, Y0 = _nonlinear_case()
    Yref, _ = evolve_fixed(b, Y0, 80.0, 82.0, 8000, "rk4")
    errs = []
    for n in (100, 200, 400):
        if method == "dp5":
            Y, h = Y0.copy(), 2.0 / n
            k1 = b.rhs(80.0, Y)
            for i in range(n):
                Y, _, k1 = dp45_step(b.rhs, 80.0 + i * h, Y, h, k1, 1.0, 1.0)
        else:
            Y, _ = evolve_fixed(b, Y0, 80.0, 82.0, n, method)
        errs.append(np.abs(Y - Yref).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(q - order) < 0.35 for q in rates), (errs, rates)


def test_dormand_prince_tableau_consistency():
    """Row sums of A equal c; both weight rows sum to 1 (consistency of the Butcher tableau)."""
    for i in range(1, 7):
        assert abs(sum(DP_A[i]) - DP_C[i]) < 1e-15
    assert abs(DP_B.sum() - 1) < 1e-15 and abs(DP_BHAT.sum() - 1) < 1e-15


def test_adaptive_controller_meets_tolerance():
    b, Y0 = _nonlinear_case()
    Yref, _ = evolve_fixed(b, Y0, 80.0, 82.0, 8000, "rk4")
    Y, r, st = evolve_adaptive(b, Y0, 80.0, 82.0, 1e-8, 1e-8, 1e-3)
    assert r == 82.0 and st.accepted > 5
    assert np.abs(Y - Yref).max() < 1e-6


# --- paper-literal state and flavour reductions -----------------------------------------------------
@pytest.mark.parametrize("nf", [2, 3])
def test_four_wavefunctions_equal_reduced_state(nf):
    """Evolving every initial particle identity's wavefunction (Sec. 3.2 NBeam array, Sec. 2 flux
    sum over alpha) equals evolving the electron-flavour density matrices with I - P for the rest."""
    if nf == 2:
        wl = Workload(name="4p", n_energy=5, n_angle=4, matter="constant", lambda_const=3.0)
    else:
        wl = Workload(name="4p3", n_flavor=3, n_energy=5, n_angle=4, dm2=(7.5e-5, -2.4e-3),
                      theta=(0.59, 0.15, 0.785), matter="constant", lambda_const=3.0)
    b = Bulb(wl)
    Y, psi = b.initial_state(), four_psi.initial_wavefunctions(b)
    r = 70.0
    for _ in range(30):
        Y = cf4_step(b.generators, r, Y, 0.1)
        psi = four_psi.cf4_step(b, r, psi, 0.1)
        r += 0.1
    assert pee(Y).min() < 0.999
    assert np.abs(four_psi.electron_density_matrices(psi) - Y).max() < 1e-12


def test_three_flavours_reduce_to_two():
    """theta12 = theta23 = 0, dm2_21 = 0: the e-tau sector is the two-flavour problem with
    (dm2_31, theta13); the mu flavour decouples."""
    wl2 = Workload(name="r2", n_energy=5, n_angle=4, dm2=(-2.4e-3, 0.0), theta=(0.1, 0, 0),
                   matter="constant", lambda_const=1.0)
    wl3 = Workload(name="r3", n_flavor=3, n_energy=5, n_angle=4, dm2=(0.0, -2.4e-3),
                   theta=(0.0, 0.1, 0.0), matter="constant", lambda_const=1.0)
    b2, b3 = Bulb(wl2), Bulb(wl3)
    Y2, _ = evolve_fixed(b2, b2.initial_state(), 70.0, 75.0, 100, "rk4")
    Y3, _ = evolve_fixed(b3, b3.initial_state(), 70.0, 75.0, 100, "rk4")
    assert pee(Y2).min() < 0.999
    assert np.abs(Y3[..., 0, 0] - Y2[..., 0, 0]).max() < 1e-12
    assert np.abs(Y3[..., 0, 2] - Y2[..., 0, 1]).max() < 1e-12
    assert np.abs(Y3[..., 1, 1]).max() < 1e-15


def test_spectra_normalisation():
    """Per-bin number luminosities sum to L/<E> per flavour (Sec. 2: L/<E> f(E), f normalised)."""
    N = number_luminosity_bins(2, 64, 1.0, 60.0, {"nue": 1e51, "nuebar": 2e51, "nux": 3e51,
                                                   "nuxbar": 3e51},
                               {"nue": 11.0, "nuebar": 16.0, "nux": 25.0, "nuxbar": 25.0})
    MeV = 1.602176634e-6
    assert abs(N[0, 0].sum() / (1e51 / (11 * MeV)) - 1) < 1e-13
    assert abs(N[1, 0].sum() / (2e51 / (16 * MeV)) - 1) < 1e-13
    assert abs(N[1, 1].sum() / (3e51 / (25 * MeV)) - 1) < 1e-13


def test_order_sensitivity_floor():
    """How much the FP64 result depends on the order of the sums over beams: the small workload
    over its parity window (2000 RK4 steps, 100 -> 200 km) with the angle and energy bins in
    reverse order (so every moment sum runs backwards), mapped back, against the plain order.
    The FP64 parity gate is max(1e-10, 10 x floor); the floor must sit well below it."""
    wl = workload_2f_small_fp64()
    g = Grid.from_workload(wl)
    rev = Grid(E=g.E[::-1].copy(), u=g.u[::-1].copy(), du=g.du[::-1].copy(), N=g.N[:, :, ::-1].copy())
    outs = []
    for grid in (g, rev):
        b = Bulb(wl, grid=grid)
        Y, _ = evolve_fixed(b, b.initial_state(), 100.0, 200.0, 2000)
        outs.append(Y)
    A, B = outs[0], outs[1][:, ::-1, ::-1]
    floor = float((np.sqrt((np.abs(A - B) ** 2).sum(axis=(-2, -1)))
                   / np.sqrt((np.abs(A) ** 2).sum(axis=(-2, -1)))).max())
    assert 0.0 < floor < 1e-11, floor


@pytest.mark.parametrize("nf", [2, 3])
def test_flux_spectra_pins(nf):
    """Flux spectra: the initial condition gives the emitted spectra; every state conserves the
    total number per energy bin (unitarity); equal e and x spectra hide any flavour change; the
    vacuum closed form fixes the nu_e flux of an evolved state."""
    kw = dict(n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.785)) if nf == 3 else {}
    wl = Workload(name="fx", n_energy=6, n_angle=5, **kw)
    b = Bulb(wl)
    g = b.grid
    F0 = b.flux_spectra(b.initial_state())
    sdu = g.du.sum()
    for s in range(2):
        assert np.allclose(F0[s, 0], g.N[s, 0] * sdu, rtol=1e-15)
        for a in range(1, nf):
            assert np.allclose(F0[s, a], g.N[s, 1] * sdu, rtol=1e-15)
    psi = np.random.default_rng(3).standard_normal((2, 5, 6, nf)) + 1j * np.random.default_rng(4).standard_normal((2, 5, 6, nf))
    psi /= np.linalg.norm(psi, axis=-1, keepdims=True)
    Y = psi[..., :, None] * np.conj(psi[..., None, :])
    F = b.flux_spectra(Y)
    for s in range(2):
        assert np.allclose(F[s].sum(axis=0), (g.N[s, 0] + (nf - 1) * g.N[s, 1]) * sdu, rtol=1e-13)
    Neq = g.N.copy()
    Neq[:, 0] = Neq[:, 1]
    beq = Bulb(wl, grid=Grid(E=g.E, u=g.u, du=g.du, N=Neq))
    assert np.allclose(beq.flux_spectra(Y)[:, 0], Neq[:, 0] * sdu, rtol=1e-13)
    if nf == 2:
        # vacuum: P_ee of the closed form at path length L_j, then Phi_e by hand
        wv = Workload(name="fxv", n_energy=6, n_angle=5, L={k: 0.0 for k in ("nue", "nuebar", "nux", "nuxbar")},
                      dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0))
        bv = Bulb(wv, grid=Grid(E=g.E, u=g.u, du=g.du, N=np.zeros_like(g.N)))
        Yv, _ = evolve_fixed(bv, bv.initial_state(), 11.0, 31.0, 4000, method="lie_rk4")
        bv = Bulb(wv, grid=g)             # the flux weights of the emitted spectra
        c = np.sqrt(1 - g.u * 121.0 / 31.0**2)
        Lp = 31.0 * c - 11.0 * np.sqrt(1 - g.u)
        pee = 1 - np.sin(0.6) ** 2 * np.sin(2.4e-3 * Lp[:, None] / (4 * g.E[None, :] * 1e6 * 197.3269804e-12)) ** 2
        want = (g.du[:, None] * (g.N[0, 0][None] * pee + g.N[0, 1][None] * (1 - pee))).sum(axis=0)
        assert np.allclose(bv.flux_spectra(Yv)[0, 0], want, rtol=1e-10)


# --- exponential midpoint rule (the paper's kind of integrator) ------------------------------------
def test_em2_order_and_embedded_error():
    """Richardson: the exponential midpoint rule is second order, its exponential-Euler partner
    first order, so their difference (the error estimate) shrinks like h^2 per step."""
    from oracle.integrate import evolve_em2, em2_step
    b, Y0 = _nonlinear_case()
    Yref, _ = evolve_fixed(b, Y0, 80.0, 82.0, 8000, "rk4")
    errs = []
    for n in (200, 400, 800):
        Y, _, _ = evolve_em2(b, Y0, 80.0, 82.0, 1, 1, 1, fixed_steps=n)
        errs.append(np.abs(Y - Yref).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(q - 2) < 0.25 for q in rates), (errs, rates)
    loc = []
    for h in (0.02, 0.01, 0.005):
        Yn, Ye = em2_step(b.generators, 80.0, Y0, h)
        loc.append(np.abs(Yn - Ye).max())
    lr = [math.log2(loc[i] / loc[i + 1]) for i in range(2)]
    assert all(abs(q - 2) < 0.25 for q in lr), (loc, lr)


def test_em2_exact_for_constant_generator():
    """A generator that does not change (vacuum + constant matter, no nu-nu coupling (mu0 = 0), all
    beams radial in the homogeneous test geometry) is integrated exactly, and the error estimate
    vanishes."""
    from oracle.integrate import em2_step
    wl = Workload(name="cst", n_energy=4, n_angle=3, matter="constant", lambda_const=3.0,
                  dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0))
    b = Bulb(wl, geometry="homogeneous", mu0=0.0)
    Y0 = b.initial_state()
    Yn, Ye = em2_step(b.generators, 50.0, Y0, 0.37)
    G = b.generators(50.0, Y0)
    U = np.stack([expm(-1j * 0.37 * g) for g in G.reshape(-1, 2, 2)]).reshape(G.shape)
    exact = U @ Y0 @ np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(Yn - exact).max() < 1e-13 and np.abs(Yn - Ye).max() < 1e-13


def test_em2_adaptive_meets_tolerance():
    from oracle.integrate import evolve_em2
    b, Y0 = _nonlinear_case()
    Yref, _ = evolve_fixed(b, Y0, 80.0, 82.0, 8000, "rk4")
    Y, r, st = evolve_em2(b, Y0, 80.0, 82.0, 1e-7, 1e-7, 1e-3)
    assert r == 82.0 and st.rejected >= 0 and st.accepted > 20
    assert np.abs(Y - Yref).max() < 1e-4


# --- commutator-free Lie RK4 with Richardson step-size control (adaptive exact propagators) -------
def _grazing_case():
    """The 4M-beam workload's physics near the neutrino sphere on a few beams: r^-3 matter, six
    energies, angle bins taken from the 2000-bin grid including the grazing last bin (cos theta =
    0.016 at r = R)."""
    j = [0, 500, 1000, 1500, 1900, 1990, 1999]
    u = np.array([(jj + 0.5) / 2000 for jj in j])
    wl = Workload(name="graze", n_energy=6, n_angle=len(j), matter="power_law")
    b = Bulb(wl, grid=Grid.from_workload(wl, u=u, du=np.full(len(j), 1.0 / len(j))))
    return b, b.initial_state()


def test_lie_richardson_exact_for_constant_generator():
    """A generator that does not change (vacuum + constant matter, no coupling, radial beams) is
    integrated exactly by the full step and by the two half steps, so the estimate vanishes."""
    from oracle.integrate import lie_richardson_step
    wl = Workload(name="cst", n_energy=4, n_angle=3, matter="constant", lambda_const=3.0,
                  dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0))
    b = Bulb(wl, geometry="homogeneous", mu0=0.0)
    Y0 = b.initial_state()
    two, full = lie_richardson_step(b.generators, 50.0, Y0, 0.37)
    G = b.generators(50.0, Y0)
    U = np.stack([expm(-1j * 0.37 * g) for g in G.reshape(-1, 2, 2)]).reshape(G.shape)
    exact = U @ Y0 @ np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(two - exact).max() < 1e-13 and np.abs(full - exact).max() < 1e-13


def test_lie_richardson_estimate_is_the_local_error():
    """Richardson for an order-4 method: the two half steps' local error is -(Y_two - Y_full)/15
    to O(h) relative, and it shrinks like h^5."""
    from oracle.integrate import lie_richardson_step, lie_richardson_error
    b, Y0 = _nonlinear_case()
    Y, _ = evolve_fixed(b, Y0, 80.0, 81.0, 4000, "lie_rk4")
    act, mis = [], []
    for h in (0.1, 0.05, 0.025):
        two, full = lie_richardson_step(b.generators, 81.0, Y, h)
        ref, _ = evolve_fixed(b, Y, 81.0, 81.0 + h, 200, "lie_rk4")
        a, est = two - ref, lie_richardson_error(two, full)
        act.append(np.abs(a).max())
        mis.append(np.abs(est + a).max() / np.abs(a).max())
    assert mis[2] < 0.15 and mis[2] < mis[1] < mis[0], mis
    rates = [math.log2(act[i] / act[i + 1]) for i in range(2)]
    assert all(abs(q - 5) < 0.3 for q in rates), (act, rates)


def test_lie_adaptive_meets_tolerance():
    from oracle.integrate import evolve_lie_adaptive
    b, Y0 = _nonlinear_case()
    Yref, _ = evolve_fixed(b, Y0, 80.0, 82.0, 8000, "rk4")
    Y, r, st = evolve_lie_adaptive(b, Y0, 80.0, 82.0, 1e-8, 1e-8, 1e-3, max_attempts=1000)
    assert r == 82.0 and st.accepted > 20
    assert np.abs(Y - Yref).max() < 2e-6                   # ~ accepted steps x tolerance


def test_lie_adaptive_steps_far_beyond_the_explicit_limit():
    """From r = R under the r^-3 matter term (1.45e6 /km, x 63 for the grazing bin) explicit Runge-
    Kutta is stable only for h |H|/cos theta below ~2.8 (2.5e-8 km here); the exact propagators
    take steps set by how fast the generator changes: 11 -> 11.01 km in a few tens of steps at
    rtol = atol = 1e-6, the median step some hundred times that limit, and the result within
    the accumulated tolerance of a run at 1e-8."""
    from oracle.integrate import evolve_lie_adaptive
    b, Y0 = _grazing_case()
    G = b.generators(11.0, Y0).reshape(-1, 2, 2)
    ev = np.linalg.eigvalsh(G)
    limit = 2.8 / (ev[:, 1] - ev[:, 0]).max()
    Y, r, st = evolve_lie_adaptive(b, Y0, 11.0, 11.01, 1e-6, 1e-6, 1e-9, max_attempts=1000)
    hs = [h for (_, h, ok) in st.steps if ok]
    assert r == 11.01 and st.accepted < 40
    assert np.median(hs) > 100 * limit and max(hs) > 1e5 * limit
    Yt, _, st8 = evolve_lie_adaptive(b, Y0, 11.0, 11.01, 1e-8, 1e-8, 1e-9, max_attempts=1000)
    assert st8.accepted < 200
    assert np.abs(Y - Yt).max() < 1e-5


# --- single-angle geometry and tabulated matter profile ----------------------------------------
def test_single_angle_geometry_is_the_bulb_on_the_radial_beam():
    """The single-angle potential equals the multi-angle bulb's potential on a radial probe beam
    when every beam carries the same state, in the limit of fine u bins (the bulb's midpoint sum
    over u converges at second order to the integral the single-angle factor closes)."""
    r = 22.0
    Y1 = None
    errs = []
    for Nu in (16, 32, 64):
        wl = Workload(name="sa", n_energy=3, n_angle=Nu)
        u = np.concatenate([(np.arange(Nu) + 0.5) / Nu, [0.0]])
        du = np.concatenate([np.full(Nu, 1.0 / Nu), [0.0]])
        b = Bulb(wl, grid=Grid.from_workload(wl, u=u, du=du))
        sa = Bulb(wl, grid=Grid.from_workload(wl, u=u, du=du), geometry="single_angle")
        Y = b.initial_state()
        Y[..., 0, 1] = 0.3
        Y[..., 1, 0] = 0.3
        Hb = b.nunu_hamiltonian(r, Y[0], Y[1])[-1]
        Hs = sa.nunu_hamiltonian(r, Y[0], Y[1])[0]
        errs.append(abs(Hb[0, 1] - Hs[0, 1]) / abs(Hs[0, 1]))
    assert errs[-1] < 2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_single_angle_bins_evolve_as_one():
    """Angle bins are indistinguishable in the single-angle geometry: four bins of weight 1/4 evolve
    exactly as one bin of weight 1, whatever their u."""
    kw = dict(n_energy=5, matter="constant", lambda_const=0.5)
    wl4, wl1 = Workload(name="s4", n_angle=4, **kw), Workload(name="s1", n_angle=1, **kw)
    g4 = Grid.from_workload(wl4, u=np.array([0.1, 0.4, 0.7, 0.95]), du=np.full(4, 0.25))
    g1 = Grid.from_workload(wl1, u=np.array([0.3]), du=np.array([1.0]))
    b4, b1 = Bulb(wl4, grid=g4, geometry="single_angle"), Bulb(wl1, grid=g1, geometry="single_angle")
    Y4, _ = evolve_fixed(b4, b4.initial_state(), 40.0, 42.0, 200, "rk4")
    Y1, _ = evolve_fixed(b1, b1.initial_state(), 40.0, 42.0, 200, "rk4")
    assert pee(Y1).min() < 0.9995
    for j in range(4):
        assert np.abs(Y4[:, j] - Y1[:, 0]).max() < 1e-13


def test_matter_table_reproduces_a_power_law():
    """A table sampled from rho0 (r_ref/r)^3 gives the power law's lambda between its points (each
    interval is interpolated as a power law), the end values outside it, and the same evolution."""
    pl = Workload(name="pl", n_energy=4, n_angle=3, matter="power_law")
    rt = [10.0, 30.0, 100.0, 300.0, 1000.0]
    tab = Workload(name="tb", n_energy=4, n_angle=3, matter="table", matter_table_r=rt,
                   matter_table_lambda=[ph.matter_strength(r, pl) for r in rt])
    for r in (10.0, 11.0, 47.3, 100.0, 777.0):
        assert abs(ph.matter_strength(r, tab) / ph.matter_strength(r, pl) - 1) < 1e-13
    assert ph.matter_strength(5.0, tab) == ph.matter_strength(10.0, pl)
    assert ph.matter_strength(2000.0, tab) == ph.matter_strength(1000.0, pl)
    Ya, _ = evolve_fixed(Bulb(pl), Bulb(pl).initial_state(), 300.0, 301.0, 50, "lie_rk4")
    Yb, _ = evolve_fixed(Bulb(tab), Bulb(tab).initial_state(), 300.0, 301.0, 50, "lie_rk4")
    assert np.abs(Ya - Yb).max() < 1e-12


def test_lie_adaptive_three_flavours_meets_the_vacuum_closed_form():
    """The adaptive commutator-free Lie RK4 on three flavours (eigendecomposition propagators):
    mu = lambda = 0 with every mixing angle and both splittings non-zero, 11 -> 211 km with a
    tolerance of 1e-10, reproduces the textbook three-flavour vacuum P_ee and P_emu (as in
    test_three_flavour_vacuum_closed_form) in a few hundred steps, and its steps grow far beyond the
    first one."""
    from oracle.integrate import evolve_lie_adaptive
    th, dm = (0.59, 0.15, 0.785), (7.5e-5, 2.4e-3)
    wl = Workload(name="vac3a", n_flavor=3, n_energy=6, n_angle=4, E_min=2.0, E_max=20.0, L=NO_L,
                  dm2=dm, theta=th)
    b = Bulb(wl)
    Y, r, st = evolve_lie_adaptive(b, b.initial_state(), 11.0, 211.0, 1e-10, 1e-10, 0.01, max_attempts=5000)
    assert r == 211.0 and st.accepted < 2000
    assert max(h for _, h, ok in st.steps if ok) > 50 * st.steps[0][1]
    c12, s12 = math.cos(th[0]), math.sin(th[0])
    c13, s13 = math.cos(th[1]), math.sin(th[1])
    c23, s23 = math.cos(th[2]), math.sin(th[2])
    Ue = [c12 * c13, s12 * c13, s13]
    Um = [-s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13]
    m2 = [0.0, dm[0], dm[1]]
    g = b.grid
    L = 211.0 * cos_theta(g.u, 11.0, 211.0) - 11.0 * np.sqrt(1.0 - g.u)
    k = 1.0 / (4 * ph.HBARC_EV_KM * 1e6)
    Pee, Pem = np.ones((4, 6)), np.zeros((4, 6))
    for i in range(3):
        for j in range(i + 1, 3):
            s2 = np.sin(k * (m2[j] - m2[i]) * L[:, None] / g.E[None, :]) ** 2
            Pee -= 4 * Ue[i] ** 2 * Ue[j] ** 2 * s2
            Pem -= 4 * Ue[i] * Um[i] * Ue[j] * Um[j] * s2
    for s in range(2):
        assert np.abs(Y[s, ..., 0, 0].real - Pee).max() < 1e-7
        assert np.abs(Y[s, ..., 1, 1].real - Pem).max() < 1e-7
