"""Extended bulb model (azimuthal bins, Sec. 2 Eq. int-v and Eq. F) on the GPU against the oracle's
extended model, and the paper's own validation: with the axial symmetry unbroken the extended
model reproduces the bulb model."""
import numpy as np
import pytest

from bulb_inputs import Workload, random_unit_states
from oracle.physics import Bulb
from oracle.extended import ExtendedBulb
from oracle.integrate import evolve_fixed, evolve_adaptive, evolve_em2
from parity_util import beams, rel_err, make_solver

pytestmark = pytest.mark.gpu

SIZES = dict(n_energy=13, n_angle=7)
NPHI = 6


def asym_state(eb, seed):
    """Near-electron states with a random azimuthal pattern (large azimuthal moments)."""
    n = eb.n
    shape = (2, len(eb.grid.u), eb.n_phi, len(eb.grid.E))
    psi = random_unit_states(n, int(np.prod(shape)), seed).reshape(*shape, n) * 0.3
    psi[..., 0] += 1.0
    psi /= np.linalg.norm(psi, axis=-1, keepdims=True)
    return psi[..., :, None] * np.conj(psi[..., None, :])


def test_extended_moments_match_oracle(xf):
    wl = Workload(name="ex", **SIZES)
    eb = ExtendedBulb(wl, NPHI)
    s = make_solver(xf, wl, n_phi=NPHI, fixed_dr_km=0.1)
    assert s.nbeams() == 2 * 13 * 7 * NPHI
    Y = asym_state(eb, 5)
    s.set_rho(beams(Y), 60.0)
    J0, J1 = s.moments()
    Jc, Js = s.moments_phi()
    R0, R1, Rc, Rs = eb.moment_matrices(60.0, Y)
    for got, ref in ((J0, R0), (J1, R1), (Jc, Rc), (Js, Rs)):
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(R1).max()
    assert np.abs(Rc).max() > 1e-3 * np.abs(R1).max()


@pytest.mark.parametrize("integrator", ["rk4", "dp45", "lie_rk4", "exp_midpoint"])
def test_extended_parity_asymmetric(xf, integrator):
    # the second-order exponential midpoint rule runs at rtol = atol = 1e-6 (~700 steps per km)
    tol = 1e-6 if integrator == "exp_midpoint" else 1e-9
    wl = Workload(name="ex", **SIZES, integrator=integrator, n_steps=40, h0=0.5, rtol=tol, atol=tol)
    eb = ExtendedBulb(wl, NPHI)
    Y0 = asym_state(eb, 7)
    r0, r1 = 100.0, 101.0
    s = make_solver(xf, wl, n_phi=NPHI, fixed_dr_km=(r1 - r0) / 40)
    s.set_rho(beams(Y0), r0)
    s.evolve(r0, r1)
    if integrator in ("rk4", "lie_rk4"):
        Y, _ = evolve_fixed(eb, Y0, r0, r1, 40, integrator)
    else:
        evolve = evolve_adaptive if integrator == "dp45" else evolve_em2
        Y, _, st = evolve(eb, Y0, r0, r1, wl.rtol, wl.atol, wl.h0)
        gs = s.stats()
        assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected)
    assert rel_err(beams(Y), beams(Y0)) > 1e-3
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10


def test_axial_symmetry_gives_the_bulb_model(xf):
    """The paper's validation: from the (axially symmetric) initial condition the extended model's
    every azimuthal copy equals the bulb model's beam."""
    wl = Workload(name="ex", **SIZES, integrator="dp45", h0=1e-3)
    se = make_solver(xf, wl, n_phi=NPHI)
    sb = make_solver(xf, wl)
    for s in (se, sb):
        s.reset(100.0)
        s.evolve(100.0, 103.0)
    Ye = se.get_rho().reshape(2, 7, NPHI, 13, 2, 2)
    Yb = sb.get_rho().reshape(2, 7, 13, 2, 2)
    assert np.abs(Yb[0, ..., 0, 0].real - 1).max() > 1e-2
    for p in range(NPHI):
        assert np.abs(Ye[:, :, p] - Yb).max() < 1e-11
    Jc, Js = se.moments_phi()
    assert np.abs(Jc).max() < 1e-12 * np.abs(se.moments()[1]).max() + 1e-300


def test_extended_mixed_against_fp64_oracle(xf):
    wl = Workload(name="exm", **SIZES, integrator="dp45", rtol=1e-9, atol=1e-9, h0=1e-3)
    eb = ExtendedBulb(wl, NPHI)
    Y0 = asym_state(eb, 11)
    Y, _, _ = evolve_adaptive(eb, Y0, 100.0, 101.0, 1e-9, 1e-9, 1e-3)
    s = make_solver(xf, wl, n_phi=NPHI, precision="mixed", rtol=1e-6, atol=1e-6)
    s.set_rho(beams(Y0), 100.0)
    s.evolve(100.0, 101.0)
    pee, _ = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(pee - ref).max() < 1e-4


@pytest.mark.parametrize("integrator", ["rk4", "lie_rk4", "exp_midpoint"])
def test_extended_mixed_other_integrators(xf, integrator):
    """The mixed extended kernels of the fixed-step and exponential integrators against the FP64
    oracle's same scheme: survival probabilities within 1e-4."""
    tol = 1e-6 if integrator == "exp_midpoint" else 1e-9
    wl = Workload(name="exm2", **SIZES, integrator=integrator, n_steps=40, h0=1e-2, rtol=tol, atol=tol)
    eb = ExtendedBulb(wl, NPHI)
    Y0 = asym_state(eb, 13)
    r0, r1 = 100.0, 101.0
    if integrator == "exp_midpoint":
        Y, _, _ = evolve_em2(eb, Y0, r0, r1, tol, tol, 1e-2)
    else:
        Y, _ = evolve_fixed(eb, Y0, r0, r1, 40, integrator)
    s = make_solver(xf, wl, n_phi=NPHI, precision="mixed", fixed_dr_km=(r1 - r0) / 40)
    s.set_rho(beams(Y0), r0)
    s.evolve(r0, r1)
    pee, _ = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - beams(Y0)[:, 0, 0].real).max() > 1e-3
    assert np.abs(pee - ref).max() < 1e-4
