"""The exponential integrators for three flavours on the GPU: every update is the propagator of
Eq. U for a 3 x 3 generator, exp(-i H dl), applied by the eigen-decomposition of H (cyclic Jacobi
sweeps in the kernel, numpy's eigh in the oracle).  FP64 against the oracle step for step, mixed
against the FP64 oracle in survival probability, the textbook three-flavour vacuum formula
directly, and the configured three-flavour range from the neutrino sphere."""
import math

import numpy as np
import pytest

from bulb_inputs import Workload
from oracle import physics as ph
from oracle.physics import Bulb, cos_theta
from parity_util import beams, rel_err, make_solver, oracle_run

pytestmark = pytest.mark.gpu

MIX3 = dict(n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.785))


@pytest.mark.parametrize("integrator,matter,r0,r1,tol", [("lie_adaptive", "none", 100.0, 103.0, 1e-9),
                                                         ("lie_adaptive", "power_law", 300.0, 302.0, 1e-9),
                                                         ("exp_midpoint", "none", 100.0, 101.0, 1e-6)])
def test_three_flavour_adaptive_exponential_fp64_parity(xf, integrator, matter, r0, r1, tol):
    """The same accepted and rejected steps as the oracle's controller and the same final states
    (the second-order exponential midpoint rule at a looser tolerance, for a bounded step count)."""
    wl = Workload(name="e3", n_energy=13, n_angle=11, **MIX3, integrator=integrator, matter=matter,
                  rtol=tol, atol=tol, h0=0.5)
    s = make_solver(xf, wl)
    s.reset(r0)
    s.evolve(r0, r1)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
    gs = s.stats()
    assert st.rejected > 0
    assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected)
    assert gs.stage_evals == st.stage_evals
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10


def test_three_flavour_lie_rk4_fp64_parity(xf):
    wl = Workload(name="l3", n_energy=13, n_angle=11, **MIX3, integrator="lie_rk4", n_steps=40, r0=100.0,
                  r1=102.0)
    s = make_solver(xf, wl)
    s.reset(100.0)
    s.evolve(100.0, 102.0)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 102.0)
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10


@pytest.mark.parametrize("integrator", ["lie_adaptive", "lie_rk4"])
def test_three_flavour_exponential_mixed_against_fp64_oracle(xf, integrator):
    """FP32 propagators and states, exact moment sums, FP64 control: P_ee within 1e-4 of the FP64
    oracle through a window with evolution."""
    wl = Workload(name="m3e", n_energy=13, n_angle=11, **MIX3, integrator=integrator, n_steps=300,
                  r0=100.0, r1=103.0, rtol=1e-9, atol=1e-9, h0=0.05)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 103.0)
    s = make_solver(xf, wl, precision="mixed", rtol=1e-6, atol=1e-6)
    s.reset(100.0)
    s.evolve(100.0, 103.0)
    pee, _ = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 1e-2
    assert np.abs(pee - ref).max() < 1e-4


def test_three_flavour_vacuum_closed_form_on_gpu(xf):
    """mu = lambda = 0: the adaptive exponential integrator reproduces the textbook three-flavour
    vacuum survival and appearance probabilities (real mixing matrix in the standard
    parametrisation) along every beam's path length, FP64 to 1e-8 and mixed (at its usual tolerance
    1e-6) to 1e-4."""
    th, dm = MIX3["theta"], MIX3["dm2"]
    wl = Workload(name="v3", n_flavor=3, n_energy=6, n_angle=4, E_min=2.0, E_max=20.0, dm2=dm, theta=th,
                  L={k: 0.0 for k in ("nue", "nuebar", "nux", "nuxbar")}, integrator="lie_adaptive",
                  rtol=1e-11, atol=1e-11, h0=0.01)
    c12, s12 = math.cos(th[0]), math.sin(th[0])
    c13, s13 = math.cos(th[1]), math.sin(th[1])
    c23, s23 = math.cos(th[2]), math.sin(th[2])
    Ue = [c12 * c13, s12 * c13, s13]
    Um = [-s12 * c23 - c12 * s23 * s13, c12 * c23 - s12 * s23 * s13, s23 * c13]
    m2 = [0.0, dm[0], dm[1]]
    g = s_grid = Bulb(wl).grid
    L = 211.0 * cos_theta(g.u, 11.0, 211.0) - 11.0 * np.sqrt(1.0 - g.u)
    k = 1.0 / (4 * ph.HBARC_EV_KM * 1e6)
    Pee, Pem = np.ones((4, 6)), np.zeros((4, 6))
    for i in range(3):
        for j in range(i + 1, 3):
            s2 = np.sin(k * (m2[j] - m2[i]) * L[:, None] / s_grid.E[None, :]) ** 2
            Pee -= 4 * Ue[i] ** 2 * Ue[j] ** 2 * s2
            Pem -= 4 * Ue[i] * Um[i] * Ue[j] * Um[j] * s2
    assert Pee.min() < 0.5
    for precision, tol in (("fp64", 1e-8), ("mixed", 1e-4)):
        s = make_solver(xf, wl, precision=precision, rtol=1e-11 if precision == "fp64" else 1e-6,
                        atol=1e-11 if precision == "fp64" else 1e-6)
        s.evolve(11.0, 211.0)
        rho = s.get_rho().reshape(2, 4, 6, 3, 3)
        for sp in range(2):
            assert np.abs(rho[sp, ..., 0, 0].real - Pee).max() < tol, precision
            assert np.abs(rho[sp, ..., 1, 1].real - Pem).max() < tol, precision
        s.close()


def test_three_flavour_configured_range_from_the_neutrino_sphere(xf):
    """The three-flavour workload's matter profile and spectra from r = R, where explicit steps are
    stability-limited: the adaptive exponential integrator takes the same steps as the oracle over
    the first 0.2 km (FP64, 22 steps growing from 1e-6 km), with the same survival probabilities."""
    wl = Workload(name="r3", n_energy=9, n_angle=7, **MIX3, matter="power_law", integrator="lie_adaptive",
                  rtol=1e-8, atol=1e-8, h0=1e-6)
    s = make_solver(xf, wl)
    s.evolve(11.0, 11.2)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), 11.0, 11.2)
    gs = s.stats()
    assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected)
    assert gs.accepted < 400
    got, ref = s.get_rho(), beams(Y)
    assert np.abs(got[:, 0, 0].real - ref[:, 0, 0].real).max() < 1e-9
