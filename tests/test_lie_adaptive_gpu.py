"""The adaptive exact-propagator integrator (XFLAT_LIE_ADAPTIVE: commutator-free Lie RK4 of Eq. U
propagators with Richardson step-size control) on the GPU against the oracle's implementation."""
import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Bulb, Grid
from parity_util import beams, rel_err, make_solver, oracle_run

pytestmark = pytest.mark.gpu

RAGGED = dict(n_energy=37, n_angle=29)          # 2146 beams: several blocks and a ragged tail


@pytest.mark.parametrize("matter,r0,r1", [("none", 100.0, 103.0), ("power_law", 300.0, 303.0)])
def test_lie_adaptive_fp64_parity(xf, matter, r0, r1):
    """Same accepted and rejected steps (a large first trial step forces rejections), the same stage
    count and the same final state as the oracle's controller."""
    wl = Workload(name="la", **RAGGED, integrator="lie_adaptive", matter=matter, rtol=1e-9, atol=1e-9,
                  h0=0.5)
    s = make_solver(xf, wl)
    s.reset(r0)
    s.evolve(r0, r1)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
    gs = s.stats()
    assert st.rejected > 0
    assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected)
    assert gs.stage_evals == st.stage_evals
    assert gs.r_km == r1
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10


def grazing():
    """r^-3 matter from r = R with angle bins of the 2000-bin grid up to the grazing last one."""
    j = [0, 250, 500, 1000, 1500, 1900, 1990, 1999]
    u = np.array([(jj + 0.5) / 2000 for jj in j])
    wl = Workload(name="graze", n_energy=33, n_angle=len(j), matter="power_law",
                  integrator="lie_adaptive", rtol=1e-6, atol=1e-6, h0=1e-9)
    return wl, Grid.from_workload(wl, u=u, du=np.full(len(j), 1.0 / len(j)))


def test_lie_adaptive_from_the_neutrino_sphere(xf):
    """From r = R, where explicit Runge-Kutta is stable only below ~2.5e-8 km: the same steps as the
    oracle (some hundred times that limit), FP64, and the same survival probabilities; mixed P_ee
    within 1e-4.  The states themselves agree only to the step's conditioning: each stage rotates
    by theta = h |K| radians (up to ~1e5 here), and a rounding difference in one stage's states
    moves the next stage's moments and so its rotation angles by theta times as much, so the tiny
    transverse components (~4e-7, the precession cone about the matter-dominated axis) differ in
    phase by up to theta^2 eps; their effect on P_ee = (1 + s_z)/2 is second order."""
    wl, g = grazing()
    s = make_solver(xf, wl, grid=g)
    s.evolve(11.0, 11.01)
    Y, st = oracle_run(wl, Bulb(wl, grid=g).initial_state(), 11.0, 11.01, grid=g)
    gs = s.stats()
    assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected)
    assert gs.accepted < 60
    got, ref = s.get_rho(), beams(Y)
    assert np.abs(got[:, 0, 0].real - ref[:, 0, 0].real).max() < 1e-10
    assert rel_err(got, ref) < 1e-5
    sm = make_solver(xf, wl, grid=g, precision="mixed")
    sm.evolve(11.0, 11.01)
    pee, _ = sm.pee()
    assert np.abs(pee - beams(Y)[:, 0, 0].real).max() < 1e-4
    assert sm.stats().accepted < 200


def test_lie_adaptive_mixed_against_fp64_oracle(xf):
    """FP32 propagators against the FP64 oracle at the same tolerance through a window of strong
    collective evolution (P_ee changes by more than 0.5): survival probabilities within 1e-4."""
    wl = Workload(name="lax", **RAGGED, integrator="lie_adaptive", rtol=1e-6, atol=1e-6, h0=1e-3)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 102.0)
    s = make_solver(xf, wl, precision="mixed")
    s.reset(100.0)
    s.evolve(100.0, 102.0)
    pee, mean = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 0.5
    assert np.abs(pee - ref).max() < 1e-4
    assert abs(mean - Bulb(wl).mean_survival(Y)) < 1e-5


def test_lie_adaptive_exact_in_vacuum_single_radius(xf):
    """Vacuum with one angle bin at u = 0 (cos theta = 1 at every r): the generator is constant, so
    every step is exact, the estimate vanishes and the steps grow by the factor 5."""
    wl = Workload(name="lav", n_energy=9, n_angle=1, L={k: 0.0 for k in ("nue", "nuebar", "nux", "nuxbar")},
                  dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0), integrator="lie_adaptive", h0=1e-3)
    g = Grid.from_workload(wl, u=np.array([0.0]), du=np.array([1.0]))
    s = make_solver(xf, wl, grid=g)
    s.evolve(11.0, 61.0)
    pee, _ = s.pee()
    ph = 2.4e-3 * 50.0 / (4 * g.E * 1e6 * 197.3269804e-12)
    ref = 1 - np.sin(0.6) ** 2 * np.sin(ph) ** 2
    assert np.abs(pee[:9] - ref).max() < 1e-11
    assert s.stats().rejected == 0 and s.stats().accepted < 12
