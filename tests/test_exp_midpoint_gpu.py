"""The exponential midpoint rule (the paper's kind of integrator: exact propagators of Eq. U with a
mid-point scheme and adaptive step control) on the GPU against the oracle's implementation."""
import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Bulb
from parity_util import beams, rel_err, make_solver, oracle_run

pytestmark = pytest.mark.gpu

RAGGED = dict(n_energy=37, n_angle=29)


@pytest.mark.parametrize("matter,r0,r1", [("none", 100.0, 101.0), ("power_law", 300.0, 301.0)])
def test_exp_midpoint_fp64_parity(xf, matter, r0, r1):
    """Same accepted and rejected steps as the oracle's controller (a large first trial step forces
    rejections) and the same final state.  A second-order method needs ~700 steps per km at
    rtol = 1e-6 here (collective evolution at 100 km), so the windows are short."""
    wl = Workload(name="em", **RAGGED, integrator="exp_midpoint", matter=matter, rtol=1e-6, atol=1e-6,
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


def test_exp_midpoint_mixed_against_fp64_oracle(xf):
    """FP32 rotations against the FP64 oracle with the same tolerance (1e-6) through 1.7e3 steps of
    strong collective evolution (P_ee changes by 0.8; the global error of the scheme at this
    tolerance is ~3e-6): survival probabilities within 3e-4."""
    wl = Workload(name="emx", **RAGGED, integrator="exp_midpoint", rtol=1e-6, atol=1e-6, h0=1e-3)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 102.0)
    s = make_solver(xf, wl, precision="mixed")
    s.reset(100.0)
    s.evolve(100.0, 102.0)
    pee, mean = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 0.5
    assert np.abs(pee - ref).max() < 3e-4
    assert abs(mean - Bulb(wl).mean_survival(Y)) < 1e-4


def test_exp_midpoint_exact_in_vacuum_single_radius(xf):
    """Vacuum with one angle bin at u = 0 (radial beams: cos theta = 1 at every r): the generator is
    constant, so every step is exact and the error estimate vanishes (steps grow by the factor 5)."""
    wl = Workload(name="emv", n_energy=9, n_angle=1, L={k: 0.0 for k in ("nue", "nuebar", "nux", "nuxbar")},
                  dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0), integrator="exp_midpoint", h0=1e-3)
    from oracle.physics import Grid
    g = Grid.from_workload(wl, u=np.array([0.0]), du=np.array([1.0]))
    s = make_solver(xf, wl, grid=g)
    s.evolve(11.0, 61.0)
    pee, _ = s.pee()
    ph = 2.4e-3 * 50.0 / (4 * g.E * 1e6 * 197.3269804e-12)
    ref = 1 - np.sin(0.6) ** 2 * np.sin(ph) ** 2
    assert np.abs(pee[:9] - ref).max() < 1e-11
    assert s.stats().rejected == 0
