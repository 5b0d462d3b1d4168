"""Mixed precision against the FP64 oracle at an intermediate size, over a window where the flavour
content changes by O(1): the survival probability of every beam within 1e-4 (the mixed form's
bar), for the explicit DP45 and the adaptive exact propagators."""
import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Bulb
from parity_util import beams, make_solver, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reference():
    """100 E x 150 u (30,000 beams), the small case's physics, 100 -> 102 km, oracle DP45 at 1e-9."""
    wl = Workload(name="mid", n_energy=100, n_angle=150, integrator="dp45", rtol=1e-9, atol=1e-9, h0=1e-3)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 102.0)
    return wl, beams(Y)[:, 0, 0].real, Bulb(wl).mean_survival(Y)


@pytest.mark.parametrize("integrator", ["dp45", "lie_adaptive"])
def test_mixed_within_1e4_of_the_oracle(xf, reference, integrator):
    wl, ref, ref_mean = reference
    assert np.abs(ref - 1.0).max() > 0.5                      # O(1) flavour change in the window
    s = make_solver(xf, wl, precision="mixed", integrator=integrator, rtol=1e-6, atol=1e-6, h0_km=1e-3)
    s.reset(100.0)
    s.evolve(100.0, 102.0)
    pee, mean = s.pee()
    assert np.abs(pee - ref).max() < 1e-4
    assert abs(mean - ref_mean) < 1e-5
