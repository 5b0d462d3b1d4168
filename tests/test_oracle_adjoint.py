"""Pins of the oracle's discrete adjoint (oracle/adjoint.py) against central finite differences of
the oracle's own forward RK4 run, on tiny inputs.

The adjoint is the exact gradient of the discrete map, so it must agree with the difference
quotient up to the quotient's own error (step 1e-6 relative: truncation ~1e-12, rounding ~1e-10
of J).  Every per-bin luminosity of both species and both flavours and the mixing angle is
checked, in windows with collective (nu-nu) evolution, without and with a matter term, for both mass
orderings, so a dropped term, a wrong sign or a transposed operand anywhere in the chain fails.
"""
import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Bulb, Grid
from oracle.integrate import evolve_fixed
from oracle.adjoint import rk4_adjoint


def forward_J(wl, grid, N, theta, r0, r1, n):
    w2 = Workload(**{**wl.to_dict(), "theta": (theta, 0.0, 0.0)})
    b = Bulb(w2, grid=Grid(E=grid.E, u=grid.u, du=grid.du, N=N))
    Y, _ = evolve_fixed(b, b.initial_state(), r0, r1, n)
    return b.mean_survival(Y)


CASES = [
    (dict(n_energy=4, n_angle=3), (100.0, 105.0), 100),
    (dict(n_energy=3, n_angle=4, dm2=(2.4e-3, 0.0), theta=(0.2, 0.0, 0.0), matter="constant",
          lambda_const=3.0, L={"nue": 4e51, "nuebar": 3e51, "nux": 1e51, "nuxbar": 1e51}),
     (100.0, 104.0), 120),
]


@pytest.mark.parametrize("kw,win,n", CASES)
def test_adjoint_matches_central_differences(kw, win, n):
    wl = Workload(name="adj", integrator="rk4", n_steps=n, **kw)
    g = Grid.from_workload(wl)
    r0, r1 = win
    b = Bulb(wl, grid=g)
    J, GN, Gth = rk4_adjoint(b, b.initial_state(), r0, r1, n)
    th = wl.theta[0]
    assert J == pytest.approx(forward_J(wl, g, g.N, th, r0, r1, n), abs=1e-14)
    eps = 1e-6
    fd = np.zeros_like(GN)
    for idx in np.ndindex(*g.N.shape):
        Np, Nm = g.N.copy(), g.N.copy()
        Np[idx] *= 1 + eps
        Nm[idx] *= 1 - eps
        fd[idx] = (forward_J(wl, g, Np, th, r0, r1, n) - forward_J(wl, g, Nm, th, r0, r1, n)) / (2 * eps)
    adj = GN * g.N                                  # d J / d log N
    assert np.abs(fd).max() > 1e-2                  # the luminosities matter in this window
    assert np.abs(adj - fd).max() < 1e-7, np.abs(adj - fd).max()
    d = 1e-6
    fdth = (forward_J(wl, g, g.N, th + d, r0, r1, n) - forward_J(wl, g, g.N, th - d, r0, r1, n)) / (2 * d)
    assert abs(fdth) > 1e-3
    assert Gth == pytest.approx(fdth, abs=1e-7)
