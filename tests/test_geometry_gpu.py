"""The single-angle and homogeneous geometries and the tabulated matter profile on the GPU against
the oracle (Sec. 2: Eq. Hnu and H_mat; the boundary's geometry and MATTER_TABLE options)."""
import math

import numpy as np
import pytest

from bulb_inputs import Workload
from oracle import physics as ph
from oracle.physics import Bulb, Grid
from oracle.integrate import evolve_fixed, evolve_adaptive
from parity_util import beams, rel_err, make_solver

pytestmark = pytest.mark.gpu

RAGGED = dict(n_energy=37, n_angle=29)


def bloch(M):
    return np.array([2 * M[0, 1].real, -2 * M[0, 1].imag, (M[0, 0] - M[1, 1]).real])


@pytest.mark.parametrize("integrator", ["rk4", "dp45"])
def test_homogeneous_parity(xf, integrator):
    """Isotropic coupling mu0 J1 (strong: mu0 = 300 /km) with every beam radial."""
    wl = Workload(name="hom", **RAGGED, integrator=integrator, n_steps=400, rtol=1e-9, atol=1e-9, h0=1e-3)
    s = make_solver(xf, wl, geometry="homogeneous", mu_const_kmi=300.0, fixed_dr_km=0.005)
    s.reset(11.0)
    s.evolve(11.0, 13.0)
    b = Bulb(wl, geometry="homogeneous", mu0=300.0)
    if integrator == "rk4":
        Y, _ = evolve_fixed(b, b.initial_state(), 11.0, 13.0, 400, "rk4")
    else:
        Y, _, st = evolve_adaptive(b, b.initial_state(), 11.0, 13.0, 1e-9, 1e-9, 1e-3)
        assert (s.stats().accepted, s.stats().rejected) == (st.accepted, st.rejected)
    assert np.abs(beams(Y)[:, 0, 0].real - 1).max() > 0.005
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10


def test_homogeneous_synchronised_precession(xf):
    """mu0 >> omega: the device's collective vector J1 precesses about B at
    omega_sync = sum_b eta_b omega_b g_b / sum_b g_b, to O(omega / (mu0 |J1|))."""
    wl = Workload(name="sync", n_energy=4, n_angle=1, E_min=5.0, E_max=30.0, dm2=(2.4e-3, 0.0),
                  theta=(0.2, 0, 0), integrator="dp45", rtol=1e-10, atol=1e-10, h0=1e-4)
    s = make_solver(xf, wl, geometry="homogeneous", mu_const_kmi=1000.0)
    b = Bulb(wl, geometry="homogeneous", mu0=1000.0)
    N = b.grid.N
    g_nu, g_bar = N[0, 0] - N[0, 1], -(N[1, 0] - N[1, 1])
    omega = 2.4e-3 / (2 * b.grid.E * 1e6 * ph.HBARC_EV_KM)
    w_sync = (np.sum(omega * g_nu) - np.sum(omega * g_bar)) / (np.sum(g_nu) + np.sum(g_bar))
    B = np.array([math.sin(0.4), 0.0, -math.cos(0.4)])
    e1 = np.array([0.0, 0.0, 1.0]) + B * math.cos(0.4)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(B, e1)
    r, phases, rs = 11.0, [], []
    s.reset(r)
    for _ in range(30):
        s.evolve(r, r + 0.1)
        r += 0.1
        j = bloch(s.moments()[1])
        phases.append(math.atan2(j @ e2, j @ e1))
        rs.append(r)
    slope = np.polyfit(rs, np.unwrap(phases), 1)[0]
    assert abs(slope / w_sync - 1) < 1.5e-2


def test_single_angle_parity(xf):
    """Single-angle geometry, DP45, with constant matter, against the oracle: same steps, 1e-10."""
    wl = Workload(name="sa", n_energy=41, n_angle=3, integrator="dp45", matter="constant",
                  lambda_const=2.0, rtol=1e-9, atol=1e-9, h0=0.5)
    s = make_solver(xf, wl, geometry="single_angle")
    s.reset(100.0)
    s.evolve(100.0, 103.0)
    b = Bulb(wl, geometry="single_angle")
    Y, _, st = evolve_adaptive(b, b.initial_state(), 100.0, 103.0, 1e-9, 1e-9, 0.5)
    assert st.rejected > 0 and (s.stats().accepted, s.stats().rejected) == (st.accepted, st.rejected)
    assert np.abs(beams(Y)[:, 0, 0].real - 1).max() > 0.1
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10
    # angle bins are indistinguishable: every bin carries the same state
    got = s.get_rho().reshape(2, 3, 41, 2, 2)
    assert np.abs(got - got[:, :1]).max() < 1e-14


def test_matter_table(xf):
    """A table sampled from the r^-3 profile reproduces the power-law run; an irregular table
    matches the oracle's table profile at 1e-10."""
    pl = Workload(name="pl", **RAGGED, integrator="dp45", matter="power_law", rtol=1e-9, atol=1e-9, h0=0.5)
    rt = [10.0, 30.0, 100.0, 300.0, 1000.0]
    tab = Workload(name="tb", **RAGGED, integrator="dp45", matter="table", rtol=1e-9, atol=1e-9, h0=0.5,
                   matter_table_r=rt, matter_table_lambda=[ph.matter_strength(r, pl) for r in rt])
    sa, sb = make_solver(xf, pl), make_solver(xf, tab)
    for s in (sa, sb):
        s.reset(200.0)
        s.evolve(200.0, 203.0)
    assert (sa.stats().accepted, sa.stats().rejected) == (sb.stats().accepted, sb.stats().rejected)
    assert rel_err(sb.get_rho(), sa.get_rho()) < 1e-12
    odd = Workload(name="odd", **RAGGED, integrator="dp45", matter="table", rtol=1e-9, atol=1e-9, h0=0.5,
                   matter_table_r=[150.0, 201.0, 202.5, 250.0], matter_table_lambda=[30.0, 2.0, 9.0, 1.0])
    so = make_solver(xf, odd)
    so.reset(200.0)
    so.evolve(200.0, 203.0)
    b = Bulb(odd)
    Y, _, st = evolve_adaptive(b, b.initial_state(), 200.0, 203.0, 1e-9, 1e-9, 0.5)
    assert (so.stats().accepted, so.stats().rejected) == (st.accepted, st.rejected)
    assert rel_err(so.get_rho(), beams(Y)) < 1e-10
