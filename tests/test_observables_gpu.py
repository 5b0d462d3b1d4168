"""Observables at chosen radii (the Sec. 3.4 validation quantities): flux spectra of every flavour
and P_ee(theta_R, E) maps from the device against the oracle, and the snapshot files."""
import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Bulb, Grid
from parity_util import beams, make_solver, oracle_run, random_state

pytestmark = pytest.mark.gpu

RAGGED = dict(n_energy=37, n_angle=29)


@pytest.mark.parametrize("nf", [2, 3])
def test_flux_spectra_match_oracle(xf, nf):
    kw = dict(n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.785)) if nf == 3 else {}
    wl = Workload(name="fx", **RAGGED, **kw)
    s = make_solver(xf, wl, fixed_dr_km=0.1)
    b = Bulb(wl)
    F0 = s.flux_spectra()
    assert np.allclose(F0, b.flux_spectra(b.initial_state()), rtol=1e-14)
    Y = random_state(wl, seed=9 + nf)
    s.set_rho(beams(Y), 40.0)
    ref = b.flux_spectra(Y)
    assert np.abs(s.flux_spectra() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_snapshots_after_evolution(xf, tmp_path):
    from paper_1912_10596_gb300 import observables as ob
    wl = Workload(name="snap", **RAGGED, integrator="dp45", h0=1e-3)
    s = make_solver(xf, wl)
    s.reset(100.0)
    files = ob.evolve_with_snapshots(s, 100.0, [102.0, 104.0], str(tmp_path / "bulb"))
    assert len(files) == 2
    d = np.load(files[-1])
    assert float(d["r_km"]) == 104.0
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 104.0)
    b = Bulb(wl)
    assert np.abs(d["pee_nu"] - Y[0, ..., 0, 0].real).max() < 1e-10
    assert np.abs(d["pee_nubar"] - Y[1, ..., 0, 0].real).max() < 1e-10
    ref = b.flux_spectra(Y)
    assert np.abs(d["flux"] - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(Y[0, ..., 0, 0].real - 1).max() > 1e-3            # flavour did change
    g = Grid.from_workload(wl)
    assert np.allclose(d["E_MeV"], g.E) and np.allclose(np.sin(d["theta_R_rad"]) ** 2, g.u)
    # number conservation per energy bin (unitarity)
    tot = d["flux"].sum(axis=1)
    assert np.allclose(tot, (g.N[:, 0] + g.N[:, 1]) * g.du.sum(), rtol=1e-12)
