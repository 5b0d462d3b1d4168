"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 path 1e-10 relative on every beam's density matrix (the integration is the same
discrete scheme on both sides, so only rounding order differs); mixed path 1e-4 absolute on the
survival probabilities against the FP64 oracle.
"""
import math

import numpy as np
import pytest

from bulb_inputs import Workload, workload_2f_small_fp64
from oracle.physics import Bulb, Grid
from oracle.integrate import evolve_fixed, evolve_adaptive, cf4_step, rk4_step, dp45_step
from parity_util import beams, rel_err, random_state, make_solver, oracle_run

pytestmark = pytest.mark.gpu

RAGGED = dict(n_energy=37, n_angle=29)          # 2146 beams: several blocks and a ragged tail


def test_moments_match_oracle(xf):
    """J0, J1 (Eq. F moments) of a random state: device reduction vs the oracle's sums."""
    for nf in (2, 3):
        kw = dict(n_flavor=3, dm2=(7.5e-5, 2.4e-3), theta=(0.59, 0.15, 0.785)) if nf == 3 else {}
        wl = Workload(name="m", **RAGGED, **kw)
        s = make_solver(xf, wl, fixed_dr_km=0.1)
        Y = random_state(wl, seed=5 + nf)
        s.set_rho(beams(Y), 40.0)
        J0, J1 = s.moments()
        R0, R1 = Bulb(wl).moment_matrices(40.0, Y)
        assert np.abs(J0 - R0).max() <= 1e-12 * np.abs(R0).max()
        assert np.abs(J1 - R1).max() <= 1e-12 * np.abs(R1).max()


def test_state_round_trip(xf):
    wl = Workload(name="rt", **RAGGED)
    for prec in ("fp64", "mixed"):
        s = make_solver(xf, wl, fixed_dr_km=0.1, precision=prec)
        Y = beams(random_state(wl, seed=3))
        s.set_rho(Y, 20.0)
        back = s.get_rho()
        tol = 1e-15 if prec == "fp64" else 1e-7
        assert np.abs(back - Y).max() < tol
        assert s.stats().r_km == 20.0


@pytest.mark.parametrize("nf", [2, 3])
def test_rk4_fixed_step_parity(xf, nf):
    if nf == 3:
        wl = Workload(name="rk4", **RAGGED, integrator="rk4", n_steps=200, n_flavor=3,
                      dm2=(7.5e-5, -2.4e-3), theta=(0.59, 0.15, 0.785), matter="power_law")
        r0, r1 = 300.0, 301.0
    else:
        wl = Workload(name="rk4", **RAGGED, integrator="rk4", n_steps=200)
        r0, r1 = 100.0, 110.0
    s = make_solver(xf, wl, fixed_dr_km=(r1 - r0) / wl.n_steps)
    s.reset(r0)
    s.evolve(r0, r1)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
    assert np.abs(beams(Y)[..., 0, 1]).max() > 1e-3          # the state did evolve
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10
    gs = s.stats()
    assert gs.accepted == 200 and gs.stage_evals == 800 and gs.r_km == r1


@pytest.mark.parametrize("matter,r0,r1", [("none", 100.0, 104.0), ("power_law", 300.0, 301.0)])
def test_dp45_adaptive_parity(xf, matter, r0, r1):
    """Same accepted and rejected steps (a large first trial step forces rejections) and the same
    final state as the oracle's controller."""
    wl = Workload(name="dp", **RAGGED, integrator="dp45", matter=matter, rtol=1e-9, atol=1e-9, h0=0.5)
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


@pytest.mark.parametrize("matter,r0,r1", [("none", 100.0, 103.0), ("power_law", 400.0, 401.0)])
def test_dp45_three_flavour_parity(xf, matter, r0, r1):
    wl = Workload(name="dp3", n_flavor=3, n_energy=13, n_angle=11, dm2=(7.5e-5, 2.4e-3),
                  theta=(0.59, 0.15, 0.785), integrator="dp45", matter=matter, rtol=1e-9,
                  atol=1e-9, h0=0.5)
    s = make_solver(xf, wl)
    s.reset(r0)
    s.evolve(r0, r1)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
    gs = s.stats()
    assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected)
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10


def test_lie_rk4_parity_and_stiff_single_step(xf):
    """Exponential (Eq. U) scheme: multi-step parity where resolved, and one step from random
    states with the small case's configured step (0.0945 km).  The one-step map couples every
    beam through the moments and rotates by theta = h |K| radians per stage; a rounding difference
    in one stage's state changes the next stage's moments and so its rotation angle by theta
    times as much, three stages deep, so differences grow like theta^3 eps: at r = 20 km
    (theta ~ 2e2) parity holds at 1e-10; at r = R (theta ~ 8e3) the test checks the deviation
    stays within theta_max^3 eps."""
    wl = Workload(name="cf", **RAGGED, integrator="lie_rk4", n_steps=100)
    s = make_solver(xf, wl, fixed_dr_km=0.05)
    s.reset(80.0)
    s.evolve(80.0, 85.0)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), 80.0, 85.0)
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10
    wl0 = workload_2f_small_fp64()
    wl0.integrator = "lie_rk4"
    h = (200.0 - 11.0) / 2000
    s0 = make_solver(xf, wl0, fixed_dr_km=h)
    b0 = Bulb(wl0)
    for r, tol in ((20.0, 1e-10), (11.0, None)):
        Yr = random_state(wl0, seed=17)
        s0.set_rho(beams(Yr), r)
        s0.evolve(r, r + h)
        ref = cf4_step(b0.generators, r, Yr, h)
        err = rel_err(s0.get_rho(), beams(ref))
        if tol is None:
            G = b0.generators(r, Yr)
            w = np.linalg.eigvalsh(G)
            theta = h * float((w[..., -1] - w[..., 0]).max())
            tol = theta**3 * 2.2e-16
        assert err < tol, (r, err, tol)


def test_small_workload_full_range(xf):
    """The 4096-beam FP64 case, 2000 fixed RK4 steps, over the radial window where the fixed step
    resolves the precession (100 -> 200 km); plus the lepton-number invariant on the GPU state."""
    wl = workload_2f_small_fp64()
    wl.r0, wl.r1 = 100.0, 200.0
    s = make_solver(xf, wl, fixed_dr_km=(wl.r1 - wl.r0) / wl.n_steps)
    s.reset(100.0)
    s.evolve(100.0, 200.0)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 200.0)
    err = rel_err(s.get_rho(), beams(Y))
    assert err < 1e-10, err


@pytest.mark.parametrize("shape", [(0, 0), (256, 3), (256, 2), (128, 4)])
def test_mixed_precision_against_fp64_oracle(xf, shape):
    """FP32 per-beam algebra with FP64 moments and step control, renormalised |s|: survival
    probabilities within 1e-4 of the FP64 oracle through a window with strong flavour evolution,
    for the default launch shape (one 512-thread block per SM) and the register budgets of the
    other shapes (768 or 512 resident threads per SM)."""
    wl = Workload(name="mx", **RAGGED, integrator="dp45", rtol=1e-9, atol=1e-9, h0=1e-3)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 110.0)
    s = make_solver(xf, wl, precision="mixed", rtol=1e-6, atol=1e-6, block_size=shape[0],
                    blocks_per_sm=shape[1])
    gs = s.stats()
    assert gs.block_size == (shape[0] or 512)
    s.reset(100.0)
    s.evolve(100.0, 110.0)
    pee, mean = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 0.5
    assert np.abs(pee - ref).max() < 1e-4
    assert abs(mean - Bulb(wl).mean_survival(Y)) < 1e-4


@pytest.mark.parametrize("integrator", ["dp45", "rk4"])
def test_mixed_three_flavours_against_fp64_oracle(xf, integrator):
    """Three flavours in mixed precision (FP32 density matrices, FP64 moments and control):
    survival probabilities within 1e-4 of the FP64 oracle through a window with evolution."""
    wl = Workload(name="m3", n_flavor=3, n_energy=13, n_angle=11, dm2=(7.5e-5, 2.4e-3),
                  theta=(0.59, 0.15, 0.785), integrator=integrator, n_steps=300, rtol=1e-9,
                  atol=1e-9, h0=1e-3)
    Y, st = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 103.0)
    s = make_solver(xf, wl, precision="mixed", rtol=1e-6, atol=1e-6, fixed_dr_km=3.0 / 300)
    s.reset(100.0)
    s.evolve(100.0, 103.0)
    pee, _ = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 1e-2
    assert np.abs(pee - ref).max() < 1e-4


def test_mixed_fixed_step_rk4_against_fp64_oracle(xf):
    """Two flavours, mixed precision, fixed-step RK4 (the FP32 pair kernels' RK4 tableau): the same
    200 steps as the oracle's FP64 run, survival probabilities within 1e-4."""
    wl = Workload(name="mr", **RAGGED, integrator="rk4", n_steps=200)
    r0, r1 = 100.0, 110.0
    s = make_solver(xf, wl, precision="mixed", fixed_dr_km=(r1 - r0) / wl.n_steps)
    s.reset(r0)
    s.evolve(r0, r1)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
    pee, _ = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 0.5
    assert np.abs(pee - ref).max() < 1e-4
    assert s.stats().accepted == 200


def test_mixed_lie_rk4_against_fp64_oracle(xf):
    """Two flavours, mixed precision, commutator-free Lie RK4 (FP32 rotations): the same 200
    steps as the oracle's FP64 run, survival probabilities within 1e-4."""
    wl = Workload(name="ml", **RAGGED, integrator="lie_rk4", n_steps=200)
    r0, r1 = 100.0, 110.0
    s = make_solver(xf, wl, precision="mixed", fixed_dr_km=(r1 - r0) / wl.n_steps)
    s.reset(r0)
    s.evolve(r0, r1)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
    pee, _ = s.pee()
    ref = beams(Y)[:, 0, 0].real
    assert np.abs(ref - 1).max() > 0.5
    assert np.abs(pee - ref).max() < 1e-4


def test_bitwise_deterministic(xf):
    wl = Workload(name="det", **RAGGED, integrator="dp45", h0=1e-3)
    outs = []
    for _ in range(2):
        s = make_solver(xf, wl)
        s.reset(100.0)
        s.evolve(100.0, 102.0)
        outs.append(s.get_rho(xf.LAYOUT_NATIVE))
    assert np.array_equal(outs[0], outs[1])


def test_vacuum_on_gpu_matches_closed_form(xf):
    wl = Workload(name="vac", **RAGGED, L={k: 0.0 for k in ("nue", "nuebar", "nux", "nuxbar")},
                  dm2=(2.4e-3, 0.0), theta=(0.3, 0, 0), integrator="dp45", rtol=1e-11, atol=1e-11,
                  h0=1e-3)
    s = make_solver(xf, wl)
    s.evolve(11.0, 31.0)
    pee, _ = s.pee()
    g = Grid.from_workload(wl)
    c = np.sqrt(1 - g.u * 121.0 / 31.0**2)
    L = 31.0 * c - 11.0 * np.sqrt(1 - g.u)
    ph = 2.4e-3 * L[:, None] / (4 * g.E[None, :] * 1e6 * 197.3269804e-12)
    ref = 1 - math.sin(0.6) ** 2 * np.sin(ph) ** 2
    assert np.abs(pee.reshape(2, wl.n_angle, wl.n_energy) - ref[None]).max() < 1e-8


def test_degenerate_cases(xf):
    # theta_v = 0 and no matter: nothing mixes, every beam stays electron flavour exactly
    wl = Workload(name="nomix", n_energy=3, n_angle=2, theta=(0.0, 0, 0), integrator="rk4",
                  n_steps=10, r0=11.0, r1=12.0)
    s = make_solver(xf, wl)
    s.evolve(11.0, 12.0)
    pee, mean = s.pee()
    assert np.all(pee == 1.0) and mean == 1.0
    # one energy, one angle: two beams
    wl1 = Workload(name="one", n_energy=1, n_angle=1, integrator="rk4", n_steps=20, r0=100.0, r1=101.0)
    s1 = make_solver(xf, wl1)
    s1.reset(100.0)
    s1.evolve(100.0, 101.0)
    Y, _ = oracle_run(wl1, Bulb(wl1).initial_state(), 100.0, 101.0)
    assert rel_err(s1.get_rho(), beams(Y)) < 1e-10
    # r1 == r0: no step
    s1.evolve(101.0, 101.0)
    assert s1.stats().accepted == 20


def test_call_order_and_arguments(xf):
    wl = Workload(name="ord", n_energy=4, n_angle=3)
    s = xf.Solver(xf.config_from_workload(wl, fixed_dr_km=0.1))
    with pytest.raises(xf.XflatError) as e:
        s.evolve(11.0, 12.0)
    assert e.value.code == xf.ERR_STATE
    s.set_spectra(Grid.from_workload(wl).N)
    with pytest.raises(xf.XflatError) as e:
        s.evolve(12.0, 13.0)                       # r0 is not the current radius
    assert e.value.code == xf.ERR_STATE
    bad = np.full((2, 2, 4), np.nan)
    with pytest.raises(xf.XflatError) as e:
        s.set_spectra(bad)
    assert e.value.code == xf.ERR_INVAL


def test_nonfinite_state_is_reported(xf):
    wl = Workload(name="nan", n_energy=4, n_angle=3, integrator="rk4", n_steps=2, r0=50.0, r1=51.0)
    s = make_solver(xf, wl)
    Y = beams(random_state(wl, seed=2))
    Y[5, 0, 1] = np.nan
    s.set_rho(Y, 50.0)
    with pytest.raises(xf.XflatError) as e:
        s.evolve(50.0, 51.0)
    assert e.value.code == xf.ERR_NONFINITE


def test_step_underflow_is_reported(xf):
    """DP45 from the neutrino sphere with the r^-3 matter potential (~1.5e6 /km at 11 km) and a
    step floor far above the step that potential allows: every trial step is rejected, the step
    shrinks below h_min and the call reports XFLAT_ERR_STEP; the handle stays usable."""
    wl = Workload(name="uf", n_energy=8, n_angle=4, integrator="dp45", matter="power_law", h0=1e-2)
    s = make_solver(xf, wl, h_min_km=1e-4)
    s.reset(11.0)
    with pytest.raises(xf.XflatError) as e:
        s.evolve(11.0, 12.0)
    assert e.value.code == xf.ERR_STEP
    st = s.stats()
    assert st.status == xf.ERR_STEP and st.accepted == 0 and st.rejected >= 3
    assert st.r_km == 11.0


def test_barrier_timeout_returns_status_and_context_survives(xf):
    """A barrier that waits for one arrival too many gives up after the configured limit; the call
    reports XFLAT_ERR_TIMEOUT and the next call on the same device works."""
    wl = Workload(name="to", n_energy=8, n_angle=4, integrator="rk4", n_steps=4, r0=100.0, r1=101.0)
    s = make_solver(xf, wl, barrier_timeout_ns=50_000_000)
    s.reset(100.0)
    s.debug_barrier_extra(1)
    with pytest.raises(xf.XflatError) as e:
        s.evolve(100.0, 101.0)
    assert e.value.code == xf.ERR_TIMEOUT
    s.debug_barrier_extra(0)
    s.reset(100.0)
    s.evolve(100.0, 101.0)
    Y, _ = oracle_run(wl, Bulb(wl).initial_state(), 100.0, 101.0)
    assert rel_err(s.get_rho(), beams(Y)) < 1e-10
