"""Batched instances: many independent bulb problems of uneven sizes advanced together by one
persistent launch, each with its own radius, step size, error control and moments.

Every instance is checked against its own oracle run and against the same instance solved alone,
and a CUDA-graph replay of the persistent launches against the same launches issued one by one.
"""
import numpy as np
import pytest

from bulb_inputs import Workload, batched_workloads
from oracle.physics import Bulb, Grid
from oracle.integrate import evolve_adaptive
from parity_util import beams, rel_err, random_state, make_solver, oracle_run

pytestmark = pytest.mark.gpu


def make_batch(xf, wls, **over):
    cfgs = [xf.config_from_workload(wl, **over) for wl in wls]
    s = xf.Solver(cfgs)
    for i, wl in enumerate(wls):
        s.set_spectra(Grid.from_workload(wl).N, inst=i)
    return s


def ic(wl):
    return beams(Bulb(wl).initial_state())


def fp64_instances():
    """Three FP64 DP45 instances: different sizes (one ragged, one with fewer beams than a block),
    hierarchies, mixing angles, luminosities, matter profiles and radial windows."""
    L3 = {k: 3e51 for k in ("nue", "nuebar", "nux", "nuxbar")}
    L03 = {k: 3e50 for k in ("nue", "nuebar", "nux", "nuxbar")}
    wls = [
        Workload(name="b0", n_energy=37, n_angle=29, integrator="dp45", h0=0.5),
        Workload(name="b1", n_energy=11, n_angle=7, dm2=(2.4e-3, 0.0), theta=(0.05, 0, 0), L=L3,
                 matter="power_law", integrator="dp45", h0=0.5),
        Workload(name="b2", n_energy=64, n_angle=3, theta=(0.2, 0, 0), L=L03, integrator="dp45", h0=0.2),
    ]
    windows = [(100.0, 104.0), (300.0, 301.0), (100.0, 102.5)]
    return wls, windows


def test_batch_instances_match_oracle_and_standalone(xf):
    wls, win = fp64_instances()
    s = make_batch(xf, wls)
    for i, (wl, (r0, _)) in enumerate(zip(wls, win)):
        s.set_rho(ic(wl), r0, inst=i)
    s.evolve_batch([r1 for _, r1 in win])
    for i, (wl, (r0, r1)) in enumerate(zip(wls, win)):
        Y, st = oracle_run(wl, Bulb(wl).initial_state(), r0, r1)
        gs = s.stats(inst=i)
        assert gs.r_km == r1
        assert (gs.accepted, gs.rejected) == (st.accepted, st.rejected), i
        got = s.get_rho(inst=i)
        assert rel_err(got, beams(Y)) < 1e-10, i
        # the same instance solved alone: a different cut of beams into blocks, so only the
        # rounding of the block partial sums may differ
        a = make_solver(xf, wl)
        a.set_rho(ic(wl), r0)
        a.evolve(r0, r1)
        sa = a.stats()
        assert (sa.accepted, sa.rejected) == (gs.accepted, gs.rejected)
        assert rel_err(got, a.get_rho()) < 1e-12, i
        J0b, J1b = s.moments(inst=i)
        J0a, J1a = a.moments()
        assert np.abs(J0b - J0a).max() <= 1e-12 * np.abs(J0a).max()
        assert np.abs(J1b - J1a).max() <= 1e-12 * np.abs(J1a).max()


def test_batch_instances_finish_independently(xf):
    """An instance whose target is already reached does not move while the others advance."""
    wls, win = fp64_instances()
    s = make_batch(xf, wls)
    for i, (wl, (r0, _)) in enumerate(zip(wls, win)):
        s.set_rho(ic(wl), r0, inst=i)
    before = s.get_rho(xf.LAYOUT_NATIVE, inst=1)
    s.evolve_batch([win[0][1], win[1][0], win[2][1]])
    assert np.array_equal(s.get_rho(xf.LAYOUT_NATIVE, inst=1), before)
    assert s.stats(inst=1).accepted == 0
    assert s.stats(inst=0).r_km == win[0][1] and s.stats(inst=2).r_km == win[2][1]


def small_mixed_instances(n=5):
    """Instances drawn like the 64-instance case (seeded sizes, luminosities, hierarchies and
    angles), shrunk, and without matter so a 5 km window shows strong collective evolution."""
    wls = batched_workloads(n_instances=n, n_energy_range=(9, 40), n_angle_range=(5, 30), r1=105.0)
    for wl in wls:
        wl.matter = "none"
        wl.h0 = 1e-3
    return wls


def test_mixed_batch_against_fp64_oracle(xf):
    wls = small_mixed_instances()
    s = make_batch(xf, wls)
    s.reset(100.0)
    s.evolve_batch([105.0] * len(wls))
    for i, wl in enumerate(wls):
        b = Bulb(wl)
        Y, r, _ = evolve_adaptive(b, b.initial_state(), 100.0, 105.0, 1e-9, 1e-9, 1e-3)
        ref = beams(Y)[:, 0, 0].real
        pee, mean = s.pee(inst=i)
        assert np.abs(pee - ref).max() < 1e-4, i
        assert abs(mean - b.mean_survival(Y)) < 1e-4, i
        assert s.stats(inst=i).r_km == 105.0


def test_graph_replay_equals_plain_launches(xf):
    """n persistent launches captured once into a CUDA graph and replayed give bit-identical states
    and step statistics to the same launches issued one by one."""
    wls = small_mixed_instances(6)
    out = []
    for graph in (False, True):
        s = make_batch(xf, wls)
        s.reset(100.0)
        s.advance([105.0] * len(wls), max_steps=3)
        if graph:
            s.advance_graph(4, max_steps=3)
            s.advance_graph(4, max_steps=3)          # replay of the cached graph
        else:
            for _ in range(8):
                s.advance(None, max_steps=3)
        st = [s.stats(inst=i) for i in range(len(wls))]
        out.append(([s.get_rho(xf.LAYOUT_NATIVE, inst=i) for i in range(len(wls))],
                    [(x.r_km, x.h_km, x.accepted, x.rejected) for x in st]))
        assert st[0].launches == 1 + 1 + 8
    assert out[0][1] == out[1][1]
    assert all(r > 100.0 for r, *_ in out[0][1])
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)


def test_graph_needs_a_preceding_advance(xf):
    wls = small_mixed_instances(2)
    s = make_batch(xf, wls)
    s.reset(100.0)
    with pytest.raises(xf.XflatError) as e:
        s.advance_graph(2, max_steps=1)
    assert e.value.code == xf.ERR_STATE
    s.advance([101.0, 101.0], max_steps=1)
    with pytest.raises(xf.XflatError) as e:
        s.advance_graph(0, max_steps=1)
    assert e.value.code == xf.ERR_INVAL
