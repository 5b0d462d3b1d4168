"""One problem over several GPUs, emulated on one: beam-shard handles run each pass in turn and the
host adds their partial moments exactly between passes (the paper's per-evaluation sum over ranks,
Sec. 3.3).  No kernel waits for another: every pass of every shard is a separate launch."""
import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Grid
from paper_1912_10596_gb300 import shard
from parity_util import make_solver, rel_err

pytestmark = pytest.mark.gpu

# 64 E x 320 u x 2 = 40,960 beams: the unsharded grid has one block per 1024 beams (256 threads) or
# 2048 (512 threads), so halves of the beam range fall on block boundaries


def shards_of(xf, wl, bounds, **over):
    g = Grid.from_workload(wl)
    out = []
    for lo, hi in bounds:
        s = xf.Solver(xf.config_from_workload(wl, **over), shard=(lo, hi))
        s.set_spectra(g.N)
        out.append(s)
    return out


@pytest.mark.parametrize("precision,integrator,tol", [("fp64", "dp45", 1e-9), ("mixed", "dp45", 1e-6),
                                                      ("fp64", "rk4", 0)])
def test_two_shards_reproduce_the_unsharded_run_bit_for_bit(xf, precision, integrator, tol):
    wl = Workload(name="sh", n_energy=64, n_angle=320, integrator=integrator, precision=precision,
                  rtol=tol or 1e-9, atol=tol or 1e-9, h0=1e-3, n_steps=40, r0=100.0, r1=101.0)
    over = {} if integrator != "rk4" else {"fixed_dr_km": 1.0 / 40}
    full = make_solver(xf, wl, **over)
    full.reset(100.0)
    full.evolve(100.0, 101.0)
    n = wl.n_beams
    parts = shards_of(xf, wl, [(0, n // 2), (n // 2, n)], **over)
    for s in parts:
        s.reset(100.0)
    steps = shard.evolve_sharded(parts, 101.0)
    st = full.stats()
    assert steps == st.accepted + st.rejected
    ref = full.get_rho(xf.LAYOUT_NATIVE)
    got = np.concatenate([parts[0].get_rho(xf.LAYOUT_NATIVE)[:, : n // 2],
                          parts[1].get_rho(xf.LAYOUT_NATIVE)[:, n // 2:]], axis=1)
    assert np.abs(ref - 1.0 * (np.arange(3)[:, None] == 2)).max() > 1e-3   # the states moved
    assert np.array_equal(got, ref)
    for s in parts:
        assert (s.stats().accepted, s.stats().rejected) == (st.accepted, st.rejected)


def test_lie_adaptive_shards(xf):
    """The adaptive exact propagators sharded in two on the block boundaries: the same steps and the
    states to 1e-12 (the sharded run repeats bit for bit; it differs from the one-launch run by
    ~1e-13, unlike the other integrators, which match it bit for bit)."""
    wl = Workload(name="shl", n_energy=64, n_angle=320, integrator="lie_adaptive", rtol=1e-9, atol=1e-9,
                  h0=1e-3)
    full = make_solver(xf, wl)
    full.reset(100.0)
    full.evolve(100.0, 101.0)
    n = wl.n_beams
    outs = []
    for rep in range(2):
        parts = shards_of(xf, wl, [(0, n // 2), (n // 2, n)])
        for s in parts:
            s.reset(100.0)
        steps = shard.evolve_sharded(parts, 101.0)
        outs.append(np.concatenate([parts[0].get_rho(xf.LAYOUT_NATIVE)[:, : n // 2],
                                    parts[1].get_rho(xf.LAYOUT_NATIVE)[:, n // 2:]], axis=1))
    st = full.stats()
    assert steps == st.accepted + st.rejected
    assert np.array_equal(outs[0], outs[1])
    assert np.abs(outs[0] - full.get_rho(xf.LAYOUT_NATIVE)).max() < 1e-12


def test_uneven_shards_agree_with_the_unsharded_run(xf):
    """Three shards of uneven sizes (other block decompositions, so other roundings inside each
    block): the same steps and the states to 1e-12."""
    wl = Workload(name="sh3", n_energy=37, n_angle=29, integrator="dp45", rtol=1e-9, atol=1e-9, h0=0.5)
    full = make_solver(xf, wl)
    full.reset(100.0)
    full.evolve(100.0, 102.0)
    n = wl.n_beams
    bounds = [(0, 512), (512, 1536), (1536, n)]
    parts = shards_of(xf, wl, bounds)
    for s in parts:
        s.reset(100.0)
    shard.evolve_sharded(parts, 102.0)
    st = full.stats()
    assert st.rejected > 0
    got = full.get_rho().copy()
    for s, (lo, hi) in zip(parts, bounds):
        assert (s.stats().accepted, s.stats().rejected) == (st.accepted, st.rejected)
        got[lo:hi] = s.get_rho()[lo:hi]
    assert rel_err(got, full.get_rho()) < 1e-12


def test_shard_handle_rejects_the_plain_calls(xf):
    wl = Workload(name="shx", n_energy=8, n_angle=8, integrator="dp45", rtol=1e-9, atol=1e-9)
    s = shards_of(xf, wl, [(0, 64)])[0]
    with pytest.raises(xf.XflatError) as e:
        s.evolve(11.0, 12.0)
    assert e.value.code == xf.ERR_STATE
    with pytest.raises(xf.XflatError):
        xf.Solver(xf.config_from_workload(wl), shard=(3, 64))      # lower bound not a multiple of 4


@pytest.mark.parametrize("integrator,tol", [("dp45", 1e-9), ("lie_adaptive", 1e-9)])
def test_three_flavour_shards(xf, integrator, tol):
    """Three flavours (18 moment words per partial): two shard handles on the block boundaries take
    the unsharded run's steps and reproduce its states (DP45 bit for bit; the adaptive exponential
    integrator to 1e-12, as for two flavours)."""
    wl = Workload(name="sh3f", n_flavor=3, n_energy=64, n_angle=160, dm2=(7.5e-5, 2.4e-3),
                  theta=(0.59, 0.15, 0.785), integrator=integrator, rtol=tol, atol=tol, h0=0.5)
    full = make_solver(xf, wl)
    full.reset(100.0)
    full.evolve(100.0, 101.0)
    n = wl.n_beams
    parts = shards_of(xf, wl, [(0, n // 2), (n // 2, n)])
    for s in parts:
        s.reset(100.0)
    steps = shard.evolve_sharded(parts, 101.0)
    st = full.stats()
    assert steps == st.accepted + st.rejected
    for s in parts:
        assert (s.stats().accepted, s.stats().rejected) == (st.accepted, st.rejected)
    ref = full.get_rho(xf.LAYOUT_NATIVE)
    got = np.concatenate([parts[0].get_rho(xf.LAYOUT_NATIVE)[:, : n // 2],
                          parts[1].get_rho(xf.LAYOUT_NATIVE)[:, n // 2:]], axis=1)
    if integrator == "dp45":
        assert np.array_equal(got, ref)
    else:
        assert np.abs(got - ref).max() < 1e-12
