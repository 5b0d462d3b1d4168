"""Parity at the full sizes of the forward workloads, on outputs the oracle can still compute.

Each case starts from seeded, coherent random states at r = R (every beam near the same flavour
state, so the nu-nu moments are large and the coupling between beams matters) and takes a few
adaptive steps with a first trial step small enough that every attempt is accepted; the oracle
takes the same steps on the same inputs.

* 4,000,000 beams, two flavours, mixed precision, DP45, matter: the launch shape the benchmark
  times (the autotuner's choice), one step (the oracle's numpy right-hand side takes seconds per
  evaluation at this size), plus the moments of the whole state against the oracle's sums.
* 262,144 beams, three flavours, FP64, DP45, matter: three steps, 1e-10.
* 64 instances (about 28 M beams), two flavours, mixed, DP45, matter: all instances advance in
  one launch; the three smallest are compared with the oracle instance by instance.
"""
import numpy as np
import pytest

from bulb_inputs import (coherent_unit_states, workload_2f_large, workload_3f_fp64,
                         batched_workloads)
from oracle.physics import Bulb, Grid
from oracle.integrate import evolve_adaptive
from parity_util import beams, rel_err

pytestmark = pytest.mark.gpu


def coherent_state(wl, seed):
    n = wl.n_flavor
    psi = coherent_unit_states(n, wl.n_beams, seed).reshape(2, wl.n_angle, wl.n_energy, n)
    return psi[..., :, None] * np.conj(psi[..., None, :])


def bloch(Y):
    """Bloch vectors (2 flavours) of beam-major matrices [n, 2, 2]."""
    return np.stack([2 * Y[:, 0, 1].real, -2 * Y[:, 0, 1].imag, (Y[:, 0, 0] - Y[:, 1, 1]).real], axis=1)


def test_large_2f_mixed_full_size(xf):
    from paper_1912_10596_gb300 import autotune
    wl = workload_2f_large("mixed")
    h0 = 5e-10
    cfg = xf.config_from_workload(wl, steps_per_launch=1, h0_km=h0)
    shape = autotune.tune(xf, [xf.config_from_workload(wl, steps_per_launch=1)], [wl.spectra()], [wl.r1])
    cfg.block_size, cfg.blocks_per_sm = shape
    s = xf.Solver(cfg)
    s.set_spectra(wl.spectra())
    Y0 = coherent_state(wl, seed=21)
    s.set_rho(beams(Y0), wl.r0)
    b = Bulb(wl)
    # moments of the whole 4M-beam state: device reduction of the FP32 state vs the oracle's sums
    # of the same (rounded) state
    Yr = s.get_rho().reshape(Y0.shape)
    J0, J1 = s.moments()
    R0, R1 = b.moment_matrices(wl.r0, Yr)
    # the sums are FP64-accurate (pinned exactly in test_mixed_reduction_gpu); what remains is the
    # FP32 rounding of the weights, here systematic: du = 1/2000 is not a float (3.8e-8 relative)
    assert np.abs(J0 - R0).max() <= 1e-7 * np.abs(R0).max()
    assert np.abs(J1 - R1).max() <= 1e-7 * np.abs(R1).max()
    assert abs(R1[0, 1]) > 0.1 * abs(R1[0, 0] - R1[1, 1])          # coherent: large off-diagonal
    s.advance([wl.r1], max_steps=1)
    st = s.stats()
    assert (st.accepted, st.rejected, st.status) == (1, 0, 0)
    Y, r, ost = evolve_adaptive(b, Y0, wl.r0, wl.r1, wl.rtol, wl.atol, h0, max_attempts=1)
    assert ost.accepted == 1 and abs(st.r_km - r) < 1e-15 * r
    got, ref, start = bloch(s.get_rho()), bloch(beams(Y)), bloch(beams(Y0))
    moved = np.linalg.norm(ref - start, axis=1)
    assert moved.max() > 1e-2                                       # the step rotated the states
    assert np.abs(got - ref).max() < 2e-6
    assert (np.linalg.norm(got - ref, axis=1) / np.maximum(moved, 1e-3)).max() < 2e-3


def test_3f_fp64_full_size(xf):
    wl = workload_3f_fp64()
    h0 = 1e-11
    s = xf.Solver(xf.config_from_workload(wl, h0_km=h0))
    s.set_spectra(Grid.from_workload(wl).N)
    Y0 = coherent_state(wl, seed=22)
    s.set_rho(beams(Y0), wl.r0)
    s.advance([wl.r1], max_steps=3)
    st = s.stats()
    Y, r, ost = evolve_adaptive(Bulb(wl), Y0, wl.r0, wl.r1, wl.rtol, wl.atol, h0, max_attempts=3)
    assert (st.accepted, st.rejected) == (ost.accepted, ost.rejected) == (3, 0)
    assert abs(st.r_km - r) < 1e-14 * r
    got = s.get_rho()
    assert rel_err(beams(Y), beams(Y0)) > 1e-3
    assert rel_err(got, beams(Y)) < 1e-10


def test_batched_64_instances_full_size(xf):
    wls = batched_workloads()
    h0 = 4e-11
    cfgs = [xf.config_from_workload(wl, h0_km=h0) for wl in wls]
    s = xf.Solver(cfgs)
    sample = sorted(range(len(wls)), key=lambda i: wls[i].n_beams)[:3]
    states = {}
    for i, wl in enumerate(wls):
        s.set_spectra(wl.spectra(), inst=i)
        Y0 = coherent_state(wl, seed=100 + i)
        if i in sample:
            states[i] = Y0
        s.set_rho(beams(Y0), wl.r0, inst=i)
    total = sum(wl.n_beams for wl in wls)
    assert total > 2e7
    s.advance([wl.r1 for wl in wls], max_steps=3)
    for i in range(len(wls)):
        st = s.stats(inst=i)
        assert (st.accepted, st.rejected, st.status) == (3, 0, 0), i
    for i in sample:
        wl = wls[i]
        Y, r, ost = evolve_adaptive(Bulb(wl), states[i], wl.r0, wl.r1, wl.rtol, wl.atol, h0,
                                    max_attempts=3)
        assert ost.accepted == 3
        assert abs(s.stats(inst=i).r_km - r) < 1e-15 * r
        got, ref = bloch(s.get_rho(inst=i)), bloch(beams(Y))
        moved = np.linalg.norm(ref - bloch(beams(states[i])), axis=1)
        assert moved.max() > 3e-3, i
        assert np.abs(got - ref).max() < 2e-6, i
