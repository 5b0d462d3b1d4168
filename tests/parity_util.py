"""Shared helpers of the GPU parity tests: run the oracle and the CUDA path on the same inputs."""
import numpy as np

from bulb_inputs import Workload, random_unit_states
from oracle.physics import Bulb, Grid
from oracle.integrate import evolve_fixed, evolve_adaptive, evolve_em2, evolve_lie_adaptive


def beams(Y):
    """Oracle state [2, N_u, N_E, n, n] -> beam-major [n_beams, n, n] (species, angle, energy)."""
    n = Y.shape[-1]
    return Y.reshape(-1, n, n)


def rel_err(A, B):
    """max_b ||A_b - B_b||_F / ||B_b||_F over beams."""
    num = np.sqrt((np.abs(A - B) ** 2).sum(axis=(-2, -1)))
    den = np.sqrt((np.abs(B) ** 2).sum(axis=(-2, -1)))
    return float((num / den).max())


def random_state(wl, seed):
    """Pure random density matrices for every beam, in the oracle's [2, N_u, N_E, n, n] shape."""
    n = wl.n_flavor
    psi = random_unit_states(n, wl.n_beams, seed).reshape(2, wl.n_angle, wl.n_energy, n)
    return psi[..., :, None] * np.conj(psi[..., None, :])


def make_solver(xf, wl, grid=None, **over):
    cfg = xf.config_from_workload(wl, **over)
    s = xf.Solver(cfg)
    g = grid if grid is not None else Grid.from_workload(wl)
    default_u = np.allclose(g.u, (np.arange(wl.n_angle) + 0.5) / wl.n_angle) and np.allclose(g.du, 1.0 / wl.n_angle)
    if default_u:
        s.set_spectra(g.N)
    else:
        s.set_spectra(g.N, g.u, g.du)
    if wl.matter == "table":
        s.set_matter_table(wl.matter_table_r, wl.matter_table_lambda)
    return s


def oracle_run(wl, Y0, r0, r1, grid=None):
    b = Bulb(wl, grid=grid)
    if wl.integrator == "exp_midpoint":
        Y, r, st = evolve_em2(b, Y0, r0, r1, wl.rtol, wl.atol, wl.h0)
        return Y, st
    if wl.integrator == "lie_adaptive":
        Y, r, st = evolve_lie_adaptive(b, Y0, r0, r1, wl.rtol, wl.atol, wl.h0)
        return Y, st
    if wl.integrator == "dp45":
        Y, r, st = evolve_adaptive(b, Y0, r0, r1, wl.rtol, wl.atol, wl.h0)
        return Y, st
    Y, st = evolve_fixed(b, Y0, r0, r1, wl.n_steps, wl.integrator)
    return Y, st
