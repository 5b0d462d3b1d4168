"""Pins of the oracle's extended bulb model (oracle/extended.py).

* The paper's own validation (Sec. 3.5): with the axial symmetry unbroken, the extended bulb
  model gives the bulb model's result, direction by direction.
* Rotating the initial state by one azimuthal bin rotates the result by one bin (the potential
  depends on phi - phi' only): a sign or index slip in the sin/cos terms breaks it.
* A state with a cos(phi) (sin(phi)) flavour modulation has Phi_sc (Phi_ss) by hand and the other
  azimuthal moment zero.
"""
import numpy as np
import pytest

from bulb_inputs import Workload, random_unit_states
from oracle.physics import Bulb
from oracle.extended import ExtendedBulb
from oracle.integrate import evolve_fixed


def _case(n_phi=5):
    wl = Workload(name="ext", n_energy=4, n_angle=3, integrator="rk4", n_steps=60)
    return wl, ExtendedBulb(wl, n_phi), Bulb(wl)


def test_axial_symmetry_reduces_to_bulb():
    wl, eb, b = _case()
    Ye, _ = evolve_fixed(eb, eb.initial_state(), 100.0, 103.0, 60)
    Yb, _ = evolve_fixed(b, b.initial_state(), 100.0, 103.0, 60)
    assert np.abs(Yb[..., 0, 0].real - 1).max() > 1e-2               # the bulb state evolved
    for p in range(eb.n_phi):
        assert np.abs(Ye[:, :, p] - Yb).max() < 1e-13


def random_extended_state(eb, seed):
    n = eb.n
    shape = (2, len(eb.grid.u), eb.n_phi, len(eb.grid.E))
    psi = random_unit_states(n, int(np.prod(shape)), seed).reshape(*shape, n)
    # near-electron states with a random azimuthal pattern (large, coherent moments)
    psi = psi * 0.3
    psi[..., 0] += 1.0
    psi /= np.linalg.norm(psi, axis=-1, keepdims=True)
    return psi[..., :, None] * np.conj(psi[..., None, :])


def test_azimuthal_shift_symmetry():
    wl, eb, _ = _case(n_phi=6)
    Y0 = random_extended_state(eb, 31)
    Y, _ = evolve_fixed(eb, Y0, 100.0, 101.0, 40)
    Ys, _ = evolve_fixed(eb, np.roll(Y0, 1, axis=2), 100.0, 101.0, 40)
    assert np.abs(np.roll(Y, 1, axis=2) - Ys).max() < 1e-12
    _, _, Phisc, Phiss = eb.moments(100.0, eb.flux_matrices(Y0[0], Y0[1]))
    assert np.abs(Phisc).max() > 1e-3 * np.abs(eb.moments(100.0, eb.flux_matrices(Y0[0], Y0[1]))[0]).max()


def test_cos_phi_modulation_moments():
    wl, eb, _ = _case(n_phi=8)
    eps = 0.01
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = eb.initial_state()
    Y = Y + eps * np.cos(eb.phi)[None, None, :, None, None, None] * X
    r = 60.0
    Phi1, Phic, Phisc, Phiss = eb.moments(r, eb.flux_matrices(Y[0], Y[1]))
    g = eb.grid
    c = eb.cos_theta(r)
    s = np.sqrt(1 - c * c)
    w = g.du * wl.R_km**2 / (2 * r * r * c) / eb.n_phi
    # F = (N_e - N_x) P + N_x I - conj((Nbar_e - Nbar_x) Pbar + Nbar_x I); the X part carries
    # (N_e - N_x) - (Nbar_e - Nbar_x) (X is real), and sum_p cos^2 phi_p = n_phi / 2
    d = (g.N[0, 0] - g.N[0, 1]).sum() - (g.N[1, 0] - g.N[1, 1]).sum()
    want = eps * (w * s).sum() * d * eb.n_phi / 2 * X
    assert np.abs(Phisc - want).max() < 1e-12 * np.abs(want).max()
    assert np.abs(Phiss).max() < 1e-12 * np.abs(want).max()


def test_sin_phi_modulation_moments():
    """A sin(phi) flavour modulation: Phi_ss by hand and Phi_sc = 0 (the mirror of the cos(phi)
    case; a swapped cos/sin weight or a sign slip in the sin phi' term fails one of the two)."""
    wl, eb, _ = _case(n_phi=8)
    eps = 0.02
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = eb.initial_state() + eps * np.sin(eb.phi)[None, None, :, None, None, None] * X
    r = 45.0
    Phi1, Phic, Phisc, Phiss = eb.moments(r, eb.flux_matrices(Y[0], Y[1]))
    g = eb.grid
    c = eb.cos_theta(r)
    s = np.sqrt(1 - c * c)
    w = g.du * wl.R_km**2 / (2 * r * r * c) / eb.n_phi
    d = (g.N[0, 0] - g.N[0, 1]).sum() - (g.N[1, 0] - g.N[1, 1]).sum()
    want = eps * (w * s).sum() * d * eb.n_phi / 2 * X          # sum_p sin^2 phi_p = n_phi / 2
    assert np.abs(Phiss - want).max() < 1e-12 * np.abs(want).max()
    assert np.abs(Phisc).max() < 1e-12 * np.abs(want).max()
