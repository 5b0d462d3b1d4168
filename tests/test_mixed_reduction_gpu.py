"""The mixed kernels' moment reduction (Eq. F, Sec. 3.4's reduction over all beams) loses nothing to
FP32 accumulation.

Each beam's contribution w_b s_b is formed in FP32 (per-beam algebra) and from there summed exactly
(fixed-point int64 per thread, exact integer warp, block and grid sums).  With weights that are
exact in FP32 (power-of-two angle bins, integer spectra summing to a power of two) and a state
whose components carry 12 significant bits, every FP32 product is exact too, so the device's
J1 = sum_b du_j F_b must equal the exact sum (math.fsum of the FP64 products) up to the final
conversions to double.  An FP32 accumulator, even a pairwise tree, misses this by ~1e-7.
"""
import math

import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Bulb, Grid

pytestmark = pytest.mark.gpu


def bloch(M):
    """Bloch vector j of a traceless 2x2 Hermitian M = (1/2) j . sigma."""
    return np.array([2 * M[0, 1].real, -2 * M[0, 1].imag, (M[0, 0] - M[1, 1]).real])


def exact_case(n_energy, n_angle, seed):
    rng = np.random.default_rng(seed)
    N = rng.integers(0, 1024, size=(2, 2, n_energy)).astype(np.float64)
    N[0, 0, 0] += N.sum() % 2
    rest = 2.0 ** math.ceil(math.log2(N.sum())) - N.sum()          # even
    N[1, :, 0] += rest / 2          # total number a power of two; every N_e - N_x stays below 2^10
    wl = Workload(name="exact", n_energy=n_energy, n_angle=n_angle, precision="mixed",
                  integrator="dp45", rtol=1e-6, atol=1e-6)
    s = rng.standard_normal((3, wl.n_beams))
    s /= np.linalg.norm(s, axis=0)
    s = np.round(s * 2048.0) / 2048.0                            # 12 significant bits at most
    return wl, N, s


@pytest.mark.parametrize("n_energy,n_angle", [(401, 512), (1000, 256)])
def test_mixed_j1_reduction_is_exact(xf, n_energy, n_angle):
    """410,624 beams with an odd energy count (beam pairs straddle angle bins: both the packed and
    the scalar accumulation paths) and 512,000 beams with an even one; J1 to 1e-13 relative."""
    wl, N, s = exact_case(n_energy, n_angle, seed=n_energy)
    sv = xf.Solver(xf.config_from_workload(wl, steps_per_launch=1))
    sv.set_spectra(N)
    sv.set_rho(s, 40.0, layout=xf.LAYOUT_NATIVE)
    J0, J1 = sv.moments()
    du = 1.0 / n_angle
    g = np.stack([N[0, 0] - N[0, 1], -(N[1, 0] - N[1, 1])])       # signed weights, nu and nubar
    w = (du * np.broadcast_to(g[:, None, :], (2, n_angle, n_energy))).ravel()
    ref = np.array([math.fsum(w * s[c]) for c in range(3)])
    scale = math.fsum(np.abs(w))
    got = bloch(J1)
    assert np.abs(got - ref).max() <= 1e-13 * scale, (got, ref)
    # J0 carries the FP32 geometry factor 1/cos theta of each angle bin: against the oracle's FP64
    # moments of the same state, within FP32 rounding of that factor
    Y = np.empty((wl.n_beams, 2, 2), dtype=np.complex128)
    Y[:, 0, 0] = 0.5 * (1 + s[2])
    Y[:, 1, 1] = 0.5 * (1 - s[2])
    Y[:, 0, 1] = 0.5 * (s[0] - 1j * s[1])
    Y[:, 1, 0] = np.conj(Y[:, 0, 1])
    Y[wl.n_beams // 2:] = np.conj(Y[wl.n_beams // 2:])            # nubar beams hold conj(Pbar)
    grid = Grid.from_workload(wl, N=N)
    R0, R1 = Bulb(wl, grid=grid).moment_matrices(40.0, Y.reshape(2, n_angle, n_energy, 2, 2))
    assert np.abs(J1 - R1).max() <= 1e-13 * scale
    assert np.abs(J0 - R0).max() <= 1e-6 * np.abs(R0).max()
    sv.close()
