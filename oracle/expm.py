"""Exponentials exp(-i H dl) of Hermitian matrices (test infrastructure only).

two_flavor_propagator follows Eq. U of the paper (Sec. 3.4): with the trace removed first
(Eq. U assumes h22 = -h11), h11 and h12 the diagonal and off-diagonal elements and
lambda = sqrt(h11^2 + |h12|^2),

    U = (1/lambda) [[lambda cos(lambda dl) - i h11 sin(lambda dl),  -i h12 sin(lambda dl)],
                    [-i h12^* sin(lambda dl),  lambda cos(lambda dl) + i h11 sin(lambda dl)]]

times the phase exp(-i tr(H)/2 dl) of the removed trace.  hermitian_propagator is the general
n x n case by eigendecomposition (numpy.linalg.eigh), used for three flavours and as a check.
"""
from __future__ import annotations

import numpy as np


def two_flavor_propagator(H: np.ndarray, dl=1.0) -> np.ndarray:
    """exp(-i H dl) for a stack of 2x2 Hermitian H [..., 2, 2] by Eq. U."""
    dl = np.asarray(dl, dtype=np.float64)
    h0 = 0.5 * (H[..., 0, 0].real + H[..., 1, 1].real)
    h11 = 0.5 * (H[..., 0, 0].real - H[..., 1, 1].real)
    h12 = H[..., 0, 1]
    lam = np.sqrt(h11 * h11 + (h12 * np.conj(h12)).real)
    x = lam * dl
    cosx = np.cos(x)
    # sin(lambda dl) / lambda, finite at lambda = 0 (np.sinc(t) = sin(pi t)/(pi t))
    s_over_lam = dl * np.sinc(x / np.pi)
    U = np.empty(H.shape, dtype=np.complex128)
    U[..., 0, 0] = cosx - 1j * h11 * s_over_lam
    U[..., 0, 1] = -1j * h12 * s_over_lam
    U[..., 1, 0] = -1j * np.conj(h12) * s_over_lam
    U[..., 1, 1] = cosx + 1j * h11 * s_over_lam
    phase = np.exp(-1j * h0 * dl)
    return U * phase[..., None, None]


def hermitian_propagator(H: np.ndarray, dl=1.0) -> np.ndarray:
    """exp(-i H dl) for a stack of Hermitian H [..., n, n] via H = V diag(w) V^dag."""
    w, V = np.linalg.eigh(H)
    ph = np.exp(-1j * w * np.asarray(dl, dtype=np.float64)[..., None])
    return (V * ph[..., None, :]) @ np.conj(np.swapaxes(V, -1, -2))


def propagator(H: np.ndarray, dl=1.0) -> np.ndarray:
    """Eq. U for two flavours, eigendecomposition otherwise."""
    if H.shape[-1] == 2:
        return two_flavor_propagator(H, dl)
    return hermitian_propagator(H, dl)


def conjugate_by(U: np.ndarray, P: np.ndarray) -> np.ndarray:
    """U P U^dagger: the density-matrix form of psi -> U psi."""
    return U @ P @ np.conj(np.swapaxes(U, -1, -2))
