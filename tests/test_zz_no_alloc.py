"""The allocation-free moment entry point (xflat_moments_2f_noalloc) against xflat_moments.

xflat_moments_2f_noalloc serves callers that cannot allocate device memory when they need the
moments (a host framework that owns the device memory pool, or a loop that must not stall on
cudaMalloc).  It reuses one fixed scratch array in the library image, so the test calls it twice
in a row and checks both results against the handle-based entry point.  This file is collected
last so that a failure here does not hide any other test.
"""
import ctypes

import numpy as np
import pytest

from bulb_inputs import Workload
from oracle.physics import Grid
from parity_util import beams, random_state, make_solver

pytestmark = pytest.mark.gpu


def bloch(J):
    """Bloch vector j of a traceless 2x2 Hermitian J = (1/2) j.sigma."""
    return np.array([2 * J[0, 1].real, -2 * J[0, 1].imag, (J[0, 0] - J[1, 1]).real])


def test_noalloc_moments_match_handle_moments(xf):
    import torch

    wl = Workload(name="na", n_energy=37, n_angle=29)
    g = Grid.from_workload(wl)
    s = make_solver(xf, wl, fixed_dr_km=0.1)
    r = 40.0
    s.set_rho(beams(random_state(wl, seed=23)), r)
    J0, J1 = s.moments()
    ref = np.concatenate([bloch(J0), bloch(J1)])

    dev = torch.device("cuda")
    nb = wl.n_beams
    state = torch.empty((3, nb), dtype=torch.float64, device=dev)
    s.get_rho(xf.LAYOUT_NATIVE, device_ptr=state.data_ptr())
    N = g.N
    wts = torch.tensor(np.stack([N[0, 0] - N[0, 1], -(N[1, 0] - N[1, 1])]), dtype=torch.float64, device=dev)
    u = torch.tensor(g.u, dtype=torch.float64, device=dev)
    du = torch.tensor(g.du, dtype=torch.float64, device=dev)
    out = torch.full((6,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731

    for call in range(2):
        out.fill_(float("nan"))
        rc = xf.xflat_moments_2f_noalloc(P(state), wl.n_energy, wl.n_angle, P(wts), P(u), P(du),
                                         wl.R_km, r, P(out), ctypes.c_void_p(stream))
        assert rc == xf.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (call, got, ref)

    # more angle bins than the scratch array holds: rejected, nothing launched
    rc = xf.xflat_moments_2f_noalloc(P(state), 1, xf.NOALLOC_MAX_ANGLES + 1, P(wts), P(u), P(du),
                                     wl.R_km, r, P(out), ctypes.c_void_p(stream))
    assert rc == xf.ERR_INVAL
