"""torch.autograd binding of the discrete adjoint (xflat_adjoint): the mean electron-neutrino
survival probability after fixed RK4 steps as a differentiable function of the per-bin number
luminosities and the vacuum mixing angle.

The CUDA library runs the forward integration and its discrete adjoint in one call, so the forward
of this Function already holds the gradient; backward only scales it by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import xflat


class MeanSurvival(torch.autograd.Function):
    """J = Pbar_ee(r1) of xflat_pee after n_steps RK4 steps from the initial condition at r0.

    N: float64 tensor [2, 2, n_energy] of per-bin number luminosities (nu / nubar, e / x);
    theta: 0-dim float64 tensor, theta_v in rad; cfg: an xflat_config (two flavours) supplying
    every other input (sizes, dm2, R, matter, launch shape).
    """

    @staticmethod
    def forward(ctx, N, theta, cfg, r0, r1, n_steps, checkpoint_every):
        c = xflat.xflat_config.from_buffer_copy(cfg)
        c.theta[0] = float(theta)
        s = xflat.Solver(c)
        try:
            s.set_spectra(N.detach().to("cpu", torch.float64).numpy())
            J, dN, dth = s.adjoint(r0, r1, n_steps, checkpoint_every)
        finally:
            s.close()
        ctx.save_for_backward(torch.as_tensor(dN, dtype=N.dtype, device=N.device),
                              torch.tensor(dth, dtype=theta.dtype, device=theta.device))
        return torch.tensor(J, dtype=N.dtype, device=N.device)

    @staticmethod
    def backward(ctx, gJ):
        dN, dth = ctx.saved_tensors
        return gJ * dN, gJ * dth, None, None, None, None, None


def mean_survival(N, theta, cfg, r0, r1, n_steps, checkpoint_every=64):
    return MeanSurvival.apply(N, theta, cfg, r0, r1, n_steps, checkpoint_every)


def spectra_from_parameters(L, w, base):
    """Per-bin number luminosities from the workload's parameters, as torch operations (so that
    autograd carries gradients to them): L = (L_nue, L_nuebar, L_nux) (tensor of 3, the unit of
    `base`), w = per-energy-bin multiplicative weights of the nu_e spectrum (tensor of n_energy),
    base[s][f][k] = the per-bin number luminosity of a unit luminosity of species s (nu, nubar)
    and flavour f (e, x).  N[0][0] = L_nue w base[0][0], N[1][0] = L_nuebar base[1][0],
    N[s][1] = L_nux base[s][1] (the x flavours share one luminosity)."""
    return torch.stack([torch.stack([L[0] * w * base[0, 0], L[2] * base[0, 1]]),
                        torch.stack([L[1] * base[1, 0], L[2] * base[1, 1]])])


def mean_survival_from_parameters(L, w, theta, base, cfg, r0, r1, n_steps, checkpoint_every=64):
    """J = Pbar_ee(r1) as a differentiable function of the three luminosities, the n_energy nu_e
    spectral weights and theta_v (see spectra_from_parameters and MeanSurvival)."""
    return MeanSurvival.apply(spectra_from_parameters(L, w, base), theta, cfg, r0, r1, n_steps,
                              checkpoint_every)
