"""Discrete adjoint of fixed-step RK4 on the bulb model's matrix equation (test infrastructure only).

Objective: the number-flux weighted electron-neutrino survival probability at the end of the
range (the quantity of the Sec. 3.4 validation figure, averaged over nu beams),
    J = sum_{j,k} du_j N_e,k P_ee(nu, j, k) / sum_{j,k} du_j N_e,k.
Parameters: the per-bin number luminosities N[species, flavour, k] that build the flux matrices
of Sec. 2, and the vacuum mixing angle theta_v of the two-flavour H_vac (Sec. 2).

"Discrete adjoint" means the exact gradient of the discrete map the forward integrator computes
(classical RK4 on dY/dr = -i [H(Y), Y] / cos theta, Eq. eom, with H depending on every beam
through the flux moments of Eq. F and Eq. Hnu), obtained by running the chain rule backwards
through the steps and stages; it is not a discretisation of the continuous adjoint equation.

Conventions.  A complex array Z is differentiated as the pair (Re Z, Im Z): its adjoint is
G = dJ/dRe Z + i dJ/dIm Z, so that dJ = Re sum conj(G) dZ.  For a product Z = A B of complex
matrices this gives G_A = G_Z B^dagger and G_B = A^dagger G_Z; for Z = conj(A), G_A = conj(G_Z).
Two flavours only (the flux matrix then needs N_e and N_x per species).
"""
from __future__ import annotations

import numpy as np

from .physics import Bulb, matter_strength, HBARC_EV_KM


def _dag(A):
    return np.conj(np.swapaxes(A, -1, -2))


def _re_inner(G, A):
    """Re sum conj(G) A over the two matrix axes."""
    return (np.conj(G) * A).real.sum(axis=(-2, -1))


def forward_pieces(bulb: Bulb, r: float, Y: np.ndarray):
    """Intermediate quantities of bulb.rhs(r, Y) that its adjoint needs."""
    P, Pb = Y[0], Y[1]
    H, Hb = bulb.hamiltonians(r, P, Pb)
    c = bulb.cos_theta(r)
    return P, Pb, H, Hb, c


def rhs_vjp(bulb: Bulb, r: float, Y: np.ndarray, V: np.ndarray):
    """Adjoint of Y -> bulb.rhs(r, Y) with cotangent V (same shape as Y).

    Returns (G_Y, G_N [2, 2, N_E], G_theta): the contribution of this evaluation to the adjoint of
    the state, of the number luminosities and of the mixing angle.
    """
    assert bulb.n == 2 and bulb.geometry == "bulb"
    P, Pb, H, Hb, c = forward_pieces(bulb, r, Y)
    VP, VPb = V[0], V[1]
    ic = (1j / c)[:, None, None, None]                       # i / cos per angle bin
    # dP = -i (H P - P H) / c  and  dPb = -i (Hb Pb - Pb Hb) / c
    GP = ic * (_dag(H) @ VP - VP @ _dag(H))
    GPb = ic * (_dag(Hb) @ VPb - VPb @ _dag(Hb))
    GH = ic * (VP @ _dag(P) - _dag(P) @ VP)
    GHb = ic * (VPb @ _dag(Pb) - _dag(Pb) @ VPb)
    # H = Hvac_k + lambda Pe + Hnn_j ;  Hb = Hvac_k - lambda Pe - conj(Hnn_j)
    GHvac = GH.sum(axis=0) + GHb.sum(axis=0)                 # [N_E, 2, 2]
    GHnn = GH.sum(axis=1) - np.conj(GHb.sum(axis=1))         # [N_u, 2, 2]
    # Hnn_j = K (Phi1 - c_j Phic),  Phi1 = sum_j w_j Fsum_j,  Phic = sum_j w_j c_j Fsum_j
    R = bulb.wl.R_km
    w = bulb.grid.du * R * R / (2.0 * r * r * c)
    GPhi1 = bulb.K * GHnn.sum(axis=0)
    GPhic = -bulb.K * np.einsum("j,jab->ab", c, GHnn)
    GFsum = w[:, None, None] * GPhi1[None] + (w * c)[:, None, None] * GPhic[None]   # [N_u, 2, 2]
    GF = np.broadcast_to(GFsum[:, None], P.shape)            # Fsum_j = sum_k F_jk
    # F = Ne P + Nx (I - P) - conj(Nbe Pb + Nbx (I - Pb))
    N = bulb.grid.N
    Ne, Nx, Nbe, Nbx = N[0, 0], N[0, 1], N[1, 0], N[1, 1]
    GP = GP + (Ne - Nx)[None, :, None, None] * GF
    GPb = GPb - (Nbe - Nbx)[None, :, None, None] * np.conj(GF)
    I = np.eye(2)
    GN = np.zeros((2, 2, len(Ne)))
    GN[0, 0] = _re_inner(GF, P).sum(axis=0)
    GN[0, 1] = _re_inner(GF, I - P).sum(axis=0)
    GN[1, 0] = -_re_inner(GF, np.conj(Pb)).sum(axis=0)
    GN[1, 1] = -_re_inner(GF, np.conj(I - Pb)).sum(axis=0)
    # H_vac(E_k) = dm2 / (4 E_k) M(theta),  M = [[-cos 2th, sin 2th], [sin 2th, cos 2th]]
    th = bulb.wl.theta[0]
    dM = 2.0 * np.array([[np.sin(2 * th), np.cos(2 * th)], [np.cos(2 * th), -np.sin(2 * th)]])
    scale = bulb.wl.dm2[0] / (4.0 * bulb.grid.E * 1e6 * HBARC_EV_KM)    # [N_E], 1/km
    Gth = float((scale * _re_inner(GHvac, dM[None].astype(np.complex128))).sum())
    return np.stack([GP, GPb]), GN, Gth


def objective(bulb: Bulb, Y: np.ndarray) -> float:
    return bulb.mean_survival(Y)


def objective_grad(bulb: Bulb, Y: np.ndarray):
    """(G_Y, explicit G_N) of the objective at the final state."""
    g = bulb.grid
    W = g.du[:, None] * g.N[0, 0][None, :]                   # [N_u, N_E]
    S = W.sum()
    Pee = Y[0, ..., 0, 0].real
    J = float((W * Pee).sum() / S)
    GY = np.zeros_like(Y)
    GY[0, ..., 0, 0] = W / S
    GN = np.zeros((2, 2, len(g.E)))
    GN[0, 0] = (g.du[:, None] * (Pee - J)).sum(axis=0) / S
    return J, GY, GN


def rk4_adjoint(bulb: Bulb, Y0: np.ndarray, r0: float, r1: float, n_steps: int):
    """J and its gradients for n_steps classical RK4 steps from (r0, Y0) to r1.

    Stores every step's state, then runs each step's stages backwards: for
    y' = y + h (k1 + 2 k2 + 2 k3 + k4) / 6 with k1 = f(r, y), k2 = f(r + h/2, y + h/2 k1),
    k3 = f(r + h/2, y + h/2 k2), k4 = f(r + h, y + h k3), the adjoint a' of y' gives
        Gk4 = h/6 a', Gk3 = h/3 a' + h f4^T Gk4, Gk2 = h/3 a' + h/2 f3^T Gk3,
        Gk1 = h/6 a' + h/2 f2^T Gk2,  a = a' + f4^T Gk4 + f3^T Gk3 + f2^T Gk2 + f1^T Gk1,
    with fi^T the adjoint of the right-hand side at stage i.  Returns (J, dJ/dN, dJ/dtheta_v).
    """
    h = (r1 - r0) / n_steps
    f = bulb.rhs
    Ys = [Y0.copy()]
    for n in range(n_steps):
        r = r0 + n * h
        y = Ys[-1]
        k1 = f(r, y)
        k2 = f(r + 0.5 * h, y + (0.5 * h) * k1)
        k3 = f(r + 0.5 * h, y + (0.5 * h) * k2)
        k4 = f(r + h, y + h * k3)
        Ys.append(y + h * (k1 / 6 + k2 / 3 + k3 / 3 + k4 / 6))
    J, a, GN = objective_grad(bulb, Ys[-1])
    Gth = 0.0
    for n in range(n_steps - 1, -1, -1):
        r = r0 + n * h
        y = Ys[n]
        k1 = f(r, y)
        y2 = y + (0.5 * h) * k1
        k2 = f(r + 0.5 * h, y2)
        y3 = y + (0.5 * h) * k2
        k3 = f(r + 0.5 * h, y3)
        y4 = y + h * k3
        Gk4 = (h / 6) * a
        g4, n4, t4 = rhs_vjp(bulb, r + h, y4, Gk4)
        Gk3 = (h / 3) * a + h * g4
        g3, n3, t3 = rhs_vjp(bulb, r + 0.5 * h, y3, Gk3)
        Gk2 = (h / 3) * a + (0.5 * h) * g3
        g2, n2, t2 = rhs_vjp(bulb, r + 0.5 * h, y2, Gk2)
        Gk1 = (h / 6) * a + (0.5 * h) * g2
        g1, n1, t1 = rhs_vjp(bulb, r, y, Gk1)
        a = a + g4 + g3 + g2 + g1
        GN = GN + n4 + n3 + n2 + n1
        Gth += t4 + t3 + t2 + t1
    return J, GN, Gth
