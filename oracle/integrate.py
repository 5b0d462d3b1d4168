"""Radial integrators for dY/dr = f(r, Y) on the matrix state (test infrastructure only).

The paper evolves the wavefunctions with the exact propagator of Eq. U and a modified mid-point
scheme with adaptive step control taken from an earlier reference that is not reproduced in the
text (Sec. 3.4).  The oracle provides the schemes the workloads name, on the paper's equation of
motion:

* ``rk4_step``   classical fourth-order Runge-Kutta on the commutator form dY/dr = -i[H,Y]/cos th;
* ``dp45_step``  the Dormand-Prince 5(4) pair (first-same-as-last, embedded fourth-order error);
* ``cf4_step``   a commutator-free Lie-group Runge-Kutta method of order four (Celledoni,
                 Marthinsen & Owren 2003) whose every update is an exact propagator exp(-i H dl)
                 of Eq. U applied as Y -> U Y U^dagger;
* ``em2_step``   the exponential midpoint rule (the Lie-group method of Runge-Kutta-Munthe-Kaas
                 type with Runge's midpoint tableau; Iserles, Munthe-Kaas, Norsett & Zanna 2000):
                 Y' = exp(-i h G(r + h/2, Y_half)) Y (...)^dagger with Y_half from an exponential
                 half step; its embedded first-order partner, the exponential Euler step with
                 G(r, Y), gives the error estimate (a 2(1) pair, controller exponent 1/2).  Every
                 update is an exact propagator of Eq. U, in the spirit of the paper's exponential
                 mid-point integration;
* ``lie_richardson_step``  the commutator-free Lie RK4 step above with adaptive control by
                 Richardson extrapolation (step doubling, Hairer, Norsett & Wanner I, Sec. II.4):
                 one step of size h and two of size h/2 from the same state; the two half steps are
                 kept and (Y_two - Y_full) / (2^4 - 1) estimates their local error.  Every update is
                 an exact propagator of Eq. U, and no exponent needs to be small: the error is set
                 by how fast the generator changes, not by its size;
* ``evolve_fixed`` / ``evolve_adaptive`` / ``evolve_em2`` / ``evolve_lie_adaptive`` drive them.

Adaptive control (a standard reading; the paper does not spell it out): the error of a step is
Err = max over beams of ||e_b||_F / (atol + rtol * max(||Y~_b||_F, ||Y~'_b||_F)), with Y~ the
traceless part and e_b the embedded error matrix; the step is accepted when Err <= 1 and the next
step is h * min(5, max(0.2, 0.9 Err^(-1/5))) (never above 1 after a rejection), clipped to h_max and
to the end of the range.  Fixed steps sit at r_n = r0 + n h with h = (r1 - r0) / n_steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .expm import propagator, conjugate_by

# Dormand-Prince 5(4) coefficients
DP_C = np.array([0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0])
DP_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
    [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84],
]
DP_B = np.array([35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0])
DP_BHAT = np.array([5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40])
DP_E = DP_B - DP_BHAT


def traceless_norm(Y: np.ndarray) -> np.ndarray:
    """Frobenius norm of the traceless part of every matrix in a stack."""
    n = Y.shape[-1]
    tr = np.trace(Y, axis1=-2, axis2=-1)
    T = Y - (tr / n)[..., None, None] * np.eye(n)
    return np.sqrt((np.abs(T) ** 2).sum(axis=(-2, -1)))


def frob(Y: np.ndarray) -> np.ndarray:
    return np.sqrt((np.abs(Y) ** 2).sum(axis=(-2, -1)))


@dataclass
class Stats:
    accepted: int = 0
    rejected: int = 0
    stage_evals: int = 0
    h_last: float = 0.0
    steps: list = field(default_factory=list)     # (r, h, accepted) per attempted step


def rk4_step(f, r, Y, h):
    k1 = f(r, Y)
    k2 = f(r + 0.5 * h, Y + (0.5 * h) * k1)
    k3 = f(r + 0.5 * h, Y + (0.5 * h) * k2)
    k4 = f(r + h, Y + h * k3)
    return Y + h * (k1 / 6 + k2 / 3 + k3 / 3 + k4 / 6)


def dp45_step(f, r, Y, h, k1, atol, rtol):
    """One Dormand-Prince attempt from (r, Y) with k1 = f(r, Y); returns (Y5, Err, k7)."""
    ks = [k1]
    for i in range(1, 7):
        Yi = Y.copy()
        for j, a in enumerate(DP_A[i]):
            if a != 0.0:
                Yi = Yi + (h * a) * ks[j]
        ks.append(f(r + DP_C[i] * h, Yi))
    Y5 = Y.copy()
    for j in range(6):
        if DP_B[j] != 0.0:
            Y5 = Y5 + (h * DP_B[j]) * ks[j]
    e = np.zeros_like(Y)
    for j in range(7):
        if DP_E[j] != 0.0:
            e = e + (h * DP_E[j]) * ks[j]
    scale = atol + rtol * np.maximum(traceless_norm(Y), traceless_norm(Y5))
    err = float((frob(e) / scale).max()) if e.size else 0.0
    return Y5, err, ks[6]


def cf4_step(G, r, Y, h, G1=None):
    """Commutator-free Lie RK4: G(r, Y) returns per-beam generators (H / cos th) so dY/dr = -i[G, Y].
    G1 = G(r, Y) if already known."""
    def E(X, Z):
        return conjugate_by(propagator(X), Z)

    if G1 is None:
        G1 = G(r, Y)
    Y2 = E(0.5 * h * G1, Y)
    G2 = G(r + 0.5 * h, Y2)
    Y3 = E(0.5 * h * G2, Y)
    G3 = G(r + 0.5 * h, Y3)
    Y4 = E(h * G3 - 0.5 * h * G1, Y2)
    G4 = G(r + h, Y4)
    first = E(h * (G1 / 4 + G2 / 6 + G3 / 6 - G4 / 12), Y)
    return E(h * (-G1 / 12 + G2 / 6 + G3 / 6 + G4 / 4), first)


RICHARDSON_DIV = 15.0   # 2^p - 1 for the order p = 4 of the commutator-free Lie RK4


def lie_richardson_step(G, r, Y, h, G1=None):
    """Commutator-free Lie RK4 from (r, Y): one step of size h and two successive steps of size h/2.
    Returns (Y_two, Y_full); the first half step and the full step share G1 = G(r, Y)."""
    if G1 is None:
        G1 = G(r, Y)
    full = cf4_step(G, r, Y, h, G1)
    half = cf4_step(G, r, Y, 0.5 * h, G1)
    two = cf4_step(G, r + 0.5 * h, half, 0.5 * h)
    return two, full


def lie_richardson_error(two, full):
    """Richardson estimate of the local error of the two half steps: (Y_two - Y_full) / (2^p - 1)
    with p = 4 (it is the error's negative: the full step's own error is 2^p times larger)."""
    return (two - full) / RICHARDSON_DIV


def evolve_lie_adaptive(bulb, Y0, r0, r1, rtol, atol, h0, h_min=1e-14, h_max=np.inf, max_steps=10**7,
                        max_attempts=None):
    """Adaptive commutator-free Lie RK4 with Richardson error control: the step keeps Y_two (two
    half steps) when Err = max_b ||Y_two - Y_full||_F / 15 / (atol + rtol max(||Y~_b||_F,
    ||Y~'_b||_F)) <= 1, and the next step is h min(5, max(0.2, 0.9 Err^(-1/5))) (never above 1
    after a rejection), clipped to h_max and to the end of the range.  Every attempt evaluates the
    generators 11 times: 3 more stages of the full step, 3 of the first half step, 4 of the second
    (its first at the half-step state), and once at the new state (the next step's first stage)."""
    G = bulb.generators
    Y = Y0.copy()
    r = r0
    h = min(h0, h_max)
    G1 = G(r, Y)
    st = Stats(stage_evals=1)
    while r < r1:
        last = r + h >= r1
        if last:
            h = r1 - r
        two, full = lie_richardson_step(G, r, Y, h, G1)
        scale = atol + rtol * np.maximum(traceless_norm(Y), traceless_norm(two))
        err = float((frob(lie_richardson_error(two, full)) / scale).max()) if Y.size else 0.0
        st.stage_evals += 11
        ok = err <= 1.0
        st.steps.append((r, h, ok))
        if ok:
            r = r1 if last else r + h
            Y = two
            G1 = G(r, Y)
            st.accepted += 1
            fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** -0.2))
        else:
            st.rejected += 1
            fac = max(0.2, 0.9 * err ** -0.2)
        st.h_last = h
        h = min(h * fac, h_max)
        if r < r1 and h < h_min:
            raise FloatingPointError(f"step size underflow at r={r}: h={h}")
        if st.accepted + st.rejected > max_steps:
            raise RuntimeError("too many steps")
        if max_attempts is not None and st.accepted + st.rejected >= max_attempts:
            break
    return Y, r, st


def em2_step(G, r, Y, h, G1=None):
    """Exponential midpoint step and its exponential-Euler partner from (r, Y) with generators
    G(r, Y) (H / cos theta per beam); G1 = G(r, Y) if already known.  Returns (Y_new, Y_euler)."""
    if G1 is None:
        G1 = G(r, Y)
    Yh = conjugate_by(propagator(0.5 * h * G1), Y)
    G2 = G(r + 0.5 * h, Yh)
    return conjugate_by(propagator(h * G2), Y), conjugate_by(propagator(h * G1), Y)


def evolve_em2(bulb, Y0, r0, r1, rtol, atol, h0, h_min=1e-14, h_max=np.inf, max_steps=10**7,
               fixed_steps=None):
    """Exponential midpoint rule: with fixed_steps, that many equal steps; otherwise adaptive with
    Err = max_b ||Y_new - Y_euler||_F / (atol + rtol max(||Y~_b||_F, ||Y~'_b||_F)), accepted when
    Err <= 1, next step h min(5, max(0.2, 0.9 Err^(-1/2))) (never above 1 after a rejection)."""
    G = bulb.generators
    Y = Y0.copy()
    st = Stats()
    if fixed_steps is not None:
        h = (r1 - r0) / fixed_steps
        for n in range(fixed_steps):
            Y, _ = em2_step(G, r0 + n * h, Y, h)
            st.stage_evals += 2
            st.accepted += 1
        st.h_last = h
        return Y, r1, st
    r = r0
    h = min(h0, h_max)
    G1 = G(r, Y)
    st.stage_evals = 1
    while r < r1:
        last = r + h >= r1
        if last:
            h = r1 - r
        Yn, Ye = em2_step(G, r, Y, h, G1)
        e = Yn - Ye
        scale = atol + rtol * np.maximum(traceless_norm(Y), traceless_norm(Yn))
        err = float((frob(e) / scale).max()) if e.size else 0.0
        st.stage_evals += 2
        ok = err <= 1.0
        st.steps.append((r, h, ok))
        if ok:
            r = r1 if last else r + h
            Y = Yn
            G1 = G(r, Y)
            st.accepted += 1
            fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** -0.5))
        else:
            st.rejected += 1
            fac = max(0.2, 0.9 * err ** -0.5)
        st.h_last = h
        h = min(h * fac, h_max)
        if r < r1 and h < h_min:
            raise FloatingPointError(f"step size underflow at r={r}: h={h}")
        if st.accepted + st.rejected > max_steps:
            raise RuntimeError("too many steps")
    return Y, r, st


def evolve_fixed(bulb, Y0, r0, r1, n_steps, method="rk4", callback=None):
    """n_steps equal steps from r0 to r1 with RK4 or CF4; callback(n, r, Y) after each step."""
    h = (r1 - r0) / n_steps
    Y = Y0.copy()
    st = Stats()
    for n in range(n_steps):
        r = r0 + n * h
        if method == "rk4":
            Y = rk4_step(bulb.rhs, r, Y, h)
        elif method == "lie_rk4":
            Y = cf4_step(bulb.generators, r, Y, h)
        else:
            raise ValueError(method)
        st.stage_evals += 4
        st.accepted += 1
        if callback is not None:
            callback(n + 1, r0 + (n + 1) * h, Y)
    st.h_last = h
    return Y, st


def evolve_adaptive(bulb, Y0, r0, r1, rtol, atol, h0, h_min=1e-14, h_max=np.inf, max_steps=10**7,
                    max_attempts=None):
    """Adaptive Dormand-Prince 5(4) with the controller in the module docstring.  With
    max_attempts, stop after that many attempted steps (accepted or rejected) short of r1."""
    f = bulb.rhs
    Y = Y0.copy()
    r = r0
    h = min(h0, h_max)
    k1 = f(r, Y)
    st = Stats(stage_evals=1)
    while r < r1:
        last = r + h >= r1
        if last:
            h = r1 - r
        Y5, err, k7 = dp45_step(f, r, Y, h, k1, atol, rtol)
        st.stage_evals += 6
        ok = err <= 1.0
        st.steps.append((r, h, ok))
        if ok:
            r = r1 if last else r + h
            Y, k1 = Y5, k7
            st.accepted += 1
            fac = 5.0 if err == 0.0 else min(5.0, max(0.2, 0.9 * err ** -0.2))
        else:
            st.rejected += 1
            fac = max(0.2, 0.9 * err ** -0.2)
        st.h_last = h
        h = min(h * fac, h_max)
        if r < r1 and h < h_min:
            raise FloatingPointError(f"step size underflow at r={r}: h={h}")
        if st.accepted + st.rejected > max_steps:
            raise RuntimeError("too many steps")
        if max_attempts is not None and st.accepted + st.rejected >= max_attempts:
            break
    return Y, r, st
