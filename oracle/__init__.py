"""Plain FP64 CPU oracle for the bulb-model radial step (arXiv:1912.10596, Sec. 2 and Sec. 3.4).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

The oracle is written from the paper's equations in their own notation: 2x2 (or 3x3) complex
density matrices psi psi^dagger for every beam, the antineutrino equation in the paper's literal
form H_bar = H_vac - H_mat - H_nunu^* (Eq. eom), the flux matrices F_alpha and the nu-nu potential
of Eq. Hnu, and the exact 2x2 propagator of Eq. U.  It shares no code with the CUDA library
(which works on Bloch vectors in a conjugated antineutrino convention) and imports nothing from it.
Its inputs come from ``bulb_inputs`` only.

Modules
-------
physics    constants, H_vac, H_mat, geometry, F_alpha, H_nunu, the right-hand side
expm       Eq. U (2x2 closed form) and a Hermitian 3x3 exponential by eigendecomposition
integrate  fixed-step RK4, adaptive Dormand-Prince 5(4), commutator-free Lie RK4 (CF4)
four_psi   the paper-literal four-wavefunction state (nu_e, nu_x, nubar_e, nubar_x per beam)
adjoint    discrete adjoint of fixed-step RK4 for the survival-probability objective
extended   the extended bulb model (azimuthal bins, four moments)

Pins (tests/test_oracle_pins.py, test_oracle_adjoint.py, test_oracle_extended.py, each mistake of
tests/test_oracle_mutations.py failing at least one): every function above is held by closed
forms (vacuum and constant-density oscillations in two and three flavours, the synchronised
collective precession), invariants (unit Bloch vectors, lepton number, trace and purity),
reductions (three flavours to two, single angle to the radial beam, extended to bulb, the four
wavefunctions to two states), hand-computed moments and textbook matter strengths, integrator
orders and exactness for constant generators, and finite differences for the adjoint.  The full
multi-angle nonlinear result of a bulb run is pinned only through those parts: the paper prints no
number for it, so beyond them its parity is unpinned.
"""
