"""Plain FP64 CPU oracle for the mapped adjoint-Lindblad method (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the library
(``paper_2203_05526_gb300``) never does, and it shares no code with it.

Modules
-------
* ``channels``  drive envelopes (own evaluation of the ``workloads.spec`` channel kinds).
* ``fock``      O1: the adjoint master equation (Eq. 3) on dense truncated number-basis
                matrices, classical RK4; plus the forward Schroedinger-picture density-matrix
                RK4, the dense Liouvillian and closed forms used to pin it.
* ``mapping``   O2: the paper's mapping step by step: normal-ordered coefficients f
                (Eq. 2), transform to g (Eq. 6), separable initial conditions (Eqs. 10, 13),
                separation constant (Eq. 304), the coupled system for G_x, G_y, R
                (Eqs. 9a-c / 303a-c) with x, d/dx, y, d/dy represented as matrices on the
                monomial basis, classical RK4, reconstruction (Eq. 11).
* ``grad``      O3: reverse-mode (discrete adjoint) gradients of the RK4 trajectory of
                O2, and central finite differences.
* ``entropy``   O4: entropy production rate of the anharmonic oscillator under the
                conventional and the secular master equations (the supplement's
                entropy-production section), a validation workload of the two dissipators.

O1 and O2 also carry the secular dissipator (Eq. 203 / Eq. S9), O2 the diagonal residual
layout and SVD initial conditions.

Parity status of every function is listed in each module's header.
"""
