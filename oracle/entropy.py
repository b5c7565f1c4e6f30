"""O4 -- entropy production rate of the anharmonic oscillator under the conventional
(Eq. 201) and the secular (Eq. 203 / Eq. S9) master equations (test infrastructure,
a validation workload of the dissipators; see the oracle package header).

What it computes (units hbar = k_B = 1, frequencies in rad/ns, kT = k_B T_E / hbar):
    Pi(t) = dS/dt - (1/T_E) dE/dt
          = -Tr[rho' ln rho] - Tr[rho'] - Tr[H rho'] / T_E
(the supplement's entropy-production section, its Eqs. 202-203)
with rho' the Schroedinger-picture generator of O1 applied to rho, H = omega a^dag a +
eta (a^dag)^2 a^2, and the initial state rho(0) = (1 - e^-c) sum_n e^(-c n) |n><n|.

Parity status (tests/test_oracle_entropy.py): pinned by the closed form of the supplement's
Eq. 204 for the conventional equation, T_E Pi(0) / kappa = (N_0 - nbar) [omega (1 - T_E / T_0)
+ 4 eta N_0] with N_0 = 1/(e^c - 1), T_0 = omega / c (sign and value); by the low-temperature
form of the supplement's Eq. 210, T_0 T_E Pi(0) / (kappa omega) ~ (T_E - T_0)(e^(-omega/T_E)
- e^(-omega/T_0)), for the secular equation; and by Pi >= 0 for the secular equation, whose stationary state is the
Gibbs state of H (detailed balance at the transition frequencies omega + 2 eta n).
"""

from __future__ import annotations

import math

import numpy as np

from workloads.spec import HTerm, Problem, SecularDamping
from .fock import FockModel


def oscillator(N: int, omega: float, eta: float, kappa: float, kT: float, secular: bool) -> Problem:
    """The anharmonic oscillator of Eq. 201 with the conventional dissipator (jumps
    sqrt(kappa (nbar+1)) a and sqrt(kappa nbar) a^dag, nbar at omega) or the secular one
    (nbar_n at omega + 2 eta n, Eq. S10), truncated at N levels."""
    h = [HTerm(omega + 0j, (1,), (1,)), HTerm(eta + 0j, (2,), (2,))]
    nb = (lambda w: 1.0 / math.expm1(w / kT)) if kT > 0 else (lambda w: 0.0)
    if secular:
        sec = [SecularDamping(0, kappa, tuple(nb(omega + 2.0 * eta * n) for n in range(N - 1)))]
        jumps = []
    else:
        from workloads.spec import Jump
        n0 = nb(omega)
        jumps = [Jump(kappa * (n0 + 1.0), ((1.0 + 0j, (0,), (1,)),))]
        if n0 > 0:
            jumps.append(Jump(kappa * n0, ((1.0 + 0j, (1,), (0,)),)))
        sec = []
    return Problem(n_modes=1, N=(N,), h_terms=h, jumps=jumps, secular=sec, measured={((0,), (0,)): 1.0},
                   T=1.0, dt=1.0)


def gaussian_state(N: int, c: float) -> np.ndarray:
    """rho(0) = (1 - e^-c) sum_n e^(-c n) |n><n| truncated at N levels (renormalised)."""
    p = np.exp(-c * np.arange(N))
    return np.diag(p / p.sum()).astype(np.complex128)


def entropy_production(problem: Problem, rho: np.ndarray, kT: float) -> float:
    """Pi = -Tr[rho' ln rho] - Tr[rho'] - Tr[H rho'] / kT for the problem's generator."""
    model = FockModel(problem)
    H = model.h_static
    drho = model.schrodinger_generator(rho, H)
    w, V = np.linalg.eigh(rho)
    ln_rho = (V * np.log(np.maximum(w, 1e-300))) @ V.conj().T
    return float(np.real(-np.trace(drho @ ln_rho) - np.trace(drho) - np.trace(H @ drho) / kT))
