"""Plain-data description of an open bosonic problem (paper Eqs. 1-3, S1-S2).

A problem is a set of bosonic modes, each truncated at ``N[j]`` Fock levels; a
Hamiltonian written as a sum of normal-ordered monomials ``h * prod_j (a_j^dag)^u_j a_j^v_j``
(Eq. 1 / Eq. S1), optionally multiplied by a time-dependent envelope (a *channel*);
Lindblad jump operators ``L_n = sum_t c_t * monomial_t`` with rate ``kappa_n`` (Eq. 3);
the measured operator A(0) given by its number-basis matrix elements; and the initial
density matrix rho0 used for expectation values.

Channel kinds and their parameter tuples (time in ns, frequencies in rad/ns):
  * ``const``: ``(re, im)``                         -> constant complex value
  * ``gauss``: ``(amp_re, amp_im, t0, sigma)``      -> amp * exp(-(t-t0)^2 / (2 sigma^2))
  * ``pwc``:   ``(t_start, seg_len, re_0, im_0, re_1, im_1, ...)`` -> piecewise-constant
    complex value, segment s covering [t_start + s*seg_len, t_start + (s+1)*seg_len)
  * ``cexp``:  ``(amp_re, amp_im, omega)``          -> amp * exp(i omega t)

An H term with ``conj=True`` multiplies its coefficient by the complex conjugate of its
channel's value (so ``eps(t) a^dag + eps(t)^* a`` is two terms on one channel).  An H term
with ``param >= 0`` has coefficient ``coef * params[param]``; these real parameters, and
the segment values of ``pwc`` channels, are what gradients are taken with respect to.

A *secular damping* entry is the paper's proper (secular) dissipator of one anharmonic mode
(Eq. 203 / Eq. S9): rate ``kappa`` and, per transition n <-> n+1, the thermal occupation
``nbar[n]`` (Eq. S10: the bath occupation at the transition frequency omega + 2 eta n;
entries beyond the tuple are 0, an empty tuple is the zero-temperature case).

Only data lives here; the envelopes are evaluated separately by each consumer.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

Index = Tuple[int, ...]

CHANNEL_KINDS = ("const", "gauss", "pwc", "cexp")


@dataclass(frozen=True)
class Channel:
    kind: str
    params: Tuple[float, ...]

    def __post_init__(self):
        if self.kind not in CHANNEL_KINDS:
            raise ValueError(f"unknown channel kind {self.kind!r}")


@dataclass(frozen=True)
class HTerm:
    coef: complex
    u: Index  # powers of a_j^dag, one per mode
    v: Index  # powers of a_j, one per mode
    channel: int = -1  # -1: static
    conj: bool = False
    param: int = -1  # -1: no gradient parameter


@dataclass(frozen=True)
class Jump:
    rate: float
    terms: Tuple[Tuple[complex, Index, Index], ...]  # (c_t, u_t, v_t)


@dataclass(frozen=True)
class SecularDamping:
    mode: int
    kappa: float
    nbar: Tuple[float, ...] = ()

    def nbar_at(self, n: int) -> float:
        return float(self.nbar[n]) if 0 <= n < len(self.nbar) else 0.0


@dataclass
class Problem:
    n_modes: int
    N: Index  # Fock truncation per mode (oracle number basis); mapping grid M defaults to N
    h_terms: List[HTerm]
    jumps: List[Jump]
    measured: Dict[Tuple[Index, Index], complex]  # <k|A(0)|l>
    T: float
    dt: float
    channels: List[Channel] = field(default_factory=list)
    params: List[float] = field(default_factory=list)
    rho0: Optional[Dict[Tuple[Index, Index], complex]] = None  # None: vacuum
    reverse_time: bool = True  # Heisenberg reading: integrate tau in [0, T] with t = T - tau
    name: str = ""
    secular: List[SecularDamping] = field(default_factory=list)

    @property
    def n_steps(self) -> int:
        n = round(self.T / self.dt)
        if abs(n * self.dt - self.T) > 1e-9 * max(1.0, self.T):
            raise ValueError("T must be a whole number of steps")
        return int(n)

    def rho0_items(self):
        if self.rho0 is None:
            z = tuple(0 for _ in range(self.n_modes))
            return {(z, z): 1.0 + 0j}
        return self.rho0
