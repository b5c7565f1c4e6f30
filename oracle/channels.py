"""Drive envelopes for the oracle (the time-dependent factors of the Hamiltonian, Eq. 301).

Parity: pinned by direct evaluation at hand-picked times in tests/test_oracle_fock.py.

Time convention (a reading of the paper's statement that the Hamiltonian is held
constant during each small step, main text after Eq. 301):
  * smooth envelopes (const, gauss, cexp) are evaluated at each RK4 stage time;
  * piecewise-constant envelopes (pwc) are evaluated at the midpoint of the RK4 step,
    so all four stages of one step see one segment value.
For the Heisenberg-picture integration the physical time of integration time tau is
t = T - tau (``reverse_time``); with ``reverse_time=False`` it is t = tau (the paper's
literal substitution of the Schroedinger Hamiltonian).
"""

from __future__ import annotations

import math

from workloads.spec import Channel


def channel_value(ch: Channel, t: float) -> complex:
    p = ch.params
    if ch.kind == "const":
        return complex(p[0], p[1])
    if ch.kind == "gauss":
        amp = complex(p[0], p[1])
        t0, sigma = p[2], p[3]
        return amp * math.exp(-((t - t0) ** 2) / (2.0 * sigma * sigma))
    if ch.kind == "cexp":
        amp = complex(p[0], p[1])
        return amp * complex(math.cos(p[2] * t), math.sin(p[2] * t))
    if ch.kind == "pwc":
        t_start, seg_len = p[0], p[1]
        n_seg = (len(p) - 2) // 2
        s = int(math.floor((t - t_start) / seg_len))
        if s < 0 or s >= n_seg:
            return 0j
        return complex(p[2 + 2 * s], p[3 + 2 * s])
    raise ValueError(ch.kind)


def physical_time(tau: float, T: float, reverse: bool) -> float:
    return T - tau if reverse else tau


def stage_value(ch: Channel, tau_step: float, c: float, dt: float, T: float, reverse: bool) -> complex:
    """Envelope value seen by the RK4 stage at tau_step + c*dt."""
    if ch.kind == "pwc":
        return channel_value(ch, physical_time(tau_step + 0.5 * dt, T, reverse))
    return channel_value(ch, physical_time(tau_step + c * dt, T, reverse))
