"""Seeded synthetic workloads shaped like the paper's test system (Eq. 301 network of
driven, damped Kerr oscillators; conventional dissipator Eq. 201 with jump operators
sqrt(kappa (1+n_th)) a and sqrt(kappa n_th) a^dag).

Units: time in ns, angular frequencies in rad/ns.  Every builder returns
``workloads.spec.Problem`` objects; nothing here evaluates the method.

Workloads
---------
* ``kerr_static``   single damped Kerr oscillator, Delta=0, K=-2pi*0.2, gamma=1e-3,
                    zero temperature, A(0)=|1><1|, T=100, dt=0.01, N=16.
* ``kerr_driven``   same oscillator at n_th=0.05 with a resonant Gaussian drive
                    eps(t)(a+a^dag), peak 2pi*0.05, sigma=10 ns, centre T/2; N=40,
                    dt=0.0025 (the RK4 imaginary-axis bound |K|/2 N(N-1) dt <= 2 sqrt 2).
* ``two_mode``      two exchange-coupled Kerr modes, Delta=(0, 2pi*0.1), K=-2pi*0.2,
                    g=2pi*0.005, gamma=1e-4 each, A(0)=|1,0><1,0|, N=12 per mode,
                    T=100, dt=0.01.
* ``kerr_batch``    B driven damped Kerr instances (B=4096 by default), seed 20220311,
                    parameters drawn in the order Delta, K, log10 gamma, drive peak,
                    measured level n, truncation N; dt=0.002, T=100.
* ``two_mode_control``  the two-mode system with a piecewise-constant complex drive
                    on mode 1 over 64 segments (seed 5526, amplitudes ~ N(0,(2pi*0.01)^2)
                    for real and imaginary parts), T=200, dt=200/64/320.
"""

from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from .spec import Channel, HTerm, Jump, Problem, SecularDamping

TWO_PI = 2.0 * math.pi


def _unit(n_modes: int, j: int, p: int) -> tuple:
    return tuple(p if i == j else 0 for i in range(n_modes))


def _zero(n_modes: int) -> tuple:
    return tuple(0 for _ in range(n_modes))


def kerr_mode_terms(n_modes: int, j: int, delta: float, kerr: float,
                    delta_param: int = -1, kerr_param: int = -1) -> List[HTerm]:
    """Delta a^dag a + (K/2) a^dag^2 a^2 on mode j (Eq. 301 with omega=Delta, eta=K/2).

    With a parameter index the coefficient becomes params[idx] * coef, so the stored
    coefficient is the multiplier of the parameter (1 for Delta, 1/2 for K)."""
    out = []
    if delta != 0.0 or delta_param >= 0:
        out.append(HTerm(1.0 + 0j if delta_param >= 0 else complex(delta),
                         _unit(n_modes, j, 1), _unit(n_modes, j, 1), param=delta_param))
    if kerr != 0.0 or kerr_param >= 0:
        out.append(HTerm(0.5 + 0j if kerr_param >= 0 else complex(kerr / 2.0),
                         _unit(n_modes, j, 2), _unit(n_modes, j, 2), param=kerr_param))
    return out


def damping_jumps(n_modes: int, j: int, gamma: float, n_th: float) -> List[Jump]:
    """Conventional dissipator (Eq. 201): sqrt(gamma(1+n_th)) a and sqrt(gamma n_th) a^dag."""
    z = _zero(n_modes)
    a = _unit(n_modes, j, 1)
    out = [Jump(gamma * (1.0 + n_th), ((1.0 + 0j, z, a),))]
    if n_th > 0.0:
        out.append(Jump(gamma * n_th, ((1.0 + 0j, a, z),)))
    return out


def projector(n_modes: int, n: Sequence[int]):
    n = tuple(int(x) for x in n)
    assert len(n) == n_modes
    return {(n, n): 1.0 + 0j}


def kerr_static(N: int = 16) -> Problem:
    return Problem(
        n_modes=1, N=(N,),
        h_terms=kerr_mode_terms(1, 0, 0.0, -TWO_PI * 0.2),
        jumps=damping_jumps(1, 0, 1e-3, 0.0),
        measured=projector(1, (1,)),
        T=100.0, dt=0.01, name="kerr_static")


def gauss_drive_terms(n_modes: int, j: int, ch: int) -> List[HTerm]:
    """eps(t) a^dag + eps(t)^* a on mode j; for a real envelope this is eps(t)(a + a^dag)."""
    z = _zero(n_modes)
    a = _unit(n_modes, j, 1)
    return [HTerm(1.0 + 0j, a, z, channel=ch, conj=False),
            HTerm(1.0 + 0j, z, a, channel=ch, conj=True)]


def kerr_driven(N: int = 40, dt: float = 0.0025, T: float = 100.0,
                n_th: float = 0.05, peak: float = TWO_PI * 0.05, sigma: float = 10.0) -> Problem:
    ch = [Channel("gauss", (peak, 0.0, T / 2.0, sigma))]
    return Problem(
        n_modes=1, N=(N,),
        h_terms=kerr_mode_terms(1, 0, 0.0, -TWO_PI * 0.2) + gauss_drive_terms(1, 0, 0),
        jumps=damping_jumps(1, 0, 1e-3, n_th),
        measured=projector(1, (1,)),
        channels=ch, T=T, dt=dt, name="kerr_driven")


def two_mode(N: int = 12, T: float = 100.0, dt: float = 0.01, g: float = TWO_PI * 0.005,
             param_ids: bool = False) -> Problem:
    """Two exchange-coupled Kerr modes; with ``param_ids`` K_1, K_2 and g are gradient
    parameters 0, 1, 2."""
    n = 2
    deltas = (0.0, TWO_PI * 0.1)
    kerrs = (-TWO_PI * 0.2, -TWO_PI * 0.2)
    terms: List[HTerm] = []
    params: List[float] = []
    for j in range(n):
        kp = -1
        if param_ids:
            kp = len(params)
            params.append(kerrs[j])
        terms += kerr_mode_terms(n, j, deltas[j], kerrs[j], kerr_param=kp)
    gp = -1
    if param_ids:
        gp = len(params)
        params.append(g)
    cg = 1.0 + 0j if param_ids else complex(g)
    # g (a_1^dag a_2 + a_2^dag a_1)
    terms.append(HTerm(cg, (1, 0), (0, 1), param=gp))
    terms.append(HTerm(cg, (0, 1), (1, 0), param=gp))
    jumps = damping_jumps(n, 0, 1e-4, 0.0) + damping_jumps(n, 1, 1e-4, 0.0)
    return Problem(n_modes=2, N=(N, N), h_terms=terms, jumps=jumps,
                   measured=projector(2, (1, 0)), T=T, dt=dt, params=params,
                   name="two_mode")


def two_mode_control(n_seg: int = 64, T: float = 200.0, steps_per_seg: int = 320,
                     seed: int = 5526, N: int = 12, amp_sigma: float = TWO_PI * 0.01) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.normal(0.0, amp_sigma, size=n_seg)
    im = rng.normal(0.0, amp_sigma, size=n_seg)
    seg_len = T / n_seg
    dt = seg_len / steps_per_seg
    vals = []
    for s in range(n_seg):
        vals += [float(re[s]), float(im[s])]
    p = two_mode(N=N, T=T, dt=dt, param_ids=True)
    p.channels = [Channel("pwc", (0.0, seg_len, *vals))]
    p.h_terms = p.h_terms + gauss_drive_terms(2, 0, 0)
    p.name = "two_mode_control"
    return p


def kerr_batch(B: int = 4096, seed: int = 20220311, T: float = 100.0, dt: float = 0.002,
               n_min: int = 10, n_max: int = 40, sigma: float = 10.0) -> List[Problem]:
    """B independent driven damped Kerr oscillators with seeded parameters.

    Draw order per instance: Delta ~ U(-2pi 0.01, 2pi 0.01); K ~ U(-2pi 0.25, -2pi 0.15);
    log10 gamma ~ U(-4, -3); drive peak ~ U(0, 2pi 0.05); n ~ U{0,1,2}; N ~ U{n_min..n_max}.
    The measured operator is |n><n|; drive eps(t)(a + a^dag) with a Gaussian envelope
    centred at T/2 with width sigma; zero temperature."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(B):
        delta = rng.uniform(-TWO_PI * 0.01, TWO_PI * 0.01)
        kerr = rng.uniform(-TWO_PI * 0.25, -TWO_PI * 0.15)
        gamma = 10.0 ** rng.uniform(-4.0, -3.0)
        peak = rng.uniform(0.0, TWO_PI * 0.05)
        n = int(rng.integers(0, 3))
        N = int(rng.integers(n_min, n_max + 1))
        ch = [Channel("gauss", (peak, 0.0, T / 2.0, sigma))]
        out.append(Problem(
            n_modes=1, N=(N,),
            h_terms=kerr_mode_terms(1, 0, delta, kerr) + gauss_drive_terms(1, 0, 0),
            jumps=damping_jumps(1, 0, gamma, 0.0),
            measured=projector(1, (n,)),
            channels=ch, T=T, dt=dt, name=f"kerr_batch[{b}]"))
    return out


def damped_ho(N: int = 20, omega: float = 1.3, gamma: float = 0.2, n_th: float = 0.3,
              measured: str = "a", T: float = 2.0, dt: float = 0.001) -> Problem:
    """Damped harmonic oscillator (K = 0) for closed-form checks; ``measured`` is 'a'
    (A(0) = a) or 'n' (A(0) = a^dag a)."""
    if measured == "a":
        meas = {((k,), (k + 1,)): complex(math.sqrt(k + 1)) for k in range(N - 1)}
    elif measured == "n":
        meas = {((k,), (k,)): complex(k) for k in range(1, N)}
    else:
        raise ValueError(measured)
    return Problem(n_modes=1, N=(N,), h_terms=kerr_mode_terms(1, 0, omega, 0.0),
                   jumps=damping_jumps(1, 0, gamma, n_th), measured=meas,
                   T=T, dt=dt, name=f"damped_ho_{measured}")


def random_problem(seed: int, n_modes: int = 1, N: int = 6, n_steps: int = 20,
                   dt: float = 0.01, with_drive: bool = True, n_th: float = 0.1,
                   dense_measured: bool = False) -> Problem:
    """A small random problem exercising every term type (for parity on tiny sizes):
    per-mode detuning, Kerr, a complex Gaussian drive, thermal damping, exchange
    coupling between neighbouring modes, a squeezing-type a^dag^2 + a^2 term and,
    for dense_measured, a random Hermitian measured operator on the low block."""
    rng = np.random.Generator(np.random.PCG64(seed))
    terms: List[HTerm] = []
    jumps: List[Jump] = []
    chans: List[Channel] = []
    for j in range(n_modes):
        terms += kerr_mode_terms(n_modes, j, rng.uniform(-1, 1), rng.uniform(-0.5, 0.5))
        jumps += damping_jumps(n_modes, j, rng.uniform(0.05, 0.3), n_th)
        if with_drive:
            chans.append(Channel("gauss", (rng.uniform(0.2, 0.8), rng.uniform(-0.5, 0.5),
                                           n_steps * dt * rng.uniform(0.2, 0.8),
                                           n_steps * dt * 0.3)))
            terms += gauss_drive_terms(n_modes, j, len(chans) - 1)
        s = complex(rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2))
        z = _zero(n_modes)
        terms.append(HTerm(s, _unit(n_modes, j, 2), z))
        terms.append(HTerm(s.conjugate(), z, _unit(n_modes, j, 2)))
    for j in range(n_modes - 1):
        g = rng.uniform(0.1, 0.4)
        u1 = tuple(1 if i == j else 0 for i in range(n_modes))
        u2 = tuple(1 if i == j + 1 else 0 for i in range(n_modes))
        terms.append(HTerm(complex(g), u1, u2))
        terms.append(HTerm(complex(g), u2, u1))
    if dense_measured:
        lo = min(3, N)
        idx = [tuple(int(c) for c in np.unravel_index(i, (lo,) * n_modes)) for i in range(lo ** n_modes)]
        m = rng.normal(size=(len(idx), len(idx))) + 1j * rng.normal(size=(len(idx), len(idx)))
        m = m + m.conj().T
        meas = {(idx[a], idx[b]): complex(m[a, b]) for a in range(len(idx)) for b in range(len(idx))}
    else:
        n = tuple(int(rng.integers(0, min(3, N))) for _ in range(n_modes))
        meas = projector(n_modes, n)
    return Problem(n_modes=n_modes, N=(N,) * n_modes, h_terms=terms, jumps=jumps,
                   measured=meas, channels=chans, T=n_steps * dt, dt=dt,
                   name=f"random[{seed}]")


# ---- secular ("proper") dissipator, Eq. 203 / Eq. S9 -----------------------------------
def thermal_nbar(omega: float, eta: float, kT: float, n_levels: int) -> tuple:
    """Eq. S10: occupation of the bath mode at the n <-> n+1 transition frequency
    omega + 2 eta n, nbar_n = 1 / (exp((omega + 2 eta n) / kT) - 1), kT = k_B T_E / hbar in
    rad/ns; kT = 0 gives the zero-temperature case.  Every transition frequency must be
    positive (a lab-frame omega well above 2 |eta| n_levels)."""
    if kT <= 0.0:
        return ()
    if any(omega + 2.0 * eta * n <= 0.0 for n in range(n_levels)):
        raise ValueError("transition frequency omega + 2 eta n <= 0 inside the truncation")
    return tuple(1.0 / math.expm1((omega + 2.0 * eta * n) / kT) for n in range(n_levels))


def kerr_secular(N: int = 12, T: float = 20.0, dt: float = 0.005, kappa: float = 0.05, kT: float = 0.0,
                 omega_q: float = TWO_PI * 5.0, drive_peak: float = TWO_PI * 0.05,
                 measured=None) -> Problem:
    """A driven Kerr oscillator (Delta = 0, K = -2pi 0.2 in the rotating frame) damped by the
    secular dissipator at rate kappa; thermal occupations from Eq. S10 at the lab-frame
    transition frequencies omega_q + 2 eta n (eta = K/2)."""
    kerr = -TWO_PI * 0.2
    nbar = thermal_nbar(omega_q, 0.5 * kerr, kT, N - 1)
    return Problem(
        n_modes=1, N=(N,),
        h_terms=kerr_mode_terms(1, 0, 0.0, kerr) + gauss_drive_terms(1, 0, 0),
        jumps=[], secular=[SecularDamping(0, kappa, nbar)],
        measured=measured if measured is not None else projector(1, (1,)),
        channels=[Channel("gauss", (drive_peak, 0.0, T / 2.0, T / 6.0))],
        T=T, dt=dt, name="kerr_secular")


def two_mode_secular(N: int = 5, T: float = 4.0, dt: float = 0.01, kappa: float = 0.1, kT: float = 0.0) -> Problem:
    """The two exchange-coupled Kerr modes with the secular dissipator on each mode and a
    Gaussian drive on mode 1."""
    p = two_mode(N=N, T=T, dt=dt)
    p.jumps = []
    p.secular = [SecularDamping(j, kappa, thermal_nbar(TWO_PI * (5.0 + 0.1 * j), -TWO_PI * 0.1, kT, N - 1))
                 for j in range(2)]
    p.channels = [Channel("gauss", (TWO_PI * 0.05, 0.0, T / 2.0, T / 6.0))]
    p.h_terms = p.h_terms + gauss_drive_terms(2, 0, 0)
    p.name = "two_mode_secular"
    return p


def secular_batch(B: int = 4096, seed: int = 20220311, T: float = 100.0, dt: float = 0.002,
                  n_min: int = 10, n_max: int = 40) -> List[Problem]:
    """kerr_batch's instances (same draws) with the secular dissipator in place of the
    conventional one, at zero temperature."""
    out = []
    for p in kerr_batch(B=B, seed=seed, T=T, dt=dt, n_min=n_min, n_max=n_max):
        gamma = p.jumps[0].rate
        p.jumps = []
        p.secular = [SecularDamping(0, gamma, ())]
        p.name = p.name.replace("kerr_batch", "secular_batch")
        out.append(p)
    return out


# ---- Table I network (lab frame), the paper's Fig. 2 workload ------------------------------
TABLE_ONE = dict(omega_q=TWO_PI * 3.5, omega_d=TWO_PI * 3.5, eta=TWO_PI * 0.25, Omega_1=TWO_PI * 0.125,
                 kappa=2e-5, J=TWO_PI * 0.01)  # rad/ns and 1/ns (Table I, in 2 pi x MHz there)


def table_one_network(n_modes: int, N: int, scaled_time: float = 10.0, steps: int = 2000) -> Problem:
    """The network of Eq. 301 with Table I's parameters in the lab frame: n_modes coupled
    anharmonic oscillators (omega_q a^dag a + eta (a^dag)^2 a^2, exchange J between every
    pair), mode 1 driven by i Omega_1 a e^(i omega_d t) + H.c., each damped by the secular
    dissipator at T_E = 0 with rate kappa; A(0) = a_1 (x) ... (x) a_n; evolved to the scaled
    time omega_q t / pi = scaled_time in `steps` RK4 steps."""
    p = TABLE_ONE
    z = _zero(n_modes)
    h: List[HTerm] = []
    for j in range(n_modes):
        a = _unit(n_modes, j, 1)
        a2 = _unit(n_modes, j, 2)
        h.append(HTerm(p["omega_q"] + 0j, a, a))
        h.append(HTerm(p["eta"] + 0j, a2, a2))
        for k in range(j + 1, n_modes):
            ak = _unit(n_modes, k, 1)
            h.append(HTerm(p["J"] + 0j, ak, a))  # J a_j a_k^dag
            h.append(HTerm(p["J"] + 0j, a, ak))  # + H.c.
    a1 = _unit(n_modes, 0, 1)
    h.append(HTerm(1j * p["Omega_1"], z, a1, channel=0))               # i Omega a e^{i omega_d t}
    h.append(HTerm(-1j * p["Omega_1"], a1, z, channel=0, conj=True))  # H.c.
    meas = {}
    for k in np.ndindex(*([N - 1] * n_modes)):
        meas[(tuple(int(x) for x in k), tuple(int(x) + 1 for x in k))] = complex(
            math.prod(math.sqrt(x + 1) for x in k))
    T = scaled_time * math.pi / p["omega_q"]
    return Problem(n_modes=n_modes, N=(N,) * n_modes, h_terms=h, jumps=[],
                   secular=[SecularDamping(j, p["kappa"], ()) for j in range(n_modes)],
                   measured=meas, channels=[Channel("cexp", (1.0, 0.0, p["omega_d"]))],
                   T=T, dt=T / steps, name=f"table_one_{n_modes}")
