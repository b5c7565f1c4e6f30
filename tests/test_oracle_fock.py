"""Pins for O1 (number-basis adjoint master equation, Eq. 3) against closed forms,
dualities and library routines -- none of which reuse O1's own arithmetic."""

import math

import numpy as np
import pytest
import scipy.linalg

from oracle import channels, fock
from workloads import configs
from workloads.spec import Channel, HTerm, Jump, Problem


def test_channel_values():
    g = Channel("gauss", (2.0, -1.0, 5.0, 2.0))
    assert channels.channel_value(g, 5.0) == complex(2.0, -1.0)
    assert abs(channels.channel_value(g, 7.0) - complex(2.0, -1.0) * math.exp(-0.5)) < 1e-15
    p = Channel("pwc", (0.0, 1.0, 1.0, 2.0, 3.0, 4.0))
    assert channels.channel_value(p, 0.5) == complex(1.0, 2.0)
    assert channels.channel_value(p, 1.0) == complex(3.0, 4.0)
    assert channels.channel_value(p, 2.5) == 0j
    c = Channel("cexp", (1.0, 0.0, math.pi))
    assert abs(channels.channel_value(c, 0.5) - 1j) < 1e-15
    # pwc is read at the step midpoint, reversed time maps tau -> T - tau
    assert channels.stage_value(p, 0.0, 1.0, 0.5, 2.0, True) == complex(3.0, 4.0)
    assert channels.stage_value(p, 0.0, 0.0, 0.5, 2.0, False) == complex(1.0, 2.0)


@pytest.mark.parametrize("n_th", [0.0, 0.3])
def test_damped_oscillator_annihilation(n_th):
    """A(0) = a: A(t) = a exp(-(i omega + gamma/2) t) (spec closed form)."""
    p = configs.damped_ho(N=24, omega=1.3, gamma=0.2, n_th=n_th, measured="a", T=2.0, dt=0.002)
    A = fock.rk4_adjoint(p)
    a = fock.ladder(24)
    ref = a * np.exp(-(1j * 1.3 + 0.1) * 2.0)
    lo = 10  # away from the truncation edge
    assert np.max(np.abs(A[:lo, :lo] - ref[:lo, :lo])) < 1e-10 * np.max(np.abs(ref[:lo, :lo]))


@pytest.mark.parametrize("n_th", [0.0, 0.3])
def test_damped_oscillator_number(n_th):
    """A(0) = a^dag a: A(t) = e^{-gamma t} a^dag a + n_th (1 - e^{-gamma t})."""
    N, gamma, T = 24, 0.2, 2.0
    p = configs.damped_ho(N=N, omega=1.3, gamma=gamma, n_th=n_th, measured="n", T=T, dt=0.002)
    A = fock.rk4_adjoint(p)
    ref = np.diag(np.arange(N) * math.exp(-gamma * T) + n_th * (1.0 - math.exp(-gamma * T)))
    lo = 10
    assert np.max(np.abs(A[:lo, :lo] - ref[:lo, :lo])) < 1e-10 * np.max(np.abs(ref[:lo, :lo]))


@pytest.mark.parametrize("m", [0, 1, 2])
def test_binomial_closed_form_kerr(m):
    """|m><m| under Kerr + zero-temperature damping: A_kk(t) = C(k,m) e^{-m g t}(1-e^{-g t})^{k-m},
    off-diagonal elements stay exactly zero (the Kerr term commutes with diagonal A)."""
    p = configs.kerr_static(N=12)
    p.measured = configs.projector(1, (m,))
    p.T = 20.0
    p.jumps = configs.damping_jumps(1, 0, 0.05, 0.0)
    A = fock.rk4_adjoint(p)
    gt = 0.05 * p.T
    for k in range(12):
        ref = math.comb(k, m) * math.exp(-m * gt) * (1 - math.exp(-gt)) ** (k - m) if k >= m else 0.0
        assert abs(A[k, k] - ref) < 1e-12
    assert np.max(np.abs(A - np.diag(np.diag(A)))) == 0.0


def _random_rho(dim, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(dim, dim)) + 1j * rng.normal(size=(dim, dim))
    rho = X @ X.conj().T
    return rho / np.trace(rho)


@pytest.mark.parametrize("seed,n_modes", [(1, 1), (2, 2)])
def test_heisenberg_schroedinger_duality(seed, n_modes):
    """Tr(rho(T) A0) from the forward density-matrix RK4 equals Tr(rho0 A(T)) from the
    reversed-time adjoint RK4 to rounding (the adjoint RK4 with reversed stage times is the
    exact transpose of the forward one).  Pins the generator, its adjoint and the time
    reading for time-dependent drives."""
    p = configs.random_problem(seed, n_modes=n_modes, N=5 if n_modes == 2 else 8,
                               n_steps=40, dt=0.02, dense_measured=True)
    A0 = fock.operator_matrix(p.measured, p.N)
    rho0 = _random_rho(A0.shape[0], seed)
    AT = fock.rk4_adjoint(p)
    rhoT = fock.schrodinger_rk4(p, rho0)
    lhs = np.trace(rhoT @ A0)
    rhs = np.trace(rho0 @ AT)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_trace_preservation_zero_temperature():
    """With jump operators that only lower (a), the compressed forward equation is
    trace preserving (with a^dag jumps the compression loses population at level N)."""
    p = configs.random_problem(3, n_modes=1, N=8, n_steps=40, dt=0.02, n_th=0.0)
    rho0 = _random_rho(8, 3)
    rhoT = fock.schrodinger_rk4(p, rho0)
    assert abs(np.trace(rhoT) - 1.0) < 1e-13


def test_pwc_duality():
    p = configs.two_mode_control(n_seg=4, T=2.0, steps_per_seg=5, N=4)
    A0 = fock.operator_matrix(p.measured, p.N)
    rho0 = _random_rho(A0.shape[0], 7)
    AT = fock.rk4_adjoint(p)
    rhoT = fock.schrodinger_rk4(p, rho0)
    assert abs(np.trace(rhoT @ A0) - np.trace(rho0 @ AT)) < 1e-12


def test_liouvillian_expm_static():
    """Static H: RK4 matches expm of the dense adjoint Liouvillian within RK4 error."""
    p = configs.random_problem(4, n_modes=1, N=7, n_steps=100, dt=0.01, with_drive=False,
                               dense_measured=True)
    model = fock.FockModel(p)
    Lsup = fock.adjoint_liouvillian(p, model.h_static)
    A0 = fock.operator_matrix(p.measured, p.N)
    ref = (scipy.linalg.expm(Lsup * p.T) @ A0.reshape(-1)).reshape(A0.shape)
    e1 = np.max(np.abs(fock.rk4_adjoint(p) - ref))
    p.dt = p.dt / 2
    e2 = np.max(np.abs(fock.rk4_adjoint(p) - ref))
    assert e2 < 1e-8 * np.max(np.abs(ref))
    assert 12.0 < e1 / e2 < 20.0  # fourth order


def test_closed_system_unitary():
    """kappa = 0, static H: A(T) = U^dag A U with U = exp(-i H T) (scipy.linalg.expm)."""
    p = configs.random_problem(5, n_modes=2, N=4, n_steps=200, dt=0.005, with_drive=False,
                               dense_measured=True)
    p.jumps = []
    model = fock.FockModel(p)
    U = scipy.linalg.expm(-1j * model.h_static * p.T)
    A0 = fock.operator_matrix(p.measured, p.N)
    ref = U.conj().T @ A0 @ U
    e1 = np.max(np.abs(fock.rk4_adjoint(p) - ref))
    p.dt = p.dt / 2
    e2 = np.max(np.abs(fock.rk4_adjoint(p) - ref))
    assert e2 < 1e-8 * np.max(np.abs(ref))
    assert 12.0 < e1 / e2 < 20.0


def test_hermiticity_and_unitality():
    p = configs.random_problem(6, n_modes=1, N=8, n_steps=50, dense_measured=True, n_th=0.0)
    A = fock.rk4_adjoint(p)
    assert np.max(np.abs(A - A.conj().T)) < 1e-13
    Id = fock.rk4_adjoint(p, A0=np.eye(8))
    assert np.max(np.abs(Id - np.eye(8))) < 1e-13


def test_thermal_truncation_reading():
    """L = a^dag enters through P (a a^dag) P = diag(1..N): the exact matrix elements of
    L^dag L in the truncated span."""
    p = Problem(n_modes=1, N=(5,), h_terms=[], jumps=[Jump(1.0, ((1.0, (1,), (0,)),))],
                measured={((0,), (0,)): 1.0}, T=0.1, dt=0.1)
    m = fock.FockModel(p)
    _, L, Ld, LdL = m.jumps[0]
    assert np.allclose(np.diag(LdL).real, np.arange(1, 6))
    assert np.allclose(L, fock.ladder(5).conj().T)
