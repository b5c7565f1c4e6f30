"""Pins for the secular ("proper") dissipator of Eq. 203 / Eq. S9 in both oracles: O1
(number basis, the printed Schroedinger form and its adjoint, coded separately) and O2 (the
mapping: separable decay in O_x / O_y plus the projector P of Eq. 302c / Eq. S15)."""

import math

import numpy as np
import pytest

from oracle import fock, mapping
from workloads import configs
from workloads.spec import HTerm, Problem, SecularDamping

TWO_PI = 2.0 * math.pi


def _random_rho(dim, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(dim, dim)) + 1j * rng.normal(size=(dim, dim))
    rho = X @ X.conj().T
    return rho / np.trace(rho)


def _osc(N, kappa, measured, delta=0.0, kerr=0.0, nbar=(), standard=False, T=2.0, dt=0.005):
    z, a = (0,), (1,)
    h = []
    if delta:
        h.append(HTerm(delta + 0j, a, a))
    if kerr:
        h.append(HTerm(0.5 * kerr + 0j, (2,), (2,)))
    return Problem(n_modes=1, N=(N,), h_terms=h,
                   jumps=configs.damping_jumps(1, 0, kappa, 0.0) if standard else [],
                   secular=[] if standard else [SecularDamping(0, kappa, tuple(nbar))],
                   measured=measured, T=T, dt=dt)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_zero_temperature_diagonal_equals_conventional(m):
    """At T_E = 0 the two dissipators differ only in the jump term, which for a diagonal
    operator is the same (Eq. S13 vs the conventional a^dag A a): |m><m| under Kerr +
    damping evolves identically, and matches the binomial closed form."""
    kappa, N = 0.3, 9
    meas = {((m,), (m,)): 1.0}
    As = fock.rk4_adjoint(_osc(N, kappa, meas, kerr=-1.3))
    Ac = fock.rk4_adjoint(_osc(N, kappa, meas, kerr=-1.3, standard=True))
    assert np.max(np.abs(As - Ac)) < 1e-13
    gt = kappa * 2.0
    for k in range(N):
        ref = math.comb(k, m) * math.exp(-m * gt) * (1 - math.exp(-gt)) ** (k - m) if k >= m else 0.0
        assert abs(As[k, k] - ref) < 1e-10


def test_annihilation_closed_form_differs_from_conventional():
    """A(0) = a under H = Delta a^dag a and the secular dissipator at T_E = 0: the off-diagonal
    elements never receive the jump term, so A_{k,k+1}(t) = sqrt(k+1) exp(-(i Delta +
    kappa (2k+1)/2) t) (Eq. S13 with delta_{k,l}); the conventional dissipator gives the
    uniform decay sqrt(k+1) exp(-(i Delta + kappa/2) t) instead."""
    kappa, delta, N, T = 0.2, 0.7, 8, 2.0
    meas = {((k,), (k + 1,)): math.sqrt(k + 1) for k in range(N - 1)}
    As = fock.rk4_adjoint(_osc(N, kappa, meas, delta=delta, T=T))
    Ac = fock.rk4_adjoint(_osc(N, kappa, meas, delta=delta, T=T, standard=True))
    for k in range(N - 1):
        ref_s = math.sqrt(k + 1) * np.exp(-(1j * delta + kappa * (2 * k + 1) / 2) * T)
        ref_c = math.sqrt(k + 1) * np.exp(-(1j * delta + kappa / 2) * T)
        assert abs(As[k, k + 1] - ref_s) < 1e-9  # RK4 error at dt = 0.005 is ~1e-10
        assert abs(Ac[k, k + 1] - ref_c) < 1e-9
    assert np.max(np.abs(np.diag(As))) == 0.0


@pytest.mark.parametrize("which", ["single", "two_mode"])
def test_adjoint_schroedinger_duality_finite_temperature(which):
    """Tr(rho(T) A0) with the printed forward equation (Eq. S9, drive, thermal nbar_n)
    equals Tr(rho0 A(T)) with the adjoint, to rounding: pins the adjoint derivation."""
    if which == "single":
        p = configs.kerr_secular(N=7, T=1.0, dt=0.01, kappa=0.3, kT=TWO_PI * 1.64,
                                 measured={((1,), (2,)): 0.4 + 0.1j, ((2,), (1,)): 0.4 - 0.1j, ((3,), (3,)): 1.0})
    else:
        p = configs.two_mode_secular(N=4, T=0.5, dt=0.01, kappa=0.3, kT=TWO_PI * 1.64)
        p.measured = {((1, 0), (0, 1)): 1.0 + 0.5j, ((0, 1), (1, 0)): 1.0 - 0.5j, ((1, 1), (1, 1)): 0.3}
    A0 = fock.operator_matrix(p.measured, p.N)
    rho0 = _random_rho(A0.shape[0], 5)
    AT = fock.rk4_adjoint(p)
    rhoT = fock.schrodinger_rk4(p, rho0)
    assert abs(np.trace(rhoT @ A0) - np.trace(rho0 @ AT)) < 1e-12


def test_unitality_and_hermiticity():
    p = configs.kerr_secular(N=7, T=1.0, dt=0.01, kappa=0.3, kT=TWO_PI * 1.64)
    I = np.eye(7)
    assert np.max(np.abs(fock.rk4_adjoint(p, A0=I) - I)) < 1e-12
    A0 = fock.operator_matrix({((1,), (2,)): 0.4 + 0.1j, ((2,), (1,)): 0.4 - 0.1j, ((0,), (0,)): 1.0}, (7,))
    AT = fock.rk4_adjoint(p, A0=A0)
    assert np.max(np.abs(AT - AT.conj().T)) < 1e-13


def test_thermal_state_is_stationary():
    """Detailed balance of Eq. S9: rho_{n+1,n+1} / rho_{n,n} = nbar_n / (1 + nbar_n) is a
    fixed point of the forward dissipator (nbar vanishing at the truncation edge)."""
    N = 8
    nbar = configs.thermal_nbar(TWO_PI * 5.0, -TWO_PI * 0.1, TWO_PI * 3.0, N - 1)
    p = _osc(N, 0.4, {((1,), (1,)): 1.0}, kerr=-1.0, nbar=nbar)
    pops = [1.0]
    for n in range(N - 1):
        pops.append(pops[-1] * nbar[n] / (1.0 + nbar[n]))
    rho = np.diag(np.array(pops) / sum(pops)).astype(complex)
    model = fock.FockModel(p)
    out = model.schrodinger_generator(rho, model.h_static)
    assert np.max(np.abs(out)) < 1e-15
    # and a non-thermal diagonal state is not
    rho2 = np.diag(np.full(N, 1.0 / N)).astype(complex)
    assert np.max(np.abs(model.schrodinger_generator(rho2, model.h_static))) > 1e-3


def test_liouvillian_contains_secular_terms():
    """The dense superoperator (column by column) generates the same evolution as RK4."""
    import scipy.linalg
    nbar = configs.thermal_nbar(TWO_PI * 5.0, -TWO_PI * 0.1, TWO_PI * 1.64, 5)
    p = _osc(6, 0.3, {((1,), (2,)): 1.0, ((2,), (1,)): 1.0}, delta=0.4, kerr=-0.8, nbar=nbar, T=1.0, dt=0.005)
    model = fock.FockModel(p)
    L = fock.adjoint_liouvillian(p, model.h_static)
    A0 = fock.operator_matrix(p.measured, p.N)
    ref = (scipy.linalg.expm(L * p.T) @ A0.reshape(-1)).reshape(A0.shape)
    assert np.max(np.abs(fock.rk4_adjoint(p) - ref)) < 1e-10


def test_mapping_generator_equals_number_basis_generator():
    """One application of the generators: O2's (decay + P) on g equals O1's adjoint secular
    dissipator on A = sqrt(k! l!) g (Eq. 6 / Eq. 8), element by element, for two modes at
    finite temperature (a dropped weight, a wrong index shift or a missing diagonal
    restriction fails this)."""
    p = configs.two_mode_secular(N=4, kT=TWO_PI * 1.64, kappa=0.37)
    p.h_terms = []
    p.channels = []
    model = mapping.MappedModel(p)
    fm = fock.FockModel(p)
    d = model.dim
    rng = np.random.default_rng(11)
    g = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Ox, Oy = model.operators(0.0, 0.0, p.dt)
    _, _, dR = model.rhs(np.zeros(d), np.zeros(d), g, Ox, Oy, 0.0, "full")
    ks = np.array([math.sqrt(math.prod(math.factorial(int(x)) for x in np.unravel_index(i, p.N))) for i in range(d)])
    A = g * np.outer(ks, ks)
    dA = fm.secular_adjoint(A)
    assert np.max(np.abs(dR * np.outer(ks, ks) - dA)) < 1e-12 * np.max(np.abs(dA))


@pytest.mark.parametrize("which", ["single", "two_mode"])
def test_all_in_R_equals_number_basis(which):
    """Linear RK4 on G (all in R) equals O1 to rounding with the secular dissipator, drive
    and thermal occupations."""
    if which == "single":
        p = configs.kerr_secular(N=8, T=0.5, dt=0.01, kappa=0.3, kT=TWO_PI * 1.64,
                                 measured={((1,), (2,)): 0.4 + 0.1j, ((2,), (1,)): 0.4 - 0.1j, ((3,), (3,)): 1.0})
    else:
        p = configs.two_mode_secular(N=4, T=0.3, dt=0.01, kappa=0.3, kT=TWO_PI * 1.64)
    A = fock.rk4_adjoint(p)
    run = mapping.rk4_mapped(p, all_in_R=True)
    assert np.max(np.abs(run.fock_matrix() - A)) < 1e-12 * np.max(np.abs(A))


def test_separated_converges_to_number_basis():
    p = configs.kerr_secular(N=7, T=0.4, dt=0.02, kappa=0.4, kT=TWO_PI * 1.64,
                             measured={((1,), (2,)): 0.4 + 0.1j, ((2,), (1,)): 0.4 - 0.1j, ((3,), (3,)): 1.0})
    errs = []
    for _ in range(2):
        A = fock.rk4_adjoint(p)
        errs.append(np.max(np.abs(mapping.rk4_mapped(p).fock_matrix() - A)))
        p = Problem(**{**p.__dict__, "dt": p.dt / 2})
    assert errs[1] < errs[0]
    assert 11.0 < errs[0] / errs[1] < 22.0


def test_off_diagonal_operator_keeps_zero_residual_without_drive():
    """Eq. S15 at T_E = 0 with A(0) = a and no drive: every separable product G_x G_y stays
    off-diagonal, so P never sources R and R stays exactly zero (the conventional
    dissipator's x y source makes it nonzero)."""
    meas = {((k,), (k + 1,)): math.sqrt(k + 1) for k in range(5)}
    run = mapping.rk4_mapped(_osc(6, 0.3, meas, delta=0.5, kerr=-0.7, T=0.5, dt=0.01))
    assert all(np.max(np.abs(ic[6])) == 0.0 for ic in run.ics)
    run_c = mapping.rk4_mapped(_osc(6, 0.3, meas, delta=0.5, kerr=-0.7, T=0.5, dt=0.01, standard=True))
    assert max(np.max(np.abs(ic[6])) for ic in run_c.ics) > 1e-3


# ---- diagonal residual layout (R as a function of x_j y_j only) --------------------------
@pytest.mark.parametrize("which", ["single_secular", "single_conventional", "two_uncoupled"])
def test_diag_layout_exact_when_dynamics_keep_diagonality(which):
    """With a diagonal measured operator, a diagonal Hamiltonian (Kerr, detuning) and either
    dissipator, every term maps diagonal to diagonal, so the full residual R stays diagonal
    and the diagonal layout must reproduce the full run to rounding."""
    if which == "two_uncoupled":
        p = configs.two_mode_secular(N=4, T=0.5, dt=0.01, kappa=0.3, kT=TWO_PI * 1.64)
        p.h_terms = [t for t in p.h_terms if sum(t.u) == sum(t.v) and all(a == b for a, b in zip(t.u, t.v))]
        p.channels = []
        p.measured = {((1, 0), (1, 0)): 1.0, ((2, 1), (2, 1)): 0.5, ((0, 0), (0, 0)): 0.2}
    else:
        meas = {((1,), (1,)): 1.0, ((3,), (3,)): -0.4}
        p = _osc(8, 0.3, meas, delta=0.4, kerr=-1.1, standard=(which == "single_conventional"),
                 nbar=(0.05, 0.06, 0.07), T=0.5, dt=0.01)
    full = mapping.rk4_mapped(p)
    for ic in full.ics:
        R = ic[6]
        assert np.max(np.abs(R - np.diag(np.diag(R)))) == 0.0
    diag = mapping.rk4_mapped(p, r_layout="diag")
    A, B = full.fock_matrix(), diag.fock_matrix()
    assert np.max(np.abs(A - B)) < 1e-14 * np.max(np.abs(A))
    assert np.max(np.abs(B - fock.rk4_adjoint(p))) < 1e-6  # the separated run vs O1 (RK4 error)


def test_diag_layout_approximation_is_first_order_in_kappa_t():
    """With a drive the residual is not diagonal; keeping its x y part is an approximation
    (the paper's observation) whose error grows like kappa t and stays well below that of
    dropping R altogether (R = 0)."""
    meas = {((k,), (k + 1,)): math.sqrt(k + 1) for k in range(7)}
    errs = {}
    for kappa in (0.002, 0.01):
        p = configs.kerr_secular(N=8, T=5.0, dt=0.01, kappa=kappa, kT=0.0, drive_peak=TWO_PI * 0.05, measured=meas)
        blk = lambda X: fock.low_block(X, (8,), 3)
        full = blk(mapping.rk4_mapped(p).fock_matrix())
        errs[kappa] = tuple(fock.eps_r(blk(mapping.rk4_mapped(p, r_layout=lay).fock_matrix()), full)
                            for lay in ("diag", "off"))
    for kappa, (e_diag, e_off) in errs.items():
        assert e_diag < 0.5 * e_off
    ratio = errs[0.01][0] / errs[0.002][0]
    assert 3.5 < ratio < 6.5, ratio
