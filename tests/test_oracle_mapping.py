"""Pins for O2 (the mapping method) against brute force, the paper's printed operators,
closed forms and O1 -- chosen so that a dropped term, a wrong sign, a swapped side
(left vs right multiplication) or a transposed operand fails one of them."""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import fock, mapping
from workloads import configs
from workloads.spec import Channel, HTerm, Jump, Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_T_basis_is_scaled_number_projector():
    """Eq. 8 summed explicitly (padded truncation) gives T_{k,l} = sqrt(k! l!) |k><l| on the
    low levels: the identity behind g_{k,l} = <k|A|l> / sqrt(k! l!)."""
    P, lo = 40, 8
    a = fock.ladder(P)
    ad = a.conj().T
    for k in range(5):
        for l in range(5):
            T = np.zeros((P, P), dtype=np.complex128)
            for j in range(P):
                T += (-1.0) ** j / math.factorial(j) * (
                    np.linalg.matrix_power(ad, k + j) @ np.linalg.matrix_power(a, l + j))
            ref = np.zeros((lo, lo))
            ref[k, l] = math.sqrt(math.factorial(k) * math.factorial(l))
            assert np.max(np.abs(T[:lo, :lo] - ref)) < 1e-10 * max(1.0, ref.max())


def test_g_from_number_basis_two_modes():
    rng = np.random.default_rng(0)
    M = (4, 3)
    A = rng.normal(size=M + M) + 1j * rng.normal(size=M + M)
    g = mapping.g_from_f(mapping.f_from_fock(A, 2), 2)
    # D^-1 A D^-1 with D = diag(sqrt(k!)) per mode
    kk = np.array([[math.sqrt(math.factorial(k1) * math.factorial(k2)) for k2 in range(3)] for k1 in range(4)])
    ref = A / (kk[:, :, None, None] * kk[None, None, :, :])
    assert np.max(np.abs(g - ref)) < 1e-12 * np.max(np.abs(ref))


def test_fock_from_f_explicit_sum():
    rng = np.random.default_rng(1)
    M = 5
    f = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    P = 2 * M
    A = np.zeros((P, P), dtype=np.complex128)
    for k in range(M):
        for l in range(M):
            A += f[k, l] * fock.monomial((k,), (l,), (P,))
    assert np.max(np.abs(mapping.fock_from_f(f, 1) - A[:M, :M])) < 1e-12 * np.max(np.abs(A[:M, :M]))


def test_round_trips():
    rng = np.random.default_rng(2)
    M = (3, 4)
    f = rng.normal(size=M + M) + 1j * rng.normal(size=M + M)
    assert np.max(np.abs(mapping.f_from_g(mapping.g_from_f(f, 2), 2) - f)) < 1e-13
    assert np.max(np.abs(mapping.f_from_fock(mapping.fock_from_f(f, 2), 2) - f)) < 1e-11


def test_projector_maps_to_single_ic():
    """|n><m| has a single non-negligible g_{n,m}(0) = 1/sqrt(n! m!) (Eq. 13 case d = m - n)."""
    for n, m in [(0, 0), (1, 1), (2, 3), (3, 1)]:
        p = configs.kerr_static(N=10)
        p.measured = {((n,), (m,)): 1.0}
        g0, ics = mapping.map_initial(p)
        assert len(ics) == 1
        (pp, qq, w), = ics
        assert pp == (n,) and qq == (m,)
        assert abs(w - 1.0 / math.sqrt(math.factorial(n) * math.factorial(m))) < 1e-15


def test_separation_constant_minimises_functional():
    """Eq. 304 is the minimiser of |G_x'/G_x|^2 + |G_y'/G_y|^2 for the uncoupled, undamped,
    undriven oscillator at t = 0 (checked by numerical minimisation)."""
    for (omega, eta, p, q) in [(1.3, -0.4, 1, 1), (0.7, 0.25, 2, 0), (-0.2, 0.1, 3, 2)]:
        prob = Problem(n_modes=1, N=(6,), h_terms=configs.kerr_mode_terms(1, 0, omega, 2 * eta),
                       jumps=[], measured={((p,), (q,)): 1.0}, T=1.0, dt=0.1)
        model = mapping.MappedModel(prob)
        a = model.Ox[p, p]  # G_x'/G_x for G_x = x^p without C
        b = model.Oy[q, q]

        def fun(z):
            C = z[0] + 1j * z[1]
            return abs(a + C) ** 2 + abs(b - C) ** 2

        res = scipy.optimize.minimize(fun, [0.0, 0.0], tol=1e-14)
        C_num = res.x[0] + 1j * res.x[1]
        assert abs(C_num - mapping.separation_constant(prob, (p,), (q,))) < 1e-6


def test_paper_Kx_Ky_table1():
    """The left/right operators of a single Table-I oscillator equal K_x, K_y as printed in
    Eqs. 302a, 302b:  K_x = (i w - k/2) x d_x + i eta x^2 d_x^2 - W e^{i wd t} d_x + W^* e^{-i wd t} x,
    K_y = (-i w - k/2) y d_y - i eta y^2 d_y^2 + W e^{i wd t} y - W^* e^{-i wd t} d_y."""
    with open(os.path.join(GOLDEN, "table1.json")) as fh:
        t1 = json.load(fh)
    to_rad_ns = 2 * math.pi * 1e-3  # 2pi x MHz -> rad/ns
    w = t1["omega_q"] * to_rad_ns
    wd = t1["omega_d"] * to_rad_ns
    eta = t1["eta"] * to_rad_ns
    W = t1["Omega_1"] * to_rad_ns * (0.6 + 0.8j)  # complex amplitude
    kappa = t1["kappa_over_2pi_MHz"] * to_rad_ns
    # H = w a^dag a + eta a^dag^2 a^2 + i W a e^{i wd t} + H.c. (Eq. 301)
    terms = [HTerm(complex(w), (1,), (1,)), HTerm(complex(eta), (2,), (2,)),
             HTerm(1j * W, (0,), (1,), channel=0, conj=False),
             HTerm(np.conj(1j * W), (1,), (0,), channel=0, conj=True)]
    M = 7
    prob = Problem(n_modes=1, N=(M,), h_terms=terms,
                   jumps=[Jump(kappa, ((1.0, (0,), (1,)),))], measured={((1,), (1,)): 1.0},
                   channels=[Channel("cexp", (1.0, 0.0, wd))], T=1.0, dt=0.1, reverse_time=False)
    model = mapping.MappedModel(prob)
    t = 0.37
    Ox, Oy = model.operators(t, 0.0, 0.1)
    X = np.diag(np.ones(M - 1), -1)
    D = np.diag(np.arange(1, M, dtype=float), 1)
    e = np.exp(1j * wd * t)
    Kx = (1j * w - kappa / 2) * X @ D + 1j * eta * X @ X @ D @ D - W * e * D + np.conj(W) * np.conj(e) * X
    Ky = (-1j * w - kappa / 2) * X @ D - 1j * eta * X @ X @ D @ D + W * e * X - np.conj(W) * np.conj(e) * D
    assert np.max(np.abs(Ox - Kx)) < 1e-12
    assert np.max(np.abs(Oy - Ky)) < 1e-12
    # the standard jump a couples x and y through kappa * x * y (sandwich)
    kap, Ld_l, L_r = model.sandwich[0]
    assert abs(kap - kappa) < 1e-18
    assert np.max(np.abs(Ld_l - X)) == 0 and np.max(np.abs(L_r - X)) == 0


def test_secular_and_standard_dissipator_agree_on_diagonal():
    """S-eq. 315: for T_E = 0, dG/dt = kappa/2 (2P - x d_x - y d_y) G; on a diagonal G the
    projector P acts as multiplication by x y, so the standard dissipator must give
    dg_kk/dt = kappa (g_{k-1,k-1} - k g_kk)."""
    kappa, M = 0.3, 8
    prob = Problem(n_modes=1, N=(M,), h_terms=[], jumps=configs.damping_jumps(1, 0, kappa, 0.0),
                   measured={((1,), (1,)): 1.0}, T=1.0, dt=0.1)
    model = mapping.MappedModel(prob)
    rng = np.random.default_rng(3)
    g = np.diag(rng.normal(size=M) + 1j * rng.normal(size=M))
    Ox, Oy = model.operators(0.0, 0.0, 0.1)
    _, _, dR = model.rhs(np.zeros(M), np.zeros(M), g, Ox, Oy, 0.0, "full")
    ref = np.zeros_like(g)
    for k in range(M):
        ref[k, k] = kappa * ((g[k - 1, k - 1] if k > 0 else 0.0) - k * g[k, k])
    assert np.max(np.abs(dR - ref)) < 1e-14


@pytest.mark.parametrize("m", [0, 1, 2])
def test_kerr_closed_form_separated(m):
    """Damped Kerr oscillator measured on |m><m| (zero temperature, no drive): with Eq. 304's C,
    G_x = x^m e^{-m g t/2}, G_y = y^m e^{-m g t/2} and
    G_x G_y + R = (x y)^m e^{-m g t} exp(x y (1 - e^{-g t})), i.e.
    R_kk = e^{-m g t}(1-e^{-g t})^{k-m}/(k-m)! for k > m and 0 otherwise."""
    M, gamma = 9, 0.05
    prob = configs.kerr_static(N=M)
    prob.h_terms = configs.kerr_mode_terms(1, 0, 0.3, -1.1)
    prob.jumps = configs.damping_jumps(1, 0, gamma, 0.0)
    prob.measured = configs.projector(1, (m,))
    prob.T, prob.dt = 10.0, 0.01
    run = mapping.rk4_mapped(prob)
    (p, q, w, C, Gx, Gy, R), = run.ics
    gt = gamma * prob.T
    ex = np.zeros(M)
    ex[m] = math.exp(-m * gt / 2)
    assert np.max(np.abs(Gx - ex)) < 1e-12
    assert np.max(np.abs(Gy - ex)) < 1e-12
    ref = np.zeros((M, M))
    for k in range(m + 1, M):
        ref[k, k] = math.exp(-m * gt) * (1 - math.exp(-gt)) ** (k - m) / math.factorial(k - m)
    assert np.max(np.abs(R - ref)) < 1e-12
    assert abs(w - 1.0 / math.factorial(m)) < 1e-15


def test_closed_system_residual_vanishes():
    """kappa = 0: Eq. 9c has no source, so R stays identically zero, and G_x G_y reproduces
    U^dag A U (scipy.linalg.expm) within RK4 error."""
    p = configs.random_problem(8, n_modes=2, N=4, n_steps=100, dt=0.005, with_drive=False)
    p.jumps = []
    run = mapping.rk4_mapped(p)
    for ic in run.ics:
        assert np.max(np.abs(ic[6])) == 0.0
    model = fock.FockModel(p)
    U = scipy.linalg.expm(-1j * model.h_static * p.T)
    A0 = fock.operator_matrix(p.measured, p.N)
    ref = U.conj().T @ A0 @ U
    assert np.max(np.abs(run.fock_matrix() - ref)) < 1e-8


@pytest.mark.parametrize("seed,n_modes,N", [(11, 1, 7), (12, 2, 4), (13, 1, 6), (14, 4, 2)])
def test_all_in_R_equals_number_basis(seed, n_modes, N):
    """With G_x = G_y = 0 and R = x^p y^q the coupled system is the linear RK4 on G; since
    g = D^-1 A D^-1 (D = diag sqrt(k!)) it must equal O1 to rounding, for every term type."""
    p = configs.random_problem(seed, n_modes=n_modes, N=N, n_steps=30, dt=0.01, dense_measured=True)
    A = fock.rk4_adjoint(p)
    run = mapping.rk4_mapped(p, all_in_R=True)
    assert np.max(np.abs(run.fock_matrix() - A)) < 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("seed,n_modes,N", [(21, 1, 7), (22, 2, 4)])
def test_separated_converges_to_number_basis(seed, n_modes, N):
    """The separated (bilinear) system is not the linear RK4 on G step by step, but both are
    fourth-order consistent with Eq. 3: the difference shrinks ~16x per halving of dt."""
    p = configs.random_problem(seed, n_modes=n_modes, N=N, n_steps=20, dt=0.02, dense_measured=True)
    errs = []
    for _ in range(2):
        A = fock.rk4_adjoint(p)
        errs.append(np.max(np.abs(mapping.rk4_mapped(p).fock_matrix() - A)))
        p.dt /= 2
        p = Problem(**{**p.__dict__})
    assert errs[1] < errs[0]
    assert 11.0 < errs[0] / errs[1] < 22.0


def test_separation_constant_only_changes_rk4_error():
    p = configs.random_problem(31, n_modes=1, N=6, n_steps=20, dt=0.01)
    A = fock.rk4_adjoint(p)
    a = mapping.rk4_mapped(p).fock_matrix()
    b = mapping.rk4_mapped(p, C_override=0.0).fock_matrix()
    assert np.max(np.abs(a - A)) < 1e-7 and np.max(np.abs(b - A)) < 1e-7


def test_hermitian_symmetry_of_separated_functions():
    """For p = q and Hermitian H: O_y = conj(O_x) and C is imaginary, so G_y = conj(G_x)."""
    p = configs.random_problem(41, n_modes=1, N=7, n_steps=30, dt=0.01)
    p.measured = configs.projector(1, (1,))
    run = mapping.rk4_mapped(p)
    (_, _, _, C, Gx, Gy, R), = run.ics
    assert abs(C.real) == 0.0
    assert np.max(np.abs(Gy - np.conj(Gx))) < 1e-13
    assert np.max(np.abs(R - R.conj().T)) < 1e-13


def test_r_layout_off_exact_without_dissipation():
    p = configs.random_problem(51, n_modes=1, N=6, n_steps=20, dt=0.01)
    p.jumps = []
    a = mapping.rk4_mapped(p, r_layout="full").fock_matrix()
    b = mapping.rk4_mapped(p, r_layout="off").fock_matrix()
    assert np.max(np.abs(a - b)) == 0.0


# ---- SVD initial conditions ----------------------------------------------------------------
def _dense_problem(seed=41, n_modes=1, N=6, steps=30):
    return configs.random_problem(seed, n_modes=n_modes, N=N, n_steps=steps, dt=0.01, dense_measured=True)


@pytest.mark.parametrize("n_modes,N", [(1, 7), (2, 3)])
def test_svd_initial_conditions_reconstruct_g0_with_fewer_systems(n_modes, N):
    p = _dense_problem(n_modes=n_modes, N=N)
    g0, ics = mapping.map_initial(p)
    svd = mapping.initial_conditions_svd(g0, n_modes)
    d = int(np.prod(p.N))
    G = sum(np.outer(gx, gy) for gx, gy in svd)
    assert np.max(np.abs(G - g0.reshape(d, d))) < 1e-13 * np.max(np.abs(g0))
    assert len(svd) <= d < len(ics)


@pytest.mark.parametrize("n_modes,N", [(1, 7), (2, 3)])
def test_svd_run_equals_monomial_run_for_equal_separation_constant(n_modes, N):
    """Every step of Eqs. 9a-c is linear in the tensor product G_x(0) (x) G_y(0) of an IC
    (the source S(G_x G_y) is bilinear in the factors), so with the same C for all ICs the
    summed result depends only on sum_i G_x^i(0) (x) G_y^i(0) = g(0): the SVD and the
    monomial decompositions must agree to rounding, with dissipation and drive."""
    p = _dense_problem(n_modes=n_modes, N=N)
    a = mapping.rk4_mapped(p, C_override=0.0).fock_matrix()
    b = mapping.rk4_mapped(p, C_override=0.0, ic_mode="svd").fock_matrix()
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))
    # with Eq. 304's per-IC constants the two differ only at the RK4-error level
    c = mapping.rk4_mapped(p).fock_matrix()
    assert np.max(np.abs(c - b)) < 1e-6 * np.max(np.abs(a))


def test_four_mode_oracles_reduce_to_three_modes():
    """A fourth mode that is idle (no coupling, drive or dissipation) and in its ground state
    in the measured operator leaves Tr(rho0 A(T)) of the first three unchanged, in the number
    basis and in the mapped solve (the four-mode oracle paths against the pinned three-mode
    ones)."""
    from workloads.spec import HTerm
    p3 = configs.random_problem(16, n_modes=3, N=3, n_steps=10, dt=0.01)
    ext = lambda k: tuple(k) + (0,)
    h = [HTerm(t.coef, ext(t.u), ext(t.v), t.channel, t.conj, t.param) for t in p3.h_terms]
    h += [HTerm(0.7 + 0j, (0, 0, 0, 1), (0, 0, 0, 1)), HTerm(-0.3 + 0j, (0, 0, 0, 2), (0, 0, 0, 2))]
    jumps = [type(j)(j.rate, tuple((c, ext(u), ext(v)) for c, u, v in j.terms)) for j in p3.jumps]
    p4 = Problem(**{**p3.__dict__, "n_modes": 4, "N": tuple(p3.N) + (3,), "h_terms": h, "jumps": jumps,
                    "measured": {(ext(k), ext(l)): v for (k, l), v in p3.measured.items()},
                    "rho0": {(ext(k), ext(l)): v for (k, l), v in p3.rho0_items().items()}})
    for solve in (lambda q: fock.rk4_adjoint(q), lambda q: mapping.rk4_mapped(q).fock_matrix()):
        A3, A4 = solve(p3), solve(p4)
        t3 = fock.expectation(A3, fock.operator_matrix(p3.rho0_items(), p3.N))
        t4 = fock.expectation(A4, fock.operator_matrix(p4.rho0_items(), p4.N))
        assert abs(t4 - t3) <= 1e-12 * max(1.0, abs(t3))
