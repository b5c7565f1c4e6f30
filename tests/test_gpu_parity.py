"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: 1e-10 relative in FP64, 1e-5 in FP32 (relative to the largest
element of the compared array or block)."""

import json
import math
import os

import numpy as np
import pytest

import paper_2203_05526_gb300 as bq

from oracle import fock, mapping
from workloads import configs
from workloads.spec import Problem

from parity import FLOOR64, compare_mapped_systems, gpu_state, rel_err, scalar_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5
TWO_MODE_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "two_mode_golden.json")

SMALL = [  # (seed, n_modes, N, steps): several tiles only for 2-3 modes, ragged sizes
    (101, 1, 7, 30),
    (102, 1, 13, 25),
    (103, 2, 4, 20),
    (104, 2, 5, 12),
    (105, 3, 3, 10),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("seed,nm,N,steps", SMALL)
@pytest.mark.parametrize("dense", [False, True])
def test_mapped_f64_state_matches_oracle(seed, nm, N, steps, dense):
    p = configs.random_problem(seed, n_modes=nm, N=N, n_steps=steps, dt=0.01, dense_measured=dense)
    st = gpu_state(p)
    st.step(p.dt, steps)
    _sync()
    run = mapping.rk4_mapped(p)
    compare_mapped_systems(st, run, TOL64)
    # observables: Tr(rho0 A) and the three-level block
    A = run.fock_matrix()
    tr = st.evaluate()[0]
    ref = A[0, 0]
    assert scalar_err(tr, ref, FLOOR64) <= TOL64, (tr, ref)
    D = int(np.prod([min(3, n) for n in p.N]))
    blk = st.fock_block(3, dim=D)[0]
    assert rel_err(blk, fock.low_block(A, p.N)) <= TOL64


@pytest.mark.parametrize("seed,nm,N,steps", SMALL)
def test_direct_f64_matches_oracle(seed, nm, N, steps):
    p = configs.random_problem(seed, n_modes=nm, N=N, n_steps=steps, dt=0.01, dense_measured=True)
    st = gpu_state(p, method="direct")
    st.step(p.dt, steps)
    _sync()
    A = fock.rk4_adjoint(p)
    info, _, _, r = st.read_system(0)
    assert rel_err(r, A.reshape(-1)) <= TOL64
    assert scalar_err(st.evaluate()[0], A[0, 0], FLOOR64) <= TOL64


def test_mapped_all_in_r_equals_direct_on_gpu():
    """Both GPU methods integrate the same generator; with M = N they agree to RK4 error."""
    p = configs.random_problem(111, n_modes=1, N=8, n_steps=40, dt=0.005, dense_measured=True)
    a = gpu_state(p)
    b = gpu_state(p, method="direct")
    a.step(p.dt, 40)
    b.step(p.dt, 40)
    _sync()
    D = 3
    assert rel_err(a.fock_block(3, dim=D), b.fock_block(3, dim=D)) < 1e-6


@pytest.mark.parametrize("seed,nm,N,steps", SMALL[:3])
def test_mapped_f32_matches_oracle(seed, nm, N, steps):
    p = configs.random_problem(seed, n_modes=nm, N=N, n_steps=steps, dt=0.01, dense_measured=True)
    st = gpu_state(p, dtype="f32")
    st.step(p.dt, steps)
    _sync()
    run = mapping.rk4_mapped(p)
    A = run.fock_matrix()
    D = int(np.prod([min(3, n) for n in p.N]))
    assert rel_err(st.fock_block(3, dim=D)[0], fock.low_block(A, p.N)) <= TOL32
    compare_mapped_systems(st, run, 1e-4)


def test_r_layout_off_and_zero_c():
    p = configs.random_problem(121, n_modes=1, N=6, n_steps=20, dt=0.01)
    for r_layout, c_mode in (("off", "eq304"), ("full", "zero")):
        st = gpu_state(p, r_layout=r_layout, c_mode=c_mode)
        st.step(p.dt, 20)
        _sync()
        run = mapping.rk4_mapped(p, r_layout=r_layout, C_override=0.0 if c_mode == "zero" else None)
        compare_mapped_systems(st, run, TOL64)


def test_graph_path_and_split_calls():
    """130 steps in one call (two CUDA-graph replays + 2 direct steps) equal 3 + 127 steps in
    two calls and the oracle: the device step counter and tau bookkeeping are exact."""
    p = configs.random_problem(131, n_modes=1, N=6, n_steps=130, dt=0.005)
    a = gpu_state(p)
    a.step(p.dt, 130)
    b = gpu_state(p)
    b.step(p.dt, 3)
    b.step(p.dt, 127)
    _sync()
    run = mapping.rk4_mapped(p)
    compare_mapped_systems(a, run, TOL64)
    compare_mapped_systems(b, run, TOL64)
    assert abs(a.time() - 130 * 0.005) < 1e-12


def test_kerr_static_full_horizon():
    """The single damped Kerr oscillator, |1><1|, 10 000 steps of 0.01 ns: mapped (M = 3) and
    direct (N = 16) against O2 / O1, and the binomial closed form."""
    p = configs.kerr_static(N=16)
    st = gpu_state(p, grid=[3])
    st.step(p.dt, p.n_steps)
    d = gpu_state(p, method="direct")
    d.step(p.dt, p.n_steps)
    _sync()
    run = mapping.rk4_mapped(p, M=(3,))
    compare_mapped_systems(st, run, TOL64)
    A = fock.rk4_adjoint(p)
    _, _, _, r = d.read_system(0)
    assert rel_err(r, A.reshape(-1)) <= TOL64
    gt = 1e-3 * p.T
    blk = st.fock_block(3, dim=3)[0]
    for k in range(3):
        ref = math.comb(k, 1) * math.exp(-gt) * (1 - math.exp(-gt)) ** (k - 1) if k >= 1 else 0.0
        assert abs(blk[k, k] - ref) < 1e-12


@pytest.mark.parametrize("dtype,tol", [("f64", TOL64), ("f32", TOL32)])
def test_kerr_driven_full_horizon(dtype, tol):
    """Finite temperature + resonant Gaussian drive, N = 40 oracle, grid M = 12, 40 000 steps."""
    p = configs.kerr_driven(N=40)
    st = gpu_state(p, grid=[12], dtype=dtype)
    st.step(p.dt, p.n_steps)
    _sync()
    run = mapping.rk4_mapped(p, M=(12,))
    A = run.fock_matrix()
    blk = st.fock_block(3, dim=3)[0]
    assert rel_err(blk, A[:3, :3]) <= tol
    if dtype == "f64":
        compare_mapped_systems(st, run, TOL64)


def test_two_mode_multi_tile_matches_oracle():
    """Two coupled modes at the full grid M = 12 (R = 20 736 points, several shared-memory tiles
    with halo windows per system): 300 steps against O2 and, in FP64, the direct method
    against O1."""
    p = configs.two_mode(N=12, T=3.0, dt=0.01)
    st = gpu_state(p)
    st.step(p.dt, p.n_steps)
    d = gpu_state(p, method="direct")
    d.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, mapping.rk4_mapped(p), TOL64)
    _, _, _, r = d.read_system(0)
    A = fock.rk4_adjoint(p)
    assert rel_err(r, A.reshape(-1)) <= TOL64


def test_three_modes_with_halo_beyond_shared_memory():
    """Three coupled modes at N = 6: the stencil's outermost stride (6^5 points) does not fit
    beside a tile in shared memory, so the stage kernel reads R from global memory; direct
    and mapped methods against O1 / O2."""
    p = configs.table_one_network(3, 6, steps=4000)
    p = Problem(**{**p.__dict__, "T": 10 * p.dt,  # the first 10 steps, two initial conditions
                   "measured": {((1, 0, 1), (0, 1, 1)): 1.0 + 0.3j, ((0, 1, 1), (1, 0, 1)): 1.0 - 0.3j}})
    d = gpu_state(p, method="direct")
    d.step(p.dt, p.n_steps)
    _sync()
    A = fock.rk4_adjoint(p)
    _, _, _, r = d.read_system(0)
    assert rel_err(r, A.reshape(-1)) <= TOL64
    m = gpu_state(p)
    m.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(m, mapping.rk4_mapped(p), TOL64)


def test_three_modes_global_read_gradients_match_oracle_adjoint():
    """Adjoint gradients of a three-mode network whose halo (5^5 points) exceeds a
    shared-memory tile, so the forward and adjoint stage kernels read R and its cotangent from
    global memory: loss and dl/dJ (the exchange coupling as a parameter) against the oracle's
    discrete adjoint."""
    from oracle import grad as ograd
    from workloads.spec import HTerm
    p = configs.table_one_network(3, 5, steps=4000)
    J = configs.TABLE_ONE["J"]
    h = [HTerm(1.0 + 0j, t.u, t.v, param=0) if (t.coef == J and t.u != t.v and sum(t.u) == 1 and sum(t.v) == 1)
         else t for t in p.h_terms]
    p = Problem(**{**p.__dict__, "h_terms": h, "params": [J], "T": 12 * p.dt,
                   "rho0": {((0, 1, 1), (1, 0, 1)): 0.4, ((1, 0, 1), (0, 1, 1)): 0.4,
                            ((1, 0, 1), (1, 0, 1)): 0.5, ((0, 1, 1), (0, 1, 1)): 0.5},
                   "measured": {((1, 0, 1), (0, 1, 1)): 1.0 + 0.3j, ((0, 1, 1), (1, 0, 1)): 1.0 - 0.3j}})
    loss_o, gt, _ = ograd.loss_and_grad(p, checkpoint_every=4)
    st = gpu_state(p)
    loss, g = st.grad(p.dt, p.n_steps, 4)
    assert abs(loss[0] - loss_o) <= 1e-12 * max(1.0, abs(loss_o))
    assert abs(g[0] - gt[0]) <= 1e-10 * abs(gt[0]), (g, gt)


@pytest.mark.parametrize("n_modes,N", [(2, 5), (3, 4)])
def test_separable_only_layout_matches_oracle(n_modes, N):
    """R = 0 (the separated equations alone): the few systems of one Table I network are
    split into chunks of [G_x | G_y] (default and tuned chunk lengths, one CTA per system
    for long chunks), against the oracle's run of the same layout."""
    p = configs.table_one_network(n_modes, N, steps=400)
    p = Problem(**{**p.__dict__, "T": 20 * p.dt})
    run = mapping.rk4_mapped(p, r_layout="off")
    for tile in (0, 32, 4096):
        st = gpu_state(p, r_layout="off")
        st.set_tune(tile=tile)
        st.step(p.dt, p.n_steps)
        _sync()
        compare_mapped_systems(st, run, TOL64)


def _with_idle_fourth_mode(p3: Problem) -> Problem:
    """The three-mode problem with a fourth mode that is neither coupled, driven nor damped
    (omega_q a^dag a + eta a^dag^2 a^2 only), in its ground state in rho0 and measured as
    |0><0|: A(t) = A_3(t) (x) |0><0| exactly, so the four-mode run reduces to the three-mode
    one (Tr(rho0 A) and gradients equal)."""
    from workloads.spec import HTerm, SecularDamping
    ext = lambda k: tuple(k) + (0,)
    tq = configs.TABLE_ONE
    h = [HTerm(t.coef, ext(t.u), ext(t.v), t.channel, t.conj, t.param) for t in p3.h_terms]
    h += [HTerm(tq["omega_q"] + 0j, (0, 0, 0, 1), (0, 0, 0, 1)), HTerm(tq["eta"] + 0j, (0, 0, 0, 2), (0, 0, 0, 2))]
    return Problem(**{**p3.__dict__, "n_modes": 4, "N": tuple(p3.N) + (3,), "h_terms": h,
                      "secular": [SecularDamping(s.mode, s.kappa, s.nbar) for s in p3.secular],
                      "measured": {(ext(k), ext(l)): v for (k, l), v in p3.measured.items()},
                      "rho0": {(ext(k), ext(l)): v for (k, l), v in p3.rho0_items().items()}})


def test_four_modes_reduce_to_three_modes():
    """Four modes (the limit of the library): direct and mapped runs and the mapped adjoint
    gradient of a network whose fourth mode is idle in its ground state, against the oracle's
    three-mode results (Tr(rho0 A(T)), dl/dJ)."""
    from oracle import grad as ograd
    from workloads.spec import HTerm
    p = configs.table_one_network(3, 3, steps=4000)
    J = configs.TABLE_ONE["J"]
    h = [HTerm(1.0 + 0j, t.u, t.v, param=0) if (t.coef == J and t.u != t.v and sum(t.u) == 1 and sum(t.v) == 1)
         else t for t in p.h_terms]
    p3 = Problem(**{**p.__dict__, "h_terms": h, "params": [J], "T": 12 * p.dt,
                    "rho0": {((0, 1, 1), (1, 0, 1)): 0.4, ((1, 0, 1), (0, 1, 1)): 0.4,
                             ((1, 0, 1), (1, 0, 1)): 0.5, ((0, 1, 1), (0, 1, 1)): 0.5},
                    "measured": {((1, 0, 1), (0, 1, 1)): 1.0 + 0.3j, ((0, 1, 1), (1, 0, 1)): 1.0 - 0.3j,
                                 ((1, 1, 0), (1, 1, 0)): 0.5}})
    p4 = _with_idle_fourth_mode(p3)
    A3 = fock.rk4_adjoint(p3)
    ref = fock.expectation(A3, fock.operator_matrix(p3.rho0_items(), p3.N))
    for method in ("direct", "mapped"):
        st = gpu_state(p4, method=method)
        st.step(p4.dt, p4.n_steps)
        _sync()
        ev = st.evaluate()[0]
        assert abs(ev - ref) <= TOL64 * max(1.0, abs(ref)), (method, ev, ref)
    loss_o, gt, _ = ograd.loss_and_grad(p3, checkpoint_every=4)
    loss, g = gpu_state(p4).grad(p4.dt, p4.n_steps, 4)
    assert abs(loss[0] - loss_o) <= 1e-12 * max(1.0, abs(loss_o))
    assert abs(g[0] - gt[0]) <= 1e-10 * abs(gt[0]), (g, gt)


def _cplx(pair):
    return np.array(pair[0]) + 1j * np.array(pair[1])


@pytest.mark.parametrize("method", ["mapped", "direct"])
def test_two_mode_full_horizon_matches_oracle_golden(method):
    """Two exchange-coupled Kerr modes (Eq. 301 network: M = 12 per mode, R = 20 736 points)
    over the full 100 ns, 10 000 RK4 steps in FP64, against the oracle's values written by
    tests/golden/make_two_mode_golden.py: the 9 x 9 low block (the paper's epsilon_r block),
    Tr(rho0 A) and 256 seeded elements of the operator (mapped: also G_x and G_y whole and 256
    elements of R), element by element at 1e-10."""
    g = json.load(open(TWO_MODE_GOLDEN))[method]
    p = configs.two_mode()
    st = gpu_state(p, method=method)
    st.step(p.dt, p.n_steps)
    _sync()
    ref_blk = _cplx(g["block"])
    blk = st.fock_block(3, dim=9)[0]
    assert rel_err(blk, ref_blk) <= TOL64
    assert fock.eps_r(blk, ref_blk) <= TOL64
    assert scalar_err(st.evaluate()[0], complex(*g["tr_rho0_A"]), FLOOR64) <= TOL64
    info, gx, gy, r = st.read_system(0)
    if method == "direct":
        ref = _cplx(g["values"])
        assert rel_err(r[g["positions"]], ref) <= TOL64
    else:
        assert abs(info["weight"] - complex(*g["weight"])) <= 1e-12 * abs(complex(*g["weight"]))
        assert abs(info["C"] - complex(*g["C"])) <= 1e-12 * max(1.0, abs(complex(*g["C"])))
        rgx, rgy, rr = _cplx(g["gx"]), _cplx(g["gy"]), _cplx(g["r_values"])
        scale = max(np.max(np.abs(rgx)), np.max(np.abs(rgy)))
        assert rel_err(gx, rgx, floor=scale) <= TOL64
        assert rel_err(gy, rgy, floor=scale) <= TOL64
        assert rel_err(r[g["r_positions"]], rr) <= TOL64
