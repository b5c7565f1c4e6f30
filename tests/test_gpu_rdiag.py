"""The diagonal residual layout (R kept only at k = l, a function of the products x_j y_j)
on the GPU against the oracle's projection of Eq. 303c onto the same entries."""

import math

import numpy as np
import pytest

import paper_2203_05526_gb300 as bq
from paper_2203_05526_gb300.binding import BQ_EINVAL, BQ_EUNSUPPORTED
from oracle import fock, mapping
from workloads import configs

from parity import compare_mapped_systems, gpu_state, rel_err

pytestmark = pytest.mark.gpu
TWO_PI = 2.0 * math.pi
TOL64, TOL32 = 1e-10, 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _sync():
    import torch
    torch.cuda.synchronize()


def _driven_secular(N=9, T=0.8, dt=0.005):
    meas = {((1,), (2,)): 0.4 + 0.1j, ((2,), (1,)): 0.4 - 0.1j, ((3,), (3,)): 1.0, ((0,), (0,)): 0.2}
    return configs.kerr_secular(N=N, T=T, dt=dt, kappa=0.4, kT=TWO_PI * 1.64, measured=meas,
                                drive_peak=TWO_PI * 0.3)


@pytest.mark.parametrize("dtype,tol", [("f64", TOL64), ("f32", TOL32)])
def test_single_mode_diag_layout_matches_oracle(dtype, tol):
    p = _driven_secular(N=12 if dtype == "f32" else 9)
    st = gpu_state(p, dtype=dtype, r_layout="diag")
    assert st.stage_variant() == "generic" and not st.solve_eligible()
    st.step(p.dt, p.n_steps)
    _sync()
    run = mapping.rk4_mapped(p, r_layout="diag")
    compare_mapped_systems(st, run, tol)
    # Tr(rho0 A) and the three-level block from the k = l entries
    A = run.fock_matrix()
    blk = st.fock_block(3, dim=3)[0]
    assert rel_err(blk, A[:3, :3]) <= tol
    ev = st.evaluate()[0]
    assert abs(ev - A[0, 0]) <= tol * max(1.0, abs(A[0, 0]))


def test_two_coupled_modes_diag_layout_matches_oracle():
    p = configs.two_mode(N=4, T=0.4, dt=0.01)
    p.channels = [configs.Channel("gauss", (TWO_PI * 0.2, 0.0, 0.2, 0.05))]
    p.h_terms = p.h_terms + configs.gauss_drive_terms(2, 0, 0)
    p.jumps = configs.damping_jumps(2, 0, 0.3, 0.1) + configs.damping_jumps(2, 1, 0.2, 0.0)
    p.measured = {((1, 0), (0, 1)): 1.0 + 0.5j, ((0, 1), (1, 0)): 1.0 - 0.5j, ((1, 1), (1, 1)): 0.3}
    st = gpu_state(p, r_layout="diag")
    st.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, mapping.rk4_mapped(p, r_layout="diag"), TOL64)


def test_diag_layout_is_exact_when_dynamics_keep_diagonality_and_stores_less():
    meas = {((1,), (1,)): 1.0, ((3,), (3,)): -0.4}
    p = configs.kerr_secular(N=10, T=0.5, dt=0.005, kappa=0.3, kT=TWO_PI * 1.64, measured=meas, drive_peak=0.0)
    full = gpu_state(p)
    diag = gpu_state(p, r_layout="diag")
    full.step(p.dt, p.n_steps)
    diag.step(p.dt, p.n_steps)
    _sync()
    for s in range(full.n_systems()):
        for x, y in zip(diag.read_system(s)[1:], full.read_system(s)[1:]):
            assert rel_err(x, y) <= 1e-13
    pad4 = lambda n: (n + 3) // 4 * 4  # every array of a system starts on a 4-element boundary
    n_sys, cs = full.n_systems(), 16
    assert diag.state_bytes() == n_sys * 3 * pad4(10) * cs          # G_x, G_y and the k = l entries
    assert full.state_bytes() == n_sys * (2 * pad4(10) + pad4(100)) * cs


def test_diag_layout_refusals():
    p = _driven_secular()
    with pytest.raises(bq.BQError) as e:
        gpu_state(p, method="direct", r_layout="diag")
    assert e.value.args[0].startswith(f"bq status {BQ_EINVAL}")


@pytest.mark.parametrize("n_modes", [1, 2])
def test_diag_layout_gradients_match_oracle_adjoint(n_modes):
    """Adjoint gradients of the projected (R(xy)) system: loss and gradients with respect to
    the H parameters and the piecewise-constant drive segments against the oracle's adjoint
    of the same layout."""
    from oracle import grad as ograd
    from workloads.spec import Channel, SecularDamping
    rng = np.random.default_rng(5)
    if n_modes == 1:
        p = configs.kerr_driven(N=6, dt=0.01, T=0.24, n_th=0.0)
        p.h_terms = (configs.kerr_mode_terms(1, 0, 0.0, 0.0, delta_param=0, kerr_param=1)
                     + configs.gauss_drive_terms(1, 0, 0))
        p.params = [0.3, -1.1]
        p.measured = {((1,), (1,)): 1.0, ((2,), (2,)): -0.4, ((0,), (1,)): 0.3 + 0.2j, ((1,), (0,)): 0.3 - 0.2j}
        p.rho0 = {((0,), (0,)): 0.5, ((1,), (1,)): 0.3, ((2,), (2,)): 0.2}
    else:
        p = configs.two_mode_control(n_seg=4, T=0.24, steps_per_seg=6, N=4)
        p.measured = {((1, 0), (1, 0)): 1.0, ((0, 1), (0, 1)): 0.5, ((0, 1), (1, 0)): 0.4 + 0.1j,
                      ((1, 0), (0, 1)): 0.4 - 0.1j}
        p.rho0 = {((0, 0), (0, 0)): 0.4, ((1, 0), (1, 0)): 0.3, ((0, 1), (0, 1)): 0.3}
    p.jumps = []
    p.secular = [SecularDamping(j, 0.6 + 0.2 * j, (0.1, 0.15, 0.2)) for j in range(n_modes)]
    n_seg = 4
    seg_len = p.T / n_seg
    vals = []
    for _ in range(n_seg):
        vals += [float(rng.normal(0, 0.5)), float(rng.normal(0, 0.5))]
    p.channels = [Channel("pwc", (0.0, seg_len, *vals))]
    p.dt = seg_len / 6
    loss_o, gt, gp = ograd.loss_and_grad(p, checkpoint_every=5, r_layout="diag")
    ref = np.concatenate([gt, gp[0].reshape(-1)])
    st = gpu_state(p, r_layout="diag")
    loss, g = st.grad(p.dt, p.n_steps, 5)
    assert abs(loss[0] - loss_o) <= 1e-12 * max(1.0, abs(loss_o))
    assert np.max(np.abs(g - ref)) <= 1e-10 * np.max(np.abs(ref)), (g, ref)
