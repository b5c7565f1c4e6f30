"""Pins for O3 (discrete adjoint of the mapped RK4 solve) against central finite
differences of the oracle's forward solve (oracle.mapping)."""

import copy

import numpy as np
import pytest

from oracle import grad
from workloads import configs
from workloads.spec import Channel, HTerm, Problem


def _small_control(n_modes=1, N=5, n_seg=4, steps_per_seg=6, seed=3):
    rng = np.random.default_rng(seed)
    if n_modes == 1:
        p = configs.kerr_driven(N=N, dt=0.01, T=0.24, n_th=0.1)
        p.h_terms = (configs.kerr_mode_terms(1, 0, 0.0, 0.0, delta_param=0, kerr_param=1)
                     + configs.gauss_drive_terms(1, 0, 0))
        p.params = [0.3, -1.1]
        p.measured = {((1,), (1,)): 1.0, ((0,), (1,)): 0.3 + 0.2j, ((1,), (0,)): 0.3 - 0.2j}
    else:
        p = configs.two_mode_control(n_seg=n_seg, T=0.24, steps_per_seg=steps_per_seg, N=N)
    seg_len = p.T / n_seg
    vals = []
    for _ in range(n_seg):
        vals += [float(rng.normal(0, 0.5)), float(rng.normal(0, 0.5))]
    p.channels = [Channel("pwc", (0.0, seg_len, *vals))]
    p.dt = seg_len / steps_per_seg
    p.rho0 = {((0,) * n_modes, (0,) * n_modes): 0.7, ((1,) + (0,) * (n_modes - 1), (1,) + (0,) * (n_modes - 1)): 0.3}
    return p


def _fd(p, h=1e-6, r_layout="full"):
    loss = lambda q: grad.loss_only(q, r_layout=r_layout)
    gt = []
    for i in range(len(p.params)):
        a, b = copy.deepcopy(p), copy.deepcopy(p)
        a.params[i] += h
        b.params[i] -= h
        gt.append((loss(a) - loss(b)) / (2 * h))
    ch = p.channels[0]
    n_seg = (len(ch.params) - 2) // 2
    gp = np.zeros((n_seg, 2))
    for s in range(n_seg):
        for r in range(2):
            a, b = copy.deepcopy(p), copy.deepcopy(p)
            pa, pb = list(ch.params), list(ch.params)
            pa[2 + 2 * s + r] += h
            pb[2 + 2 * s + r] -= h
            a.channels = [Channel("pwc", tuple(pa))]
            b.channels = [Channel("pwc", tuple(pb))]
            gp[s, r] = (loss(a) - loss(b)) / (2 * h)
    return np.array(gt), gp


@pytest.mark.parametrize("n_modes,N,ck", [(1, 5, 7), (2, 3, 5)])
def test_adjoint_matches_central_differences(n_modes, N, ck):
    p = _small_control(n_modes=n_modes, N=N)
    loss, gt, gp = grad.loss_and_grad(p, checkpoint_every=ck)
    assert abs(loss - grad.loss_only(p)) < 1e-13
    ft, fp = _fd(p)
    scale = max(np.max(np.abs(ft)), np.max(np.abs(fp)))
    assert np.max(np.abs(gt - ft)) < 1e-7 * scale, (gt, ft)
    assert np.max(np.abs(gp[0] - fp)) < 1e-7 * scale, (gp[0], fp)


def test_checkpoint_interval_does_not_change_gradient():
    p = _small_control()
    a = grad.loss_and_grad(p, checkpoint_every=1)
    b = grad.loss_and_grad(p, checkpoint_every=100)
    assert np.max(np.abs(a[1] - b[1])) < 1e-14
    assert np.max(np.abs(a[2][0] - b[2][0])) < 1e-14


@pytest.mark.parametrize("n_modes,N", [(1, 5), (2, 3)])
def test_adjoint_with_secular_dissipator_matches_central_differences(n_modes, N):
    """The secular dissipator (Eq. 203 / Eq. S9 at finite temperature) in place of the jump
    operators: the transposed projector P^T on b_R and on the separable source."""
    from workloads.spec import SecularDamping
    p = _small_control(n_modes=n_modes, N=N)
    p.jumps = []
    p.secular = [SecularDamping(j, 0.6 + 0.2 * j, (0.1, 0.15, 0.2)) for j in range(n_modes)]
    p.measured = ({((1,), (1,)): 1.0, ((0,), (1,)): 0.3 + 0.2j, ((1,), (0,)): 0.3 - 0.2j} if n_modes == 1 else
                  {((1, 0), (1, 0)): 1.0, ((0, 1), (1, 0)): 0.4 + 0.1j, ((1, 0), (0, 1)): 0.4 - 0.1j})
    loss, gt, gp = grad.loss_and_grad(p, checkpoint_every=5)
    assert abs(loss - grad.loss_only(p)) < 1e-13
    ft, fp = _fd(p)
    scale = max(np.max(np.abs(ft)), np.max(np.abs(fp)))
    assert np.max(np.abs(gt - ft)) < 1e-7 * scale, (gt, ft)
    assert np.max(np.abs(gp[0] - fp)) < 1e-7 * scale, (gp[0], fp)


@pytest.mark.parametrize("n_modes,N", [(1, 5), (2, 3)])
def test_adjoint_with_diagonal_residual_layout_matches_central_differences(n_modes, N):
    """R kept only on k = l (the R(xy) layout) with the secular dissipator: the adjoint of
    the projected system (D on b_R, on the R part of J^T and on the final cotangent) against
    central differences of the same projected forward solve; the loss differs from the full
    layout's (the projection is an approximation), the gradient machinery must not."""
    from workloads.spec import SecularDamping
    p = _small_control(n_modes=n_modes, N=N)
    p.jumps = []
    p.secular = [SecularDamping(j, 0.6 + 0.2 * j, (0.1, 0.15, 0.2)) for j in range(n_modes)]
    p.measured = ({((1,), (1,)): 1.0, ((2,), (2,)): -0.4, ((0,), (1,)): 0.3 + 0.2j, ((1,), (0,)): 0.3 - 0.2j}
                  if n_modes == 1 else
                  {((1, 0), (1, 0)): 1.0, ((0, 1), (0, 1)): 0.5, ((0, 1), (1, 0)): 0.4 + 0.1j,
                   ((1, 0), (0, 1)): 0.4 - 0.1j})
    loss, gt, gp = grad.loss_and_grad(p, checkpoint_every=5, r_layout="diag")
    assert abs(loss - grad.loss_only(p, r_layout="diag")) < 1e-13
    assert abs(loss - grad.loss_only(p)) > 1e-9  # the layouts differ
    ft, fp = _fd(p, r_layout="diag")
    scale = max(np.max(np.abs(ft)), np.max(np.abs(fp)))
    assert np.max(np.abs(gt - ft)) < 1e-7 * scale, (gt, ft)
    assert np.max(np.abs(gp[0] - fp)) < 1e-7 * scale, (gp[0], fp)
    full = grad.loss_and_grad(p, checkpoint_every=5)
    assert np.max(np.abs(full[1] - gt)) > 1e-9 * scale  # a dropped projection would not show here otherwise


def _fd_direct(p, h=1e-6):
    loss = grad.loss_only_direct
    gt = []
    for i in range(len(p.params)):
        a, b = copy.deepcopy(p), copy.deepcopy(p)
        a.params[i] += h
        b.params[i] -= h
        gt.append((loss(a) - loss(b)) / (2 * h))
    ch = p.channels[0]
    n_seg = (len(ch.params) - 2) // 2
    gp = np.zeros((n_seg, 2))
    for s in range(n_seg):
        for r in range(2):
            a, b = copy.deepcopy(p), copy.deepcopy(p)
            pa, pb = list(ch.params), list(ch.params)
            pa[2 + 2 * s + r] += h
            pb[2 + 2 * s + r] -= h
            a.channels = [Channel("pwc", tuple(pa))]
            b.channels = [Channel("pwc", tuple(pb))]
            gp[s, r] = (loss(a) - loss(b)) / (2 * h)
    return np.array(gt), gp


@pytest.mark.parametrize("n_modes,N,ck,secular", [(1, 5, 7, False), (2, 3, 5, False), (1, 5, 4, True)])
def test_direct_adjoint_matches_central_differences(n_modes, N, ck, secular):
    """The discrete adjoint of the number-basis RK4 solve (O1) against central differences
    of O1 itself: thermal jump operators (a and a^dag), H-term parameters (Delta, K; on two
    modes K_1, K_2, g) and complex piecewise-constant segments, or the secular dissipator."""
    from workloads.spec import SecularDamping
    p = _small_control(n_modes=n_modes, N=N)
    if secular:
        p.jumps = []
        p.secular = [SecularDamping(0, 0.6, (0.1, 0.15, 0.2))]
    loss, gt, gp = grad.loss_and_grad_direct(p, checkpoint_every=ck)
    assert abs(loss - grad.loss_only_direct(p)) < 1e-13
    ft, fp = _fd_direct(p)
    scale = max(np.max(np.abs(ft)), np.max(np.abs(fp)))
    assert scale > 1e-3
    assert np.max(np.abs(gt - ft)) < 1e-7 * scale, (gt, ft)
    assert np.max(np.abs(gp[0] - fp)) < 1e-7 * scale, (gp[0], fp)


def test_direct_adjoint_checkpoint_interval_and_transpose():
    """Checkpoint intervals change nothing; the transposed generator satisfies
    <B, F(A)> = <F^T(B), A> for random A, B (the identity the pull-back relies on)."""
    from oracle import fock
    p = _small_control(n_modes=2, N=3)
    a = grad.loss_and_grad_direct(p, checkpoint_every=1)
    b = grad.loss_and_grad_direct(p, checkpoint_every=1000)
    assert np.max(np.abs(a[1] - b[1])) < 1e-14
    assert np.max(np.abs(a[2][0] - b[2][0])) < 1e-14
    model = fock.FockModel(p)
    rng = np.random.default_rng(1)
    d = model.dim
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    B = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    H = model.hamiltonian(0.05, 0.5, p.dt)
    lhs = np.sum(B * model.adjoint_generator(A, H))
    rhs = np.sum(grad._direct_transpose(model, B, H) * A)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
