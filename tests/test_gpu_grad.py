"""Adjoint gradients on the GPU (bq_grad and the torch.autograd.Function over it) against
the oracle's discrete adjoint (oracle.grad), central finite differences and each other."""

import copy
import json
import os

import numpy as np
import pytest

from oracle import grad as ograd
from workloads import configs
from workloads.spec import Channel

from parity import gpu_state

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "control_golden.json")


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


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
    p.rho0 = {((0,) * n_modes, (0,) * n_modes): 0.7,
              ((1,) + (0,) * (n_modes - 1), (1,) + (0,) * (n_modes - 1)): 0.3}
    return p


def _flat_oracle(gt, gp):
    return np.concatenate([gt, gp[0].reshape(-1)])


@pytest.mark.parametrize("n_modes,N,ck", [(1, 5, 7), (2, 3, 5), (2, 4, 24)])
def test_grad_matches_oracle_adjoint(n_modes, N, ck):
    p = _small_control(n_modes=n_modes, N=N)
    loss_o, gt, gp = ograd.loss_and_grad(p, checkpoint_every=ck)
    st = gpu_state(p)
    loss, g = st.grad(p.dt, p.n_steps, ck)
    ref = _flat_oracle(gt, gp)
    assert abs(loss[0] - loss_o) <= 1e-12 * max(1.0, abs(loss_o))
    assert np.max(np.abs(g - ref)) <= 1e-10 * np.max(np.abs(ref)), (g, ref)
    assert abs(st.time()) == 0.0  # the state is left as it was


def test_batched_gradients_equal_single_problem_gradients():
    """Three problems with different drives, parameters and measured operators in one state:
    per-problem losses and gradient slots equal those of one problem per state, and the first
    problem's against the oracle."""
    ps = [_small_control(n_modes=2, N=3, seed=s) for s in (3, 4, 5)]
    ps[1].params = [p * 1.1 for p in ps[1].params]
    ps[2].measured = {((0, 1), (0, 1)): 1.0}
    st = gpu_state(ps)
    loss, g = st.grad(ps[0].dt, ps[0].n_steps, 5)
    n_per = g.size // 3
    for b, p in enumerate(ps):
        l1, g1 = gpu_state(p).grad(p.dt, p.n_steps, 5)
        assert abs(loss[b] - l1[0]) <= 1e-13 * max(1.0, abs(l1[0]))
        assert np.max(np.abs(g[b * n_per:(b + 1) * n_per] - g1)) <= 1e-12 * np.max(np.abs(g1))
    loss_o, gt, gp = ograd.loss_and_grad(ps[0], checkpoint_every=5)
    ref = _flat_oracle(gt, gp)
    assert np.max(np.abs(g[:n_per] - ref)) <= 1e-10 * np.max(np.abs(ref))


def _coop_vs_per_stage(p, ck, n_steps=None, **tune):
    n_steps = p.n_steps if n_steps is None else n_steps
    out = []
    for coop in (0, 1):
        st = gpu_state(p)
        st.set_tune(grad_coop=coop, **tune)
        assert st.get_tune()["grad_coop"] == coop
        out.append(st.grad(p.dt, n_steps, ck) + (st,))
    (l0, g0, _), (l1, g1, st) = out
    assert abs(l1[0] - l0[0]) <= 1e-14 * max(1.0, abs(l0[0]))
    assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0))
    assert abs(st.time()) == 0.0
    return l1, g1


@pytest.mark.parametrize("ck", [5, 7, 24])
def test_grad_cooperative_segments_match_per_stage_launches_and_oracle(ck):
    """The cooperative segment kernels (one launch per checkpoint segment and direction, grid
    barriers between the stages) against one launch per stage (equal up to the order of the
    gradient atomics) and against the oracle's adjoint, for even and odd segment lengths."""
    p = _small_control(n_modes=2, N=4, n_seg=4, steps_per_seg=6)
    _, g = _coop_vs_per_stage(p, ck)
    loss_o, gt, gp = ograd.loss_and_grad(p, checkpoint_every=ck)
    ref = _flat_oracle(gt, gp)
    assert np.max(np.abs(g - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("record_segments", [3, -1])
def test_grad_recorded_segments_skip_recomputation(record_segments):
    """A workspace with more recordings: the forward pass records the last segments and the
    backward sweep does not recompute them (-1: all five segments).  Equal to the default
    workspace up to the order of the gradient atomics, and to the oracle."""
    import paper_2203_05526_gb300 as bq
    p = _small_control(n_modes=2, N=4, n_seg=4, steps_per_seg=6)
    l0, g0 = gpu_state(p).grad(p.dt, p.n_steps, 5)
    st = gpu_state(p)
    n0 = bq.launch_count()
    l1, g1 = st.grad(p.dt, p.n_steps, 5, record_segments=record_segments)
    launches = bq.launch_count() - n0
    n_rec = 5 if record_segments < 0 else record_segments
    # cooperative launches: one forward per segment, one recomputation per unrecorded
    # segment, one adjoint per segment, plus evaluation and seeding
    assert launches <= 5 + (5 - n_rec) + 5 + 3, launches
    assert abs(l1[0] - l0[0]) <= 1e-14 * max(1.0, abs(l0[0]))
    assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0))
    loss_o, gt, gp = ograd.loss_and_grad(p, checkpoint_every=5)
    ref = _flat_oracle(gt, gp)
    assert np.max(np.abs(g1 - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert abs(st.time()) == 0.0


def test_grad_cooperative_segments_with_more_items_than_ctas():
    """The full-size two-mode control state with 32-point tiles: more work items per stage
    than resident CTAs, so each CTA takes several items per stage (40 steps, segments of 7)."""
    _coop_vs_per_stage(configs.two_mode_control(), 7, n_steps=40, tile=32)


@pytest.mark.parametrize("n_modes,N,ck", [(1, 5, 7), (2, 3, 5)])
def test_grad_with_secular_dissipator_matches_oracle_adjoint(n_modes, N, ck):
    """The secular dissipator at finite temperature in place of the jump operators: the
    adjoint kernels apply the transposed projector only on diagonal index pairs."""
    from workloads.spec import SecularDamping
    p = _small_control(n_modes=n_modes, N=N)
    p.jumps = []
    p.secular = [SecularDamping(j, 0.6 + 0.2 * j, (0.1, 0.15, 0.2)) for j in range(n_modes)]
    loss_o, gt, gp = ograd.loss_and_grad(p, checkpoint_every=ck)
    st = gpu_state(p)
    loss, g = st.grad(p.dt, p.n_steps, ck)
    ref = _flat_oracle(gt, gp)
    assert abs(loss[0] - loss_o) <= 1e-12 * max(1.0, abs(loss_o))
    assert np.max(np.abs(g - ref)) <= 1e-10 * np.max(np.abs(ref)), (g, ref)


def test_grad_direct_method_matches_finite_differences():
    p = _small_control(n_modes=1, N=5)
    st = gpu_state(p, method="direct")
    loss, g = st.grad(p.dt, p.n_steps, 6)
    h = 1e-6

    def loss_at(q):
        s = gpu_state(q, method="direct")
        s.step(q.dt, q.n_steps)
        return s.evaluate()[0].real

    fd = []
    for i in range(len(p.params)):
        a, b = copy.deepcopy(p), copy.deepcopy(p)
        a.params[i] += h
        b.params[i] -= h
        fd.append((loss_at(a) - loss_at(b)) / (2 * h))
    ch = p.channels[0]
    for j in range(len(ch.params) - 2):
        a, b = copy.deepcopy(p), copy.deepcopy(p)
        pa, pb = list(ch.params), list(ch.params)
        pa[2 + j] += h
        pb[2 + j] -= h
        a.channels = [Channel("pwc", tuple(pa))]
        b.channels = [Channel("pwc", tuple(pb))]
        fd.append((loss_at(a) - loss_at(b)) / (2 * h))
    fd = np.array(fd)
    err = float(np.max(np.abs(g - fd)) / np.max(np.abs(fd)))
    print("direct adjoint", g.tolist(), "fd", fd.tolist(), "rel err", err)
    assert err <= 1e-7


@pytest.mark.parametrize("n_modes,N,ck,secular", [(1, 5, 6, False), (2, 3, 5, False), (1, 5, 4, True)])
def test_grad_direct_method_matches_oracle_adjoint(n_modes, N, ck, secular):
    """The number-basis method's gradient on the GPU against the oracle's discrete adjoint of
    its own number-basis solve (oracle.grad.loss_and_grad_direct), element by element."""
    from workloads.spec import SecularDamping
    p = _small_control(n_modes=n_modes, N=N)
    if secular:
        p.jumps = []
        p.secular = [SecularDamping(0, 0.6, (0.1, 0.15, 0.2))]
    loss_o, gt, gp = ograd.loss_and_grad_direct(p, checkpoint_every=ck)
    st = gpu_state(p, method="direct")
    loss, g = st.grad(p.dt, p.n_steps, ck)
    ref = _flat_oracle(gt, gp)
    assert abs(loss[0] - loss_o) <= 1e-12 * max(1.0, abs(loss_o))
    err = float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))
    assert err <= 1e-10, (err, g, ref)


def test_checkpoint_interval_and_autograd():
    import torch
    from paper_2203_05526_gb300.autograd import measured_probability
    p = _small_control(n_modes=2, N=3)
    st = gpu_state(p)
    _, g1 = st.grad(p.dt, p.n_steps, 1)
    _, g2 = st.grad(p.dt, p.n_steps, 1000)
    assert np.max(np.abs(g1 - g2)) <= 1e-13 * np.max(np.abs(g1))
    theta = torch.tensor(p.params, dtype=torch.float64, requires_grad=True)
    ch = p.channels[0]
    pwc = torch.tensor(np.array(ch.params[2:]).reshape(-1, 2), dtype=torch.float64, requires_grad=True)
    l = measured_probability(p, theta, pwc, checkpoint_every=5)
    l.backward()
    P = len(p.params)
    assert np.max(np.abs(theta.grad.numpy() - g1[:P])) <= 1e-13 * np.max(np.abs(g1))
    assert np.max(np.abs(pwc.grad.numpy().reshape(-1) - g1[P:])) <= 1e-13 * np.max(np.abs(g1))


def test_control_problem_full_size():
    """Two-mode control problem at full size: 64 segments, 20 480 steps, checkpoint every 160
    steps; against the oracle's adjoint (golden file) and central differences (h = 1e-6) on
    sampled parameters."""
    p = configs.two_mode_control()
    st = gpu_state(p)
    loss, g = st.grad(p.dt, p.n_steps, 160)
    assert np.all(np.isfinite(g)) and g.shape == (3 + 128,)
    if os.path.exists(GOLDEN):
        gold = json.load(open(GOLDEN))
        ref = np.concatenate([gold["grad_theta"], np.array(gold["grad_pwc"]).reshape(-1)])
        assert abs(loss[0] - gold["loss"]) <= 1e-10 * max(1.0, abs(gold["loss"]))
        assert np.max(np.abs(g - ref)) <= 1e-8 * np.max(np.abs(ref))
    h = 1e-6

    def loss_at(q):
        s = gpu_state(q)
        s.step(q.dt, q.n_steps)
        return s.evaluate()[0].real

    for i in (0, 2):  # K_1 and g
        a, b = copy.deepcopy(p), copy.deepcopy(p)
        a.params[i] += h
        b.params[i] -= h
        fd = (loss_at(a) - loss_at(b)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g)))
    ch = p.channels[0]
    for j in (0, 77):  # Re of segment 0, Im of segment 38
        a, b = copy.deepcopy(p), copy.deepcopy(p)
        pa, pb = list(ch.params), list(ch.params)
        pa[2 + j] += h
        pb[2 + j] -= h
        a.channels = [Channel("pwc", tuple(pa))]
        b.channels = [Channel("pwc", tuple(pb))]
        fd = (loss_at(a) - loss_at(b)) / (2 * h)
        assert abs(g[3 + j] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g)))
