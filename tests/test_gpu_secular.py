"""The secular dissipator (Eq. 203 / Eq. S9) on the GPU: the diagonal-restricted projector
term in every stage kernel that runs it (pipelined, one CTA per system, tiled) against the
oracles, element by element."""

import math

import numpy as np
import pytest

from oracle import fock, mapping
from workloads import configs

from parity import compare_mapped_systems, gpu_state, rel_err

pytestmark = pytest.mark.gpu
TWO_PI = 2.0 * math.pi
TOL64, TOL32 = 1e-10, 1e-5
KT = TWO_PI * 1.64  # nbar_0 ~ 0.05 at 5 GHz


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _sync():
    import torch
    torch.cuda.synchronize()


def _single(N=9, T=0.6, dt=0.005, kT=KT, dense=True, drive=TWO_PI * 0.3):
    meas = ({((1,), (2,)): 0.4 + 0.1j, ((2,), (1,)): 0.4 - 0.1j, ((3,), (3,)): 1.0, ((0,), (0,)): 0.2}
            if dense else None)
    return configs.kerr_secular(N=N, T=T, dt=dt, kappa=0.4, kT=kT, measured=meas, drive_peak=drive)


@pytest.mark.parametrize("kT", [0.0, KT])
def test_single_mode_mapped_f64_matches_oracle(kT):
    p = _single(kT=kT)
    run = mapping.rk4_mapped(p)
    st = gpu_state(p)
    assert st.stage_variant() == "pipelined"
    st.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, run, TOL64)
    st = gpu_state(p)
    st.set_tune(stage_path="system")  # one CTA per system, per-term programs
    st.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, run, TOL64)


def test_general_pipelined_path_with_mixed_dissipators():
    """Secular damping at finite temperature (two diagonal-restricted terms) plus a
    conventional thermal jump pair: three sandwich terms take the pipelined kernel's
    per-term loop instead of the merged one."""
    p = _single(N=8)
    p.jumps = configs.damping_jumps(1, 0, 0.1, 0.2)
    st = gpu_state(p)
    assert st.stage_variant() == "pipelined"
    st.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, mapping.rk4_mapped(p), TOL64)


def test_single_mode_mapped_f32_matches_oracle():
    p = _single(N=12, T=0.6)
    st = gpu_state(p, dtype="f32")
    st.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, mapping.rk4_mapped(p), TOL32)


def test_direct_method_matches_number_basis_oracle():
    p = _single(N=10)
    st = gpu_state(p, method="direct")
    st.step(p.dt, p.n_steps)
    _sync()
    A = fock.rk4_adjoint(p)
    _, _, _, r = st.read_system(0)
    assert rel_err(r, A.reshape(-1)) <= TOL64


def test_two_modes_match_oracle():
    p = configs.two_mode_secular(N=4, T=0.4, dt=0.01, kappa=0.3, kT=KT)
    p.measured = {((1, 0), (0, 1)): 1.0 + 0.5j, ((0, 1), (1, 0)): 1.0 - 0.5j, ((1, 1), (1, 1)): 0.3}
    st = gpu_state(p)
    st.step(p.dt, p.n_steps)
    _sync()
    compare_mapped_systems(st, mapping.rk4_mapped(p), TOL64)
    d = gpu_state(p, method="direct")
    d.step(p.dt, p.n_steps)
    _sync()
    _, _, _, r = d.read_system(0)
    assert rel_err(r, fock.rk4_adjoint(p).reshape(-1)) <= TOL64


def test_projector_never_sources_off_diagonal_products():
    """A(0) = a without drive at T_E = 0: every G_x G_y product is off-diagonal, so the
    residual stays exactly zero on the GPU too (a missing diagonal restriction would
    source it at every point)."""
    N = 8
    meas = {((k,), (k + 1,)): math.sqrt(k + 1) for k in range(N - 1)}
    p = configs.kerr_secular(N=N, T=0.5, dt=0.005, kappa=0.4, kT=0.0, measured=meas, drive_peak=0.0)
    st = gpu_state(p)
    st.step(p.dt, p.n_steps)
    _sync()
    for s in range(st.n_systems()):
        _, gx, gy, r = st.read_system(s)
        assert np.max(np.abs(r)) == 0.0
        assert np.max(np.abs(gx)) > 0.0
    compare_mapped_systems(st, mapping.rk4_mapped(p), TOL64)


def test_batch_schedules_and_persistent_solves():
    ps = configs.secular_batch(B=48, T=0.2, dt=0.002, n_min=10, n_max=20)
    st = gpu_state(ps, dtype="f32")
    assert st.stage_variant() == "pipelined" and st.solve_eligible()
    tune = st.autotune(ps[0].dt, trial_steps=2)
    assert tune["stage_path"] in ("pipe", "system") and tune["solve_kernel"] in ("merged", "program", "step")
    st.solve(ps[0].dt, ps[0].n_steps)  # the tuned solve (a persistent launch, or stepping)
    _sync()
    for i in (0, 23, 47):
        compare_mapped_systems(st, mapping.rk4_mapped(ps[i]), TOL32, sys_offset=i, n_sys=i + 1)
    # both persistent-solve kernels against streamed stepping, FP64
    ps64 = configs.secular_batch(B=24, T=0.1, dt=0.002, n_min=8, n_max=30)
    for p in ps64[::5]:
        p.secular = [configs.SecularDamping(0, 0.3, (0.05, 0.06, 0.07))]
    ref = gpu_state(ps64)
    ref.step(ps64[0].dt, ps64[0].n_steps)
    _sync()
    for kernel in ("merged", "program"):
        sv = gpu_state(ps64)
        sv.set_tune(solve_kernel=kernel)
        sv.solve(ps64[0].dt, ps64[0].n_steps)
        _sync()
        for i in range(0, 24, 5):
            for x, y in zip(sv.read_system(i)[1:], ref.read_system(i)[1:]):
                if x is not None:
                    assert rel_err(x, y) <= 1e-10, (kernel, i)
