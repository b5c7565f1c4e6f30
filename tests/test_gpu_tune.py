"""Schedule selection (bq_get_tune / bq_set_tune / bq_autotune): the autotuner leaves the
state untouched, every schedule computes the same RK4 step, and requests for schedules a
state cannot run are refused."""

import numpy as np
import pytest

import paper_2203_05526_gb300 as bq
from paper_2203_05526_gb300.binding import BQ_EUNSUPPORTED
from oracle import mapping
from workloads import configs

from parity import compare_mapped_systems, gpu_state, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _sync():
    import torch
    torch.cuda.synchronize()


def _snapshot(st):
    import torch
    host = torch.empty(st.state_bytes(), dtype=torch.uint8, pin_memory=True)
    st.store_state(host.data_ptr())
    _sync()
    return host.numpy().copy()


def _batch(n=300, dt=0.002, steps=12):
    return configs.kerr_batch(B=n, T=steps * dt, dt=dt, n_min=10, n_max=40)


def test_autotune_restores_state_and_time():
    ps = _batch()
    st = gpu_state(ps, dtype="f32")
    st.step(ps[0].dt, 3)
    _sync()
    before, t0 = _snapshot(st), st.time()
    tune = st.autotune(ps[0].dt, trial_steps=4)
    after, t1 = _snapshot(st), st.time()
    assert np.array_equal(before, after)
    assert t0 == t1
    assert tune["n_candidates"] >= 3  # pipe schedules + one CTA per system + solve kernels
    assert tune["step_us"] > 0 and tune["solve_us"] > 0
    assert st.get_tune() == tune


@pytest.mark.parametrize("n", [64, 2000])
def test_every_step_schedule_computes_the_same_step(n):
    """Pipelined schedules (slots, CTAs per SM, all steps of a call in one launch or one launch
    per stage) run the same stage code: bitwise equal states and observables, with one system
    per CTA (64 instances) and with many per CTA in ragged sizes (2000).  The
    one-CTA-per-system path evaluates the same stencil from per-term programs: equal to FP32
    rounding, and both match the FP64 oracle."""
    ps = _batch(n=n)
    dt, n = ps[0].dt, 12
    ref = gpu_state(ps, dtype="f32")
    assert ref.get_tune()["stage_path"] == "pipe"
    ref.step(dt, n)
    base = _snapshot(ref)
    assert ref.get_tune()["pipe_fused"] == 1
    for slots, cap, fused in ((3, 0, 1), (2, 1, 1), (4, 2, 1), (2, 0, 0), (3, 1, 0)):
        st = gpu_state(ps, dtype="f32")
        st.set_tune(stage_path="pipe", pipe_slots=slots, pipe_ctas_per_sm=cap, pipe_fused=fused)
        if fused:
            st.step(dt, n)
        else:
            for _ in range(n):  # one launch per stage, one call per step
                st.step(dt, 1)
        assert np.array_equal(_snapshot(st), base), (slots, cap, fused)
        assert np.array_equal(st.evaluate(), ref.evaluate()), (slots, cap, fused)
    st = gpu_state(ps, dtype="f32")
    st.set_tune(stage_path="system")
    st.step(dt, n)
    _sync()
    for i in (0, 17, 63):
        run = mapping.rk4_mapped(ps[i])
        compare_mapped_systems(st, run, 1e-5, sys_offset=i, n_sys=i + 1)
        compare_mapped_systems(ref, run, 1e-5, sys_offset=i, n_sys=i + 1)


def test_solve_kernels_agree_and_tuned_solve_matches_streaming():
    ps = _batch(n=96)
    dt, n = ps[0].dt, 12
    streamed = gpu_state(ps, dtype="f64")
    streamed.step(dt, n)
    _sync()
    for kernel in ("merged", "program"):
        for cap in (0, 1):
            st = gpu_state(ps, dtype="f64")
            st.set_tune(solve_kernel=kernel, solve_ctas_per_sm=cap)
            st.solve(dt, n)
            _sync()
            for i in (0, 41, 95):
                for x, y in zip(st.read_system(i)[1:], streamed.read_system(i)[1:]):
                    if x is not None:
                        assert rel_err(x, y) <= 1e-10, (kernel, cap, i)
    st = gpu_state(ps, dtype="f64")
    st.autotune(dt, trial_steps=3)
    st.solve(dt, n)
    _sync()
    for x, y in zip(st.read_system(5)[1:], streamed.read_system(5)[1:]):
        if x is not None:
            assert rel_err(x, y) <= 1e-10
    # bq_solve with BQ_SOLVE_STEP runs bq_step: bitwise the streamed result
    st = gpu_state(ps, dtype="f64")
    st.set_tune(solve_kernel="step")
    assert st.get_tune()["solve_kernel"] == "step"
    st.solve(dt, n)
    _sync()
    for i in (0, 41, 95):
        for x, y in zip(st.read_system(i)[1:], streamed.read_system(i)[1:]):
            if x is not None:
                assert np.array_equal(x, y)


def test_unavailable_schedules_are_refused():
    two = configs.two_mode(N=4)
    st = gpu_state(two)  # two modes: tiled path only, no persistent solve
    assert st.get_tune()["stage_path"] == "tiled"
    with pytest.raises(bq.BQError) as e:
        st.set_tune(stage_path="pipe")
    assert e.value.args[0].startswith(f"bq status {BQ_EUNSUPPORTED}")
    with pytest.raises(bq.BQError):
        st.set_tune(stage_path="system")
    one = gpu_state(_batch(n=4))
    with pytest.raises(bq.BQError):
        one.set_tune(stage_path="pipe", pipe_slots=9)
    with pytest.raises(bq.BQError):
        one.set_tune(stage_path="tiled")
    tune = st.autotune(two.dt, trial_steps=2)
    assert tune["stage_path"] == "tiled" and tune["solve_kernel"] == "step"


def test_tile_lengths_compute_the_same_step_and_gradients():
    """The tiled kernels evaluate every point from the same sources whatever the tile length
    and wherever the sources come from (shared-memory halo windows or global reads): the step
    and the adjoint gradients agree with the default tiling to rounding, and the autotuner
    keeps a valid tile."""
    p = configs.two_mode_control(n_seg=3, T=0.18, steps_per_seg=6, N=7)
    p.measured = {((1, 0), (0, 1)): 0.7 + 0.2j, ((0, 1), (1, 0)): 0.7 - 0.2j, ((1, 0), (1, 0)): 1.0,
                  ((2, 1), (0, 0)): 0.3, ((0, 0), (2, 1)): 0.3}
    ref = gpu_state(p)
    assert ref.get_tune()["stage_path"] == "tiled" and ref.get_tune()["tile"] == 0
    assert ref.get_tune()["lanes"] == 4  # a small launch: four lanes per point
    ref.step(p.dt, p.n_steps)
    _sync()
    l0, g0 = gpu_state(p).grad(p.dt, p.n_steps, 6)
    for tile, gread in ((32, 0), (96, 0), (192, 0), (1024, 0), (32, 1), (47, 1), (256, 1)):
        st = gpu_state(p)
        st.set_tune(tile=tile, gread=gread)
        assert st.get_tune()["tile"] == tile and st.get_tune()["gread"] == gread
        st.step(p.dt, p.n_steps)
        _sync()
        for s in range(ref.n_systems()):
            for x, y in zip(st.read_system(s)[1:], ref.read_system(s)[1:]):
                if y is not None:
                    assert rel_err(x, y) <= 1e-13, (tile, s)
        gs = gpu_state(p)
        gs.set_tune(tile=tile, gread=gread)
        l1, g1 = gs.grad(p.dt, p.n_steps, 6)
        assert abs(l1[0] - l0[0]) <= 1e-13 * max(1.0, abs(l0[0]))
        assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0)), tile
    st = gpu_state(p)
    with pytest.raises(bq.BQError):
        st.set_tune(tile=16)
    with pytest.raises(bq.BQError):
        st.set_tune(lanes=3)
    tune = st.autotune(p.dt, trial_steps=2)
    # a tile of the fixed list, or one of the tiles that give at most 1, 2 or 3 items per SM
    assert (tune["tile"] == 0 or tune["tile"] >= 32) and tune["lanes"] in (1, 2, 4)
    assert tune["n_candidates"] >= 2
    st.step(p.dt, p.n_steps)
    _sync()
    for x, y in zip(st.read_system(0)[1:], ref.read_system(0)[1:]):
        if y is not None:
            assert rel_err(x, y) <= 1e-13


@pytest.mark.parametrize("n_modes", [2, 3])
def test_lanes_per_point_split_the_same_sums(n_modes):
    """One, two or four lanes per point sum the same terms in different groupings: the step
    and the adjoint gradients agree to rounding and match the oracle; the separable part runs
    in work items of its own (several chunks of [G_x | G_y] per split system)."""
    if n_modes == 2:
        p = configs.two_mode_control(n_seg=3, T=0.18, steps_per_seg=6, N=7)
        p.measured = {((1, 0), (0, 1)): 0.7 + 0.2j, ((0, 1), (1, 0)): 0.7 - 0.2j, ((1, 0), (1, 0)): 1.0,
                      ((2, 1), (0, 0)): 0.3, ((0, 0), (2, 1)): 0.3}
    else:
        p = configs.random_problem(11, n_modes=3, N=3, n_steps=12, dt=0.01)
    run = mapping.rk4_mapped(p)
    res, grads = {}, {}
    for lanes in (1, 2, 4):
        st = gpu_state(p)
        st.set_tune(lanes=lanes, tile=64)
        assert st.get_tune()["lanes"] == lanes
        st.step(p.dt, p.n_steps)
        _sync()
        compare_mapped_systems(st, run, 1e-10)
        res[lanes] = [st.read_system(s) for s in range(st.n_systems())]
        if n_modes == 2:
            gs = gpu_state(p)
            gs.set_tune(lanes=lanes, tile=64)
            grads[lanes] = gs.grad(p.dt, p.n_steps, 6)
    for lanes in (2, 4):
        for a, b in zip(res[lanes], res[1]):
            for x, y in zip(a[1:], b[1:]):
                if y is not None:
                    assert rel_err(x, y) <= 1e-13, lanes
        if grads:
            (l1, g1), (l0, g0) = grads[lanes], grads[1]
            assert abs(l1[0] - l0[0]) <= 1e-13 * max(1.0, abs(l0[0]))
            assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0)), lanes


def test_gradient_autotuner_keeps_a_candidate_and_the_gradient():
    """bq_autotune_grad times bq_grad under every tiled schedule: the state is unchanged,
    the chosen schedule is one of the candidates, and the gradient afterwards equals the
    default schedule's to rounding."""
    p = configs.two_mode_control(n_seg=3, T=0.18, steps_per_seg=6, N=7)
    ref = gpu_state(p)
    l0, g0 = ref.grad(p.dt, p.n_steps, 6)
    st = gpu_state(p)
    before, t0 = _snapshot(st), st.time()
    tune = st.autotune_grad(p.dt, trial_steps=8, checkpoint_every=4)
    assert np.array_equal(_snapshot(st), before) and st.time() == t0
    assert tune["n_candidates"] >= 24 and tune["grad_us"] > 0
    assert tune["tile"] in (0, 32, 64, 96, 128, 192, 256, 512) and tune["lanes"] in (1, 2, 4)
    assert st.get_tune()["tile"] == tune["tile"] and st.get_tune()["lanes"] == tune["lanes"]
    l1, g1 = st.grad(p.dt, p.n_steps, 6)
    assert abs(l1[0] - l0[0]) <= 1e-13 * max(1.0, abs(l0[0]))
    assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0))
