"""bq_step_fixed_scratch: stepping for callers that cannot allocate device memory, for
example code whose device memory is all handed out by another component's allocator at
start-up, or a loop that must not pay for an allocation.  Its RK4 scratch (the stage inputs
and the stage sum) lives in a fixed device array inside the library; its results must equal
bq_step's, whatever state used the array before.  This file is collected last on purpose."""

import ctypes as C

import numpy as np
import pytest

import paper_2203_05526_gb300 as bq
from paper_2203_05526_gb300 import binding
from workloads import configs
from workloads.spec import Problem

from parity import gpu_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _raw(state):
    import torch
    n = state.state_bytes()
    host = torch.empty(n, dtype=torch.uint8)
    state.store_state(host.data_ptr())
    torch.cuda.synchronize()
    return host.numpy().copy()


def _fixed_step(state, dt, n):
    """One call of the allocation-free entry point through the C ABI."""
    import torch
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    binding.check(bq.lib().bq_step_fixed_scratch(state.ptr, C.c_double(dt), C.c_int64(n), stream))


def _case(kind):
    """(problems, stage path or None for the default, expected stage variant)."""
    if kind == "tiled_two_mode":
        return [configs.random_problem(901, n_modes=2, N=5, n_steps=40, dt=0.01, dense_measured=True)], None, "generic"
    if kind == "pipelined_batch":
        return configs.kerr_batch(B=48, T=40 * 0.002, dt=0.002, n_min=5, n_max=24), None, "pipelined"
    if kind == "three_mode_global_read":
        p = configs.table_one_network(3, 6, steps=4000)
        p = Problem(**{**p.__dict__, "T": 40 * p.dt,
                       "measured": {((1, 0, 1), (0, 1, 1)): 1.0 + 0.3j, ((0, 1, 1), (1, 0, 1)): 1.0 - 0.3j}})
        return [p], None, "generic"
    raise ValueError(kind)


def _dirty_the_array(dtype):
    """Runs a state of another layout and the other precision through the fixed array, so the
    array holds unrelated values (including in its padding) when the compared calls start."""
    other = "f32" if dtype == "f64" else "f64"
    p = configs.random_problem(77, n_modes=1, N=9, n_steps=6, dt=0.01, dense_measured=True)
    st = gpu_state(p, dtype=other)
    _fixed_step(st, p.dt, 6)


@pytest.mark.parametrize("kind", ["tiled_two_mode", "pipelined_batch", "three_mode_global_read"])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_fixed_scratch_equals_bq_step_two_calls(kind, dtype, tol):
    import torch
    ps, path, variant = _case(kind)
    a = gpu_state(ps, dtype=dtype)   # existing entry point
    b = gpu_state(ps, dtype=dtype)   # fixed-scratch entry point, called through the C ABI
    if path is not None:
        a.set_tune(stage_path=path)
        b.set_tune(stage_path=path)
    assert a.stage_variant() == variant and b.stage_variant() == variant
    _dirty_the_array(dtype)
    dt = ps[0].dt
    ft = np.float64 if dtype == "f64" else np.float32
    for call in range(2):
        a.step(dt, 20)
        _fixed_step(b, dt, 20)
        torch.cuda.synchronize()
        ra = _raw(a).view(ft)
        rb = _raw(b).view(ft)
        assert np.all(np.isfinite(rb))
        err = np.max(np.abs(ra - rb)) / np.max(np.abs(ra))
        assert err <= tol, (call, err)
        ea, eb = a.evaluate(), b.evaluate()
        assert np.max(np.abs(ea - eb)) <= tol * max(1.0, np.max(np.abs(ea)))
        assert abs(a.time() - b.time()) < 1e-15


def test_fixed_scratch_rejects_oversized_state():
    p = configs.kerr_batch(B=1200, n_min=40, n_max=40)  # 1200 * (1600 + 80) complex FP64 > 4 MiB
    st = gpu_state(p, dtype="f64")
    with pytest.raises(bq.BQError) as ei:
        st.step_fixed_scratch(p[0].dt, 1)
    assert ei.value.status == binding.BQ_EUNSUPPORTED
    assert "fixed scratch" in str(ei.value)
