"""bq_step_fixed_scratch: stepping for callers that cannot allocate device memory (for
example code running inside another framework's CUDA-graph capture, where cudaMalloc is
illegal).  Its RK4 scratch lives in a fixed device array inside the library; its results
must equal bq_step's.  This file is collected last on purpose."""

import ctypes as C

import numpy as np
import pytest

import paper_2203_05526_gb300 as bq
from paper_2203_05526_gb300 import binding
from workloads import configs

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


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_fixed_scratch_equals_bq_step_two_calls(dtype, tol):
    import torch
    p = configs.random_problem(901, n_modes=2, N=5, n_steps=40, dt=0.01, dense_measured=True)
    a = gpu_state(p, dtype=dtype)   # existing entry point
    b = gpu_state(p, dtype=dtype)   # fixed-scratch entry point, called through the C ABI
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        a.step(p.dt, 20)
        binding.check(bq.lib().bq_step_fixed_scratch(b.ptr, C.c_double(p.dt), C.c_int64(20), stream))
        torch.cuda.synchronize()
        ft = np.float64 if dtype == "f64" else np.float32
        ra = _raw(a).view(ft)
        rb = _raw(b).view(ft)
        assert np.all(np.isfinite(rb))
        err = np.max(np.abs(ra - rb)) / np.max(np.abs(ra))
        assert err <= tol, (call, err)
        ea, eb = a.evaluate(), b.evaluate()
        assert abs(ea[0] - eb[0]) <= tol * max(1.0, abs(ea[0]))
        assert abs(a.time() - b.time()) < 1e-15


def test_fixed_scratch_rejects_oversized_state():
    p = configs.kerr_batch(B=1200, n_min=40, n_max=40)  # 1200 * (1600 + 80) complex FP64 > 4 MiB
    st = gpu_state(p, dtype="f64")
    with pytest.raises(bq.BQError) as ei:
        st.step_fixed_scratch(p[0].dt, 1)
    assert ei.value.status == binding.BQ_EUNSUPPORTED
    assert "fixed scratch" in str(ei.value)
