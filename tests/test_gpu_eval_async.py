"""bq_evaluate_async: Tr(rho0_b A_b) enqueued on a stream into device or pinned host memory,
equal (bitwise) to the synchronising bq_evaluate on the pipelined path (per-system
contributions of the last stage, summed per problem on the device) and on the evaluation
kernel's path."""

import numpy as np
import pytest

from workloads import configs

from parity import gpu_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_2203_05526_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _interleaved(ev):
    return np.stack([ev.real, ev.imag], 1).ravel()


def _case(kind):
    if kind == "pipelined_batch":
        return configs.kerr_batch(B=48, T=30 * 0.002, dt=0.002, n_min=5, n_max=24), "pipelined"
    return [configs.random_problem(903, n_modes=2, N=5, n_steps=30, dt=0.01, dense_measured=True)], "generic"


@pytest.mark.parametrize("kind", ["pipelined_batch", "two_mode_dense"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_evaluate_async_equals_evaluate(kind, dtype):
    import torch
    ps, variant = _case(kind)
    st = gpu_state(ps, dtype=dtype)
    assert st.stage_variant() == variant
    stream = torch.cuda.Stream()
    host = torch.full((2 * len(ps),), np.nan, dtype=torch.float64, pin_memory=True)
    dev = torch.full((2 * len(ps),), np.nan, dtype=torch.float64, device="cuda")
    for _ in range(3):
        st.step(ps[0].dt, 10, stream=stream)
        st.evaluate_async(host.data_ptr(), stream=stream)
        st.evaluate_async(dev.data_ptr(), stream=stream)
        stream.synchronize()
        ref = _interleaved(st.evaluate(stream=stream))
        assert np.all(np.isfinite(ref))
        assert np.array_equal(host.numpy(), ref)
        assert np.array_equal(dev.cpu().numpy(), ref)


def test_evaluate_async_is_ordered_on_its_stream():
    """Results of successive steps land in distinct buffers in stream order without any host
    synchronisation in between."""
    import torch
    ps, _ = _case("pipelined_batch")
    a = gpu_state(ps, dtype="f64")
    b = gpu_state(ps, dtype="f64")
    stream = torch.cuda.Stream()
    bufs = [torch.empty(2 * len(ps), dtype=torch.float64, pin_memory=True) for _ in range(4)]
    for buf in bufs:
        a.step(ps[0].dt, 5, stream=stream)
        a.evaluate_async(buf.data_ptr(), stream=stream)
    stream.synchronize()
    for buf in bufs:
        b.step(ps[0].dt, 5)
        assert np.array_equal(buf.numpy(), _interleaved(b.evaluate()))
