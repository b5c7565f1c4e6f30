"""SVD initial conditions (BQ_IC_SVD) on the GPU: fewer systems for operators with many
non-zero elements, the same summed result as the monomial decomposition."""

import numpy as np
import pytest

from oracle import mapping
from workloads import configs

from parity import gpu_state, rel_err

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


def _g_total(st):
    """sum over systems of w (G_x G_y^T + R) in the monomial basis, from read_system."""
    tot = None
    for s in range(st.n_systems()):
        info, gx, gy, r = st.read_system(s)
        d = gx.size
        g = info["weight"] * (np.outer(gx, gy) + (r.reshape(d, d) if r is not None else 0.0))
        tot = g if tot is None else tot + g
    return tot


@pytest.mark.parametrize("n_modes,N,dtype,tol", [(1, 8, "f64", 1e-10), (2, 4, "f64", 1e-10), (1, 8, "f32", 1e-5)])
def test_svd_ics_match_the_monomial_decomposition(n_modes, N, dtype, tol):
    """At equal separation constants (zero) the summed result depends only on g(0), so the
    SVD systems must reproduce the oracle's monomial run."""
    p = configs.random_problem(43, n_modes=n_modes, N=N, n_steps=30, dt=0.01, dense_measured=True)
    st = gpu_state(p, dtype=dtype, ic_mode="svd")
    mono = gpu_state(p, dtype=dtype, c_mode="zero")
    d = int(np.prod(p.N))
    assert st.n_systems() <= d < mono.n_systems()  # rank <= prod M < non-zero elements here
    st.step(p.dt, p.n_steps)
    _sync()
    run = mapping.rk4_mapped(p, C_override=0.0)
    ref = run.g_total().reshape(d, d)
    assert rel_err(_g_total(st), ref) <= tol
    mono.step(p.dt, p.n_steps)
    _sync()
    assert rel_err(st.evaluate(), mono.evaluate()) <= tol


def test_svd_ics_gradients_equal_monomial_gradients():
    """The discrete solve is linear in g(0) at equal separation constants, so the losses and
    the parameter gradients of the two decompositions agree to rounding."""
    p = configs.two_mode_control(n_seg=3, T=0.18, steps_per_seg=6, N=3)
    p.measured = {((1, 0), (0, 1)): 0.7 + 0.2j, ((0, 1), (1, 0)): 0.7 - 0.2j, ((1, 0), (1, 0)): 1.0,
                  ((2, 1), (0, 0)): 0.3, ((0, 0), (2, 1)): 0.3, ((1, 1), (1, 1)): -0.5}
    a = gpu_state(p, ic_mode="svd")
    b = gpu_state(p, c_mode="zero")
    la, ga = a.grad(p.dt, p.n_steps, 6)
    lb, gb = b.grad(p.dt, p.n_steps, 6)
    assert abs(la[0] - lb[0]) <= 1e-12 * max(1.0, abs(lb[0]))
    assert np.max(np.abs(ga - gb)) <= 1e-10 * np.max(np.abs(gb))
