"""torch.autograd.Function over the library's adjoint solve (bq_grad).

``measured_probability(spec, theta, pwc)`` returns l = Re Tr(rho0 A(T)) for the problem
described by ``spec`` (a ``workloads.spec.Problem``-like object) with its real parameters
replaced by ``theta`` and the segment values of its piecewise-constant channel replaced by
``pwc`` (shape (n_seg, 2): real and imaginary parts).  Its backward pass returns the
gradient computed by the discrete adjoint kernels (checkpointed every ``checkpoint_every``
steps).  Argument marshalling only: the forward solve, the adjoint sweep and all
reductions run in libbq.so.
"""

from __future__ import annotations

import copy

import numpy as np
import torch

from . import binding


def _spec_with(spec, theta, pwc, channel):
    s = copy.deepcopy(spec)
    s.params = [float(x) for x in theta]
    ch = s.channels[channel]
    assert ch.kind == "pwc", "the controlled channel must be piecewise constant"
    vals = []
    for re, im in pwc:
        vals += [float(re), float(im)]
    s.channels[channel] = type(ch)("pwc", (ch.params[0], ch.params[1], *vals))
    return s


class MeasuredProbability(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, pwc, spec, channel, method, dtype, checkpoint_every, grid):
        s = _spec_with(spec, theta.detach().cpu().numpy(), pwc.detach().cpu().numpy(), channel)
        h = binding.problem_from_spec(s)
        st = binding.State([h], binding.map_opts(method=method, dtype=dtype, horizon=s.T, dt=s.dt,
                                                 reverse_time=s.reverse_time, grid=grid))
        loss, g = st.grad(s.dt, s.n_steps, checkpoint_every)
        P = len(s.params)
        # slots: theta, then (Re, Im) of every segment of every pwc channel in channel order
        off = P
        for c, chn in enumerate(s.channels):
            if c == channel:
                break
            if chn.kind == "pwc":
                off += len(chn.params) - 2
        n_seg = pwc.shape[0]
        g_theta = torch.tensor(g[:P], dtype=theta.dtype)
        g_pwc = torch.tensor(g[off:off + 2 * n_seg].reshape(n_seg, 2), dtype=pwc.dtype)
        ctx.save_for_backward(g_theta, g_pwc)
        return torch.tensor(float(loss[0]), dtype=theta.dtype)

    @staticmethod
    def backward(ctx, gout):
        g_theta, g_pwc = ctx.saved_tensors
        return gout * g_theta, gout * g_pwc, None, None, None, None, None, None


def measured_probability(spec, theta: torch.Tensor, pwc: torch.Tensor, channel: int = 0, method: str = "mapped",
                         dtype: str = "f64", checkpoint_every: int = 160, grid=None) -> torch.Tensor:
    return MeasuredProbability.apply(theta, pwc, spec, channel, method, dtype, checkpoint_every, grid)
