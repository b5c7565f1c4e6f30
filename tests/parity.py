"""Helpers that run one seeded problem through the CUDA path (C ABI) and through the
oracle, and compare them element by element."""

from __future__ import annotations

import numpy as np

import paper_2203_05526_gb300 as bq
from oracle import fock, mapping


def gpu_state(specs, method="mapped", dtype="f64", grid=None, r_layout="full", c_mode="eq304", basis="auto",
              ic_mode="monomial"):
    if not isinstance(specs, (list, tuple)):
        specs = [specs]
    s0 = specs[0]
    handles = [bq.problem_from_spec(s) for s in specs]
    opts = bq.map_opts(method=method, dtype=dtype, grid=grid, r_layout=r_layout, c_mode=c_mode, basis=basis,
                       reverse_time=s0.reverse_time, horizon=s0.T, dt=s0.dt, ic_mode=ic_mode)
    return bq.State(handles, opts)


def rel_err(a, ref, floor=0.0):
    a = np.asarray(a)
    ref = np.asarray(ref)
    scale = max(float(np.max(np.abs(ref))) if ref.size else 0.0, floor)
    if scale == 0.0:
        return float(np.max(np.abs(a))) if a.size else 0.0
    return float(np.max(np.abs(a - ref)) / scale)


# Floors of the scalar-observable tolerance (|x - x_ref| <= tol * max(|x_ref|, floor)): a value
# below the floor is compared in absolute terms at tol * floor.
FLOOR64 = 1e-14
FLOOR32 = 1e-7


def scalar_err(x, ref, floor):
    """|x - ref| / max(|ref|, floor) for a scalar observable such as Tr(rho0 A)."""
    return abs(complex(x) - complex(ref)) / max(abs(complex(ref)), floor)


def compare_mapped_systems(state, run, tol, sys_offset=0, n_sys=None):
    """Every system (initial condition) of ``state`` against the oracle run's IC with the
    same (p, q): G_x, G_y and R element by element, relative to the IC's largest value."""
    M = run.model.M
    ics = {(int(np.ravel_multi_index(p, M)), int(np.ravel_multi_index(q, M))): ic for ic in run.ics
           for p, q in [(ic[0], ic[1])]}
    n_sys = state.n_systems() if n_sys is None else n_sys
    worst = 0.0
    assert n_sys - sys_offset == len(ics), (n_sys, len(ics))
    for s in range(sys_offset, n_sys):
        info, gx, gy, r = state.read_system(s)
        ic = ics[(info["p"], info["q"])]
        _, _, w, C, Gx, Gy, R = ic
        assert abs(info["weight"] - w) <= 1e-12 * abs(w)
        assert abs(info["C"] - C) <= 1e-12 * max(1.0, abs(C))
        scale = max(np.max(np.abs(Gx)), np.max(np.abs(Gy)), np.max(np.abs(R)))
        for a, ref in ((gx, Gx), (gy, Gy), (r, R.reshape(-1) if r is not None else None)):
            if a is None:
                continue
            e = rel_err(a, ref, floor=1e-6 * scale)
            worst = max(worst, e)
    assert worst <= tol, worst
    return worst


def oracle_block(A: np.ndarray, N, lo=3):
    return fock.low_block(A, N, lo)
