"""CPU-only checks of the C ABI: the library loads, exports every function include/bq.h
declares, and its host logic (problem validation, planning, stability bound) behaves."""

import ctypes as C
import os
import re

import pytest

import paper_2203_05526_gb300 as bq
from paper_2203_05526_gb300 import binding
from workloads import configs
from workloads.spec import HTerm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2203_05526_gb300 import build
    build.build()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bq_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    L = bq.lib()
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(bq.exported_symbols()) <= set(names)


def required(spec, **kw):
    h = bq.problem_from_spec(spec)
    arr = (C.c_void_p * 1)(h.ptr.value)
    n = C.c_size_t()
    st = bq.lib().bq_required_bytes(arr, 1, C.byref(bq.map_opts(**kw)), C.byref(n))
    return st, n.value


def test_required_bytes_and_layout():
    st, n = required(configs.kerr_driven(N=40), grid=[12], dt=0.0025, horizon=100.0)
    assert st == 0 and n > 4 * 16 * (12 * 12 + 2 * 12)
    st64, n64 = required(configs.kerr_driven(N=40), grid=[12], dt=0.0025, horizon=100.0, dtype="f32")
    assert st64 == 0 and n64 < n


def test_unstable_dt_refused():
    # N = 40 Kerr at dt = 0.01: |K|/2 * 39 * 38 * dt ~ 9.3 > 2 sqrt 2
    st, _ = required(configs.kerr_driven(N=40), method="direct", dt=0.01, horizon=100.0)
    assert st == binding.BQ_EUNSTABLE_DT
    st, _ = required(configs.kerr_driven(N=40), method="direct", dt=0.0025, horizon=100.0)
    assert st == 0


def test_non_hermitian_hamiltonian_refused():
    p = configs.kerr_driven(N=8)
    p.h_terms = p.h_terms[:-1]  # drop the conjugate drive term
    st, _ = required(p, dt=0.001)
    assert st == binding.BQ_EINVAL
    assert "Hermitian" in bq.lib().bq_last_error().decode()


def test_bad_arguments():
    with pytest.raises(bq.BQError):
        bq.ProblemHandle(0, [4])
    with pytest.raises(bq.BQError):
        bq.ProblemHandle(5, [4, 4, 4, 4, 4])  # more than BQ_MAX_MODES = 4
    h = bq.ProblemHandle(1, [4])
    with pytest.raises(bq.BQError):
        h.add_h_term(1.0, [1], [1], channel=3)
    with pytest.raises(bq.BQError):
        h.add_channel("gauss", [1.0, 0.0, 1.0, 0.0])  # sigma = 0


def test_too_many_modes_grid_unsupported():
    st, _ = required(configs.kerr_static(N=200), dt=1e-4)
    assert st == binding.BQ_EUNSUPPORTED


def test_four_mode_networks_plan_and_scale_with_the_layout():
    """Planning (host only) of the Table I network with four modes: the mapped layouts need
    far less memory per initial condition than the conventional matrix, the direct method
    holds the N^8 matrix, and the diagonal residual layout sits between R = 0 and full R."""
    p = configs.table_one_network(4, 4, steps=4000)
    sizes = {}
    for name, kw in (("direct", dict(method="direct")), ("full", {}), ("diag", dict(r_layout="diag")),
                     ("off", dict(r_layout="off"))):
        st, n = required(p, dt=p.dt, horizon=p.T, **kw)
        assert st == 0, (name, bq.lib().bq_last_error().decode())
        sizes[name] = n
    assert sizes["off"] < sizes["diag"] < sizes["full"]
    assert sizes["direct"] > 5 * 16 * 4 ** 8  # five complex FP64 arrays of the 4^8 matrix


def _plan(specs, **kw):
    specs = specs if isinstance(specs, (list, tuple)) else [specs]
    return bq.plan([bq.problem_from_spec(s) for s in specs], bq.map_opts(dt=specs[0].dt, horizon=specs[0].T, **kw))


def test_work_decomposition_of_a_large_two_mode_system():
    """One 2-mode system of 20 736 R points and 288 G points (the control problem): split into
    256-point R tiles (a single system cannot fill the GPU otherwise) plus 64-point chunks of
    [G_x | G_y]; four lanes per point; capacity for 32-point tiles."""
    p = configs.two_mode_control()
    info = _plan(p, dtype="f64")
    assert info["stage_variant"] == "generic" and info["n_systems"] == 1
    assert info["n_work"] == 20736 // 256 + 288 // 64 + 1  # 81 R tiles, 5 G chunks (4 full + 1 of 32)
    assert info["work_cap"] == 20736 // 32 + 288 // 32
    assert info["lanes"] == 4


def test_work_decomposition_of_small_batches_and_layouts():
    """Three-mode Table I network (125 initial conditions of 216 points per mode space):
    separable-only systems (R = 0) are split into 64-point chunks, R(xy) systems into one R
    tile plus chunks, full-R systems (46 656 points each) into tiles; large batches of small
    single-mode systems stay one CTA per system on the single-mode paths."""
    p = configs.table_one_network(3, 6, steps=2000)
    off = _plan(p, r_layout="off")
    assert off["n_systems"] == 125 and off["n_work"] == 125 * 7  # 432 G points -> 7 chunks
    diag = _plan(p, r_layout="diag")
    assert diag["n_work"] == 125 * 8  # + one 216-point R tile
    assert diag["smem_bytes"] >= off["smem_bytes"] + 16 * 216  # plus the staged R window
    batch = configs.kerr_batch(B=512, T=1.0, dt=0.002)
    b = _plan(batch, dtype="f32")
    assert b["stage_variant"] == "pipelined" and b["n_work"] == 512 and b["lanes"] == 1


def test_svd_initial_conditions_plan_fewer_systems():
    """Host Jacobi SVD of g(0) (BQ_IC_SVD): a dense measured operator on a two-mode grid of
    d = 16 points needs at most d systems (its rank), against one per non-zero element of
    g(0) for the monomial decomposition."""
    p = configs.random_problem(43, n_modes=2, N=4, n_steps=4, dt=0.01, dense_measured=True)
    mono = _plan(p, c_mode="zero")
    svd = _plan(p, ic_mode="svd")
    assert svd["n_systems"] <= 16 < mono["n_systems"]
    assert svd["total_elems"] < mono["total_elems"]
