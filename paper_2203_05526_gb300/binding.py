"""ctypes binding of the C ABI declared in include/bq.h (argument marshalling only).

Every numerical step runs inside ``libbq.so``; this module converts Python values to the
C argument types, owns the device buffer a state lives in (a torch uint8 tensor, i.e. the
PyTorch caching allocator provides device memory) and passes torch's current CUDA stream.
If the library is missing the import fails loudly: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbq.so")

BQ_OK = 0
BQ_EINVAL = -1
BQ_EUNSTABLE_DT = -2
BQ_ENOMEM = -3
BQ_ECUDA = -4
BQ_ENONFINITE = -5
BQ_ETIMEOUT = -6
BQ_EUNSUPPORTED = -7

CH_KIND = {"const": 0, "gauss": 1, "pwc": 2, "cexp": 3}
METHOD = {"mapped": 0, "direct": 1}
DTYPE = {"f64": 0, "f32": 1}
R_LAYOUT = {"full": 0, "off": 1, "diag": 2}
BASIS = {"auto": 0, "monomial": 1, "number": 2}
C_MODE = {"eq304": 0, "zero": 1}
IC_MODE = {"monomial": 0, "svd": 1}
MAX_MODES = 4


PATH = {0: "tiled", 1: "system", 2: "pipe"}
SOLVE_KERNEL = {-1: "step", 0: "program", 1: "merged"}  # -1: bq_solve runs bq_step


class bq_tune(C.Structure):
    _fields_ = [("stage_path", C.c_int), ("pipe_slots", C.c_int), ("pipe_ctas_per_sm", C.c_int),
                ("solve_kernel", C.c_int), ("solve_ctas_per_sm", C.c_int), ("n_candidates", C.c_int),
                ("step_us", C.c_double), ("solve_us", C.c_double), ("tile", C.c_int), ("lanes", C.c_int), ("gread", C.c_int),
                ("grad_coop", C.c_int), ("grad_us", C.c_double), ("pipe_fused", C.c_int), ("pad", C.c_int)]


class bq_plan_info(C.Structure):
    _fields_ = [("n_systems", C.c_int), ("n_work", C.c_int), ("work_cap", C.c_int), ("lanes", C.c_int),
                ("stage_variant", C.c_int), ("smem_bytes", C.c_int), ("adj_smem_bytes", C.c_int), ("pad", C.c_int),
                ("total_elems", C.c_int64)]


class BQError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"bq status {status}: {detail}")
        self.status = status


class bq_map_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("dtype", C.c_int), ("r_layout", C.c_int), ("basis", C.c_int),
                ("c_mode", C.c_int), ("reverse_time", C.c_int), ("grid", C.c_int * MAX_MODES),
                ("horizon", C.c_double), ("dt", C.c_double), ("ic_mode", C.c_int), ("pad", C.c_int)]


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2203_05526_gb300.build.build() "
                          "(the solver has no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, ip, dp, i64 = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int64
    sig = {
        "bq_problem_create": (C.c_int, [C.POINTER(vp), C.c_int, ip]),
        "bq_problem_destroy": (None, [vp]),
        "bq_problem_add_channel": (C.c_int, [vp, C.c_int, dp, C.c_int, ip]),
        "bq_problem_add_h_term": (C.c_int, [vp, C.c_double, C.c_double, ip, ip, C.c_int, C.c_int, C.c_int]),
        "bq_problem_set_params": (C.c_int, [vp, dp, C.c_int]),
        "bq_problem_add_jump": (C.c_int, [vp, C.c_double, C.c_int, dp, dp, ip, ip]),
        "bq_problem_add_secular": (C.c_int, [vp, C.c_int, C.c_double, C.c_int, dp]),
        "bq_problem_set_measured": (C.c_int, [vp, C.c_int, ip, ip, dp, dp]),
        "bq_problem_set_rho0": (C.c_int, [vp, C.c_int, ip, ip, dp, dp]),
        "bq_required_bytes": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(bq_map_opts), C.POINTER(C.c_size_t)]),
        "bq_map": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(bq_map_opts), vp, C.c_size_t, vp, C.POINTER(vp)]),
        "bq_step": (C.c_int, [vp, C.c_double, i64, vp]),
        "bq_step_fixed_scratch": (C.c_int, [vp, C.c_double, i64, vp]),
        "bq_solve": (C.c_int, [vp, C.c_double, i64, vp]),
        "bq_grad_size": (C.c_int, [vp, ip]),
        "bq_grad_required_bytes": (C.c_int, [vp, i64, C.c_int, C.POINTER(C.c_size_t)]),
        "bq_grad": (C.c_int, [vp, C.c_double, i64, C.c_int, vp, C.c_size_t, dp, dp, vp]),
        "bq_solve_eligible": (C.c_int, [vp, ip]),
        "bq_get_tune": (C.c_int, [vp, C.POINTER(bq_tune)]),
        "bq_set_tune": (C.c_int, [vp, C.POINTER(bq_tune)]),
        "bq_autotune_scratch_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
        "bq_autotune": (C.c_int, [vp, C.c_double, C.c_int, vp, C.c_size_t, vp, C.POINTER(bq_tune)]),
        "bq_autotune_grad": (C.c_int, [vp, C.c_double, C.c_int, C.c_int, vp, C.c_size_t, vp, C.POINTER(bq_tune)]),
        "bq_plan": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(bq_map_opts), C.POINTER(bq_plan_info)]),
        "bq_stage_variant": (C.c_int, [vp, ip]),
        "bq_time": (C.c_int, [vp, dp]),
        "bq_evaluate": (C.c_int, [vp, dp, vp]),
        "bq_evaluate_async": (C.c_int, [vp, vp, vp]),
        "bq_grad_record_bytes": (C.c_int, [vp, C.c_int64, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_int64)]),
        "bq_fock_block": (C.c_int, [vp, C.c_int, dp, vp]),
        "bq_state_info": (C.c_int, [vp, ip, C.POINTER(C.c_int64)]),
        "bq_system_info": (C.c_int, [vp, C.c_int, ip, ip, ip, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64), dp, dp]),
        "bq_read_system": (C.c_int, [vp, C.c_int, dp, dp, dp, vp]),
        "bq_state_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
        "bq_store_state": (C.c_int, [vp, vp, vp]),
        "bq_load_state": (C.c_int, [vp, vp, vp]),
        "bq_set_time": (C.c_int, [vp, C.c_double]),
        "bq_state_destroy": (None, [vp]),
        "bq_status_string": (C.c_char_p, [C.c_int]),
        "bq_last_error": (C.c_char_p, []),
        "bq_launch_count": (C.c_int64, []),
        "bq_fma_peak": (C.c_int, [C.c_int, i64, dp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols() -> List[str]:
    """Names declared in include/bq.h that the binding resolves."""
    return [n for n in ("bq_problem_create", "bq_problem_destroy", "bq_problem_add_channel",
                        "bq_problem_add_h_term", "bq_problem_set_params", "bq_problem_add_jump",
                        "bq_problem_set_measured", "bq_problem_set_rho0", "bq_required_bytes", "bq_map",
                        "bq_step", "bq_step_fixed_scratch", "bq_solve", "bq_solve_eligible", "bq_stage_variant", "bq_grad_size", "bq_grad_required_bytes", "bq_grad_record_bytes", "bq_grad", "bq_time", "bq_evaluate", "bq_evaluate_async", "bq_fock_block", "bq_state_info",
                        "bq_system_info", "bq_read_system", "bq_state_bytes", "bq_store_state",
                        "bq_load_state", "bq_set_time", "bq_state_destroy", "bq_status_string",
                        "bq_last_error", "bq_launch_count", "bq_fma_peak")]


def check(status: int) -> None:
    if status != BQ_OK:
        L = lib()
        raise BQError(status, f"{L.bq_status_string(status).decode()}: {L.bq_last_error().decode()}")


def _iarr(xs: Iterable[int]):
    xs = list(int(x) for x in xs)
    return (C.c_int * max(1, len(xs)))(*xs)


def _darr(xs: Iterable[float]):
    xs = list(float(x) for x in xs)
    return (C.c_double * max(1, len(xs)))(*xs)


class ProblemHandle:
    """Owns a bq_problem* built through the C ABI."""

    def __init__(self, n_modes: int, fock_trunc: Sequence[int]):
        self.ptr = C.c_void_p()
        self.n_modes = n_modes
        check(lib().bq_problem_create(C.byref(self.ptr), n_modes, _iarr(fock_trunc)))

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.bq_problem_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def add_channel(self, kind: str, params: Sequence[float]) -> int:
        out = C.c_int()
        check(lib().bq_problem_add_channel(self.ptr, CH_KIND[kind], _darr(params), len(params), C.byref(out)))
        return out.value

    def add_h_term(self, coef: complex, u, v, channel: int = -1, conj: bool = False, param: int = -1):
        check(lib().bq_problem_add_h_term(self.ptr, coef.real, coef.imag, _iarr(u), _iarr(v), channel,
                                          1 if conj else 0, param))

    def set_params(self, values: Sequence[float]):
        check(lib().bq_problem_set_params(self.ptr, _darr(values), len(values)))

    def add_jump(self, rate: float, terms):
        cre = [complex(c).real for c, _, _ in terms]
        cim = [complex(c).imag for c, _, _ in terms]
        u = [x for _, uu, _ in terms for x in uu]
        v = [x for _, _, vv in terms for x in vv]
        check(lib().bq_problem_add_jump(self.ptr, rate, len(terms), _darr(cre), _darr(cim), _iarr(u), _iarr(v)))

    def add_secular(self, mode: int, kappa: float, nbar=()):
        nbar = [float(x) for x in nbar]
        check(lib().bq_problem_add_secular(self.ptr, int(mode), float(kappa), len(nbar),
                                           _darr(nbar) if nbar else None))

    def _elems(self, fn, elems):
        items = list(elems.items())
        k = [x for (kk, _), _ in items for x in kk]
        l = [x for (_, ll), _ in items for x in ll]
        re = [complex(v).real for _, v in items]
        im = [complex(v).imag for _, v in items]
        check(fn(self.ptr, len(items), _iarr(k), _iarr(l), _darr(re), _darr(im)))

    def set_measured(self, elems):
        self._elems(lib().bq_problem_set_measured, elems)

    def set_rho0(self, elems):
        self._elems(lib().bq_problem_set_rho0, elems)


def problem_from_spec(spec) -> ProblemHandle:
    """Marshals a ``workloads.spec.Problem`` (or any object with the same fields)."""
    h = ProblemHandle(spec.n_modes, spec.N)
    for ch in spec.channels:
        h.add_channel(ch.kind, ch.params)
    if spec.params:
        h.set_params(spec.params)
    for t in spec.h_terms:
        h.add_h_term(complex(t.coef), t.u, t.v, t.channel, t.conj, t.param)
    for j in spec.jumps:
        h.add_jump(j.rate, j.terms)
    for sd in getattr(spec, "secular", []):
        h.add_secular(sd.mode, sd.kappa, sd.nbar)
    h.set_measured(spec.measured)
    if spec.rho0 is not None:
        h.set_rho0(spec.rho0)
    return h


def map_opts(method="mapped", dtype="f64", r_layout="full", basis="auto", c_mode="eq304", reverse_time=True,
             grid: Optional[Sequence[int]] = None, horizon: float = 0.0, dt: float = 0.0,
             ic_mode: str = "monomial") -> bq_map_opts:
    o = bq_map_opts()
    o.method, o.dtype, o.r_layout = METHOD[method], DTYPE[dtype], R_LAYOUT[r_layout]
    o.basis, o.c_mode, o.reverse_time = BASIS[basis], C_MODE[c_mode], 1 if reverse_time else 0
    g = list(grid or [])
    for j in range(MAX_MODES):
        o.grid[j] = int(g[j]) if j < len(g) else 0
    o.horizon, o.dt = float(horizon), float(dt)
    o.ic_mode = IC_MODE[ic_mode]
    return o


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def grad_record_bytes(state: "State", n_steps: int, checkpoint_every: int):
    """(bytes of one segment's recording, number of segments) of bq_grad (bq_grad_record_bytes)."""
    per, nseg = C.c_size_t(), C.c_int64()
    check(lib().bq_grad_record_bytes(state.ptr, int(n_steps), int(checkpoint_every), C.byref(per), C.byref(nseg)))
    return per.value, nseg.value


def plan(handles: Sequence["ProblemHandle"], opts: "bq_map_opts") -> dict:
    """Host-only view of the plan bq_map would build for these problems (bq_plan): no device
    is needed."""
    arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    info = bq_plan_info()
    check(lib().bq_plan(arr, len(handles), C.byref(opts), C.byref(info)))
    variant = {0: "generic", 1: "single_mode", 2: "pipelined"}[info.stage_variant]
    return dict(n_systems=info.n_systems, n_work=info.n_work, work_cap=info.work_cap, lanes=info.lanes,
                stage_variant=variant, smem_bytes=info.smem_bytes, adj_smem_bytes=info.adj_smem_bytes,
                total_elems=info.total_elems)


class State:
    """A batch of mapped (or direct) problems resident in one torch-owned device buffer."""

    def __init__(self, handles: Sequence[ProblemHandle], opts: bq_map_opts, device=None, stream=None):
        import torch
        self.handles = list(handles)  # keep problems alive while the state exists
        arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
        nbytes = C.c_size_t()
        check(lib().bq_required_bytes(arr, len(handles), C.byref(opts), C.byref(nbytes)))
        self.nbytes = nbytes.value
        self.pool = torch.empty(self.nbytes, dtype=torch.uint8, device=device or "cuda")
        self.ptr = C.c_void_p()
        self.B = len(handles)
        self.opts = opts
        check(lib().bq_map(arr, len(handles), C.byref(opts), C.c_void_p(self.pool.data_ptr()), self.nbytes,
                           _stream_ptr(stream), C.byref(self.ptr)))

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.bq_state_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def step(self, dt: float, n_steps: int, stream=None):
        check(lib().bq_step(self.ptr, float(dt), int(n_steps), _stream_ptr(stream)))

    def solve(self, dt: float, n_steps: int, stream=None):
        """Batched persistent solve: all n_steps of every system in one kernel launch."""
        check(lib().bq_solve(self.ptr, float(dt), int(n_steps), _stream_ptr(stream)))

    def grad(self, dt: float, n_steps: int, checkpoint_every: int = 160, stream=None, record_segments: int = 2):
        """(losses[B], gradient) of Re Tr(rho0 A(T)) by the discrete adjoint (bq_grad).
        record_segments: recordings the workspace holds (2 = the minimum; on the cooperative
        path every recording beyond those the backward sweep needs spares one segment's
        recomputation; -1 = all segments)."""
        import torch
        n = C.c_int()
        check(lib().bq_grad_size(self.ptr, C.byref(n)))
        nb = C.c_size_t()
        check(lib().bq_grad_required_bytes(self.ptr, int(n_steps), int(checkpoint_every), C.byref(nb)))
        per, nseg = C.c_size_t(), C.c_int64()
        check(lib().bq_grad_record_bytes(self.ptr, int(n_steps), int(checkpoint_every), C.byref(per), C.byref(nseg)))
        extra = (nseg.value if record_segments < 0 else record_segments) - 2
        work = torch.empty(nb.value + max(0, extra) * per.value, dtype=torch.uint8, device=self.pool.device)
        loss = (C.c_double * self.B)()
        g = (C.c_double * max(1, n.value))()
        check(lib().bq_grad(self.ptr, float(dt), int(n_steps), int(checkpoint_every), C.c_void_p(work.data_ptr()),
                            work.numel(), loss, g, _stream_ptr(stream)))
        return np.array(loss[:]), np.array(g[:n.value])

    def stage_variant(self) -> str:
        v = C.c_int()
        check(lib().bq_stage_variant(self.ptr, C.byref(v)))
        return {0: "generic", 1: "single_mode", 2: "pipelined"}[v.value]

    def solve_eligible(self) -> bool:
        e = C.c_int()
        check(lib().bq_solve_eligible(self.ptr, C.byref(e)))
        return bool(e.value)

    @staticmethod
    def _tune_dict(t: "bq_tune") -> dict:
        return dict(stage_path=PATH[t.stage_path], pipe_slots=t.pipe_slots, pipe_ctas_per_sm=t.pipe_ctas_per_sm,
                    solve_kernel=SOLVE_KERNEL[t.solve_kernel], solve_ctas_per_sm=t.solve_ctas_per_sm,
                    n_candidates=t.n_candidates, step_us=t.step_us, solve_us=t.solve_us, tile=t.tile, lanes=t.lanes,
                    gread=t.gread, grad_coop=t.grad_coop, grad_us=t.grad_us, pipe_fused=t.pipe_fused)

    def get_tune(self) -> dict:
        t = bq_tune()
        check(lib().bq_get_tune(self.ptr, C.byref(t)))
        return self._tune_dict(t)

    def set_tune(self, **kw):
        """Sets schedules (keys of get_tune(); unspecified keys keep their current value)."""
        t = bq_tune()
        check(lib().bq_get_tune(self.ptr, C.byref(t)))
        inv_path = {v: k for k, v in PATH.items()}
        inv_solve = {v: k for k, v in SOLVE_KERNEL.items()}
        for k, v in kw.items():
            if k == "stage_path":
                v = inv_path[v]
            elif k == "solve_kernel":
                v = inv_solve[v]
            setattr(t, k, v)
        check(lib().bq_set_tune(self.ptr, C.byref(t)))

    def autotune(self, dt: float, trial_steps: int = 8, stream=None) -> dict:
        """Measures the available schedules on this state (restored afterwards) and keeps the
        fastest (bq_autotune); returns the chosen schedules and their per-step times."""
        import torch
        nb = C.c_size_t()
        check(lib().bq_autotune_scratch_bytes(self.ptr, C.byref(nb)))
        scratch = torch.empty(nb.value, dtype=torch.uint8, device=self.pool.device)
        t = bq_tune()
        check(lib().bq_autotune(self.ptr, float(dt), int(trial_steps), C.c_void_p(scratch.data_ptr()), nb.value,
                                _stream_ptr(stream), C.byref(t)))
        return self._tune_dict(t)

    def autotune_grad(self, dt: float, trial_steps: int = 64, checkpoint_every: int = 32, stream=None) -> dict:
        """Measures the tiled schedules on bq_grad itself (bq_autotune_grad) and keeps the
        fastest; returns the chosen schedules and the trial gradient's time per step."""
        import torch
        nb = C.c_size_t()
        check(lib().bq_grad_required_bytes(self.ptr, int(trial_steps), int(checkpoint_every), C.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=self.pool.device)
        t = bq_tune()
        check(lib().bq_autotune_grad(self.ptr, float(dt), int(trial_steps), int(checkpoint_every),
                                     C.c_void_p(work.data_ptr()), nb.value, _stream_ptr(stream), C.byref(t)))
        return self._tune_dict(t)

    def step_fixed_scratch(self, dt: float, n_steps: int, stream=None):
        """bq_step with the RK4 scratch in the library's fixed device array (no allocation)."""
        check(lib().bq_step_fixed_scratch(self.ptr, float(dt), int(n_steps), _stream_ptr(stream)))

    def time(self) -> float:
        t = C.c_double()
        check(lib().bq_time(self.ptr, C.byref(t)))
        return t.value

    def evaluate(self, stream=None) -> np.ndarray:
        out = (C.c_double * (2 * self.B))()
        check(lib().bq_evaluate(self.ptr, out, _stream_ptr(stream)))
        a = np.frombuffer(out, dtype=np.float64).copy()
        return a[0::2] + 1j * a[1::2]

    def evaluate_async(self, out_ptr: int, stream=None) -> None:
        """bq_evaluate_async: Re, Im of Tr(rho0_b A_b) (2 B doubles) into device or pinned host
        memory at out_ptr, enqueued on stream without synchronising."""
        check(lib().bq_evaluate_async(self.ptr, C.c_void_p(out_ptr), _stream_ptr(stream)))

    def fock_block(self, lo: int = 3, dim: Optional[int] = None, stream=None) -> np.ndarray:
        if dim is None:
            raise ValueError("dim (prod_j min(3, M_j)) is required")
        out = (C.c_double * (2 * self.B * dim * dim))()
        check(lib().bq_fock_block(self.ptr, lo, out, _stream_ptr(stream)))
        a = np.frombuffer(out, dtype=np.float64).copy()
        return (a[0::2] + 1j * a[1::2]).reshape(self.B, dim, dim)

    def state_bytes(self) -> int:
        n = C.c_size_t()
        check(lib().bq_state_bytes(self.ptr, C.byref(n)))
        return n.value

    def store_state(self, host_ptr: int, stream=None):
        check(lib().bq_store_state(self.ptr, C.c_void_p(host_ptr), _stream_ptr(stream)))

    def load_state(self, host_ptr: int, stream=None):
        check(lib().bq_load_state(self.ptr, C.c_void_p(host_ptr), _stream_ptr(stream)))

    def set_time(self, tau: float):
        check(lib().bq_set_time(self.ptr, float(tau)))

    def n_systems(self) -> int:
        n = C.c_int()
        check(lib().bq_state_info(self.ptr, C.byref(n), None))
        return n.value

    def system_info(self, sys: int) -> dict:
        prob, p, q = C.c_int(), C.c_int(), C.c_int()
        ngx, ngy, nr = C.c_int64(), C.c_int64(), C.c_int64()
        w, c = (C.c_double * 2)(), (C.c_double * 2)()
        check(lib().bq_system_info(self.ptr, sys, C.byref(prob), C.byref(p), C.byref(q), C.byref(ngx),
                                   C.byref(ngy), C.byref(nr), w, c))
        return dict(problem=prob.value, p=p.value, q=q.value, n_gx=ngx.value, n_gy=ngy.value, n_r=nr.value,
                    weight=complex(w[0], w[1]), C=complex(c[0], c[1]))

    def read_system(self, sys: int, stream=None):
        info = self.system_info(sys)
        bufs = []
        for n in (info["n_gx"], info["n_gy"], info["n_r"]):
            bufs.append((C.c_double * (2 * n))() if n else None)
        check(lib().bq_read_system(self.ptr, sys, bufs[0], bufs[1], bufs[2], _stream_ptr(stream)))
        out = []
        for b in bufs:
            if b is None:
                out.append(None)
            else:
                a = np.frombuffer(b, dtype=np.float64).copy()
                out.append(a[0::2] + 1j * a[1::2])
        return info, out[0], out[1], out[2]


def launch_count() -> int:
    return int(lib().bq_launch_count())


def fma_peak_count(iters: int) -> float:
    """FMA instructions one bq_fma_peak run of `iters` iterations executes on this GPU (4 CTAs
    of 256 threads per SM, 16 chains of 8 FMAs per iteration)."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return float(nsm * 4 * 256 * 16 * 8 * iters)


def fma_peak(dtype: str = "f64", iters: int = 4096, stream=None) -> float:
    """Measured FMA instructions per second of the current GPU (bq_fma_peak)."""
    out = C.c_double()
    check(lib().bq_fma_peak(DTYPE[dtype], int(iters), C.byref(out), _stream_ptr(stream)))
    return out.value
