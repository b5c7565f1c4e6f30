"""Benchmark of the mapped adjoint-Lindblad solver on GB300.

Default workload (N = 1 GPU): a batch of driven, damped Kerr oscillators drawn from the
seeded 4096-instance distribution (``workloads.configs.kerr_batch``: Delta, K, gamma, drive
peak, measured level n in {0,1,2}, truncation N in 10..40), scaled to 65 536 instances so
that the state (4 arrays x ~0.4 GB in complex FP32) is far larger than the 129 MB L2 and
the fused RK4 stage kernel streams from HBM.  One bench *step* is one classical RK4 time
step (dt = 0.002 ns; four fused stage kernels: drive envelopes, stencils, separable
source, RK4 combine) of every instance followed by the per-instance observable
Tr(rho0 A) (warp reductions).  ``value`` = grid-point RK-stage updates per second.

Other keys: ``roofline`` (the stage kernel against the measured HBM copy bandwidth),
``e2e`` (the same step through the C ABI with the state loaded from pinned host memory
and the observables read back every step), ``cpu_baseline`` (the FP64 oracle timed on a
bounded sample of the same workload on the host cores), ``clocks`` (nvidia-smi sampled
during the timed region), ``gpu_launches`` (library kernel launches in the timed region),
``batched`` (4096 full-horizon solves: one persistent launch vs streamed stage kernels vs
one instance per launch), ``grads`` (the 131-parameter control gradient, and 16 control
problems batched in one state vs one problem per state), ``methods`` (memory and time per
step, and accuracy, of the conventional number-basis method vs the mapping with full R, with
R kept at k = l and with R = 0, on secular-dissipator instances),
``secular`` (the paper's secular dissipator on the same instances: updates/s and HBM GB/s),
``fig2`` (Fig. 2's right panels: Table I networks of 1-3 oscillators, truncation tuned to
epsilon_r <= 1e-4 per method, stored elements and time per step; ``--only-fig2`` adds four
oscillators and the left panels, against scaled time), and ``config.schedule`` (the
schedule bq_autotune picked for the timed state).  The gradient legs tune their states with
bq_autotune_grad (``--grad-tune TILE,LANES,GREAD`` fixes the schedule instead).

``--impl reference`` times the oracle (the plain FP64 CPU implementation) on the same
workload, each step a bounded sample.  Multi-GPU: every rank solves its own shard of
independent instances (replicas, weak scaling); no collective is on the data path.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-point RK-stage updates/s"
DT = 0.002
HORIZON = 100.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--instances", type=int, default=65536, help="instances per GPU")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 4096-instance full-solve leg")
    ap.add_argument("--no-grads", action="store_true", help="skip the adjoint-gradient leg")
    ap.add_argument("--only-solve", action="store_true",
                    help="profiling aid: only the persistent batched solve of --instances for --solve-steps steps")
    ap.add_argument("--solve-steps", type=int, default=2000)
    ap.add_argument("--only-grad", action="store_true",
                    help="profiling aid: only the adjoint gradient of the control problem for --grad-steps steps")
    ap.add_argument("--grad-steps", type=int, default=None)
    ap.add_argument("--only-fig2", action="store_true", help="profiling aid: only the Fig. 2 leg")
    ap.add_argument("--grad-tune", default=None, metavar="TILE,LANES,GREAD",
                    help="profiling aid: tiled schedule of the gradient leg's state instead of the autotuned one")
    ap.add_argument("--no-autotune", action="store_true",
                    help="profiling aid: keep the default schedule of the timed state (no tuning launches)")
    ap.add_argument("--n-range", type=int, nargs=2, default=(10, 40), metavar=("LO", "HI"),
                    help="profiling aid: Fock truncation range of the kerr_batch instances (default 10 40)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_range(n_inst: int, rank: int):
    """Indices of the seeded kerr_batch stream solved by this rank (rank-major shards of
    n_inst instances: replicas with no exchange between ranks)."""
    return range(n_inst * rank, n_inst * (rank + 1))


N_RANGE = (10, 40)  # Fock truncation range of the instances (--n-range)

# Floating-point operations per grid-point RK stage of the merged stencil on this workload (an
# FMA counts two): diagonal (2 + 6), four neighbour terms (4 x 8), one sandwich term with its
# separable source (18), the RK4 combine (13 on average over the four stages).
FLOP_PER_POINT_STAGE = 70

# DRAM traffic of the fused step kernel per launch (one RK4 step), from one ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum on the default workload (65 536 instances,
# N 10..40, complex FP32); reported only while the kernel's definition is the one that was
# measured and the workload and schedule are the default ones.
STAGE_TRAFFIC = {"kernel": "k_steps_pipe", "kernel_sha256": "949f8d985de5897de22854d894da70500ec858ba4f77546fd9882996cfca5a19",
                 "instances": 65536, "n_range": (10, 40), "dtype": "f32", "bytes_per_launch": 7.575e9}


def stage_kernel_sha256(names=("pipe_stage", "pipe_combine", "k_steps_pipe")) -> str:
    """sha256 of the definitions (each from its template line to the closing brace at column
    0) of the functions that make up the measured kernel, in bq_kernels.cu."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2203_05526_gb300", "csrc", "bq_kernels.cu")).read()
    h = hashlib.sha256()
    for name in names:
        a = src.index(f" {name}(")
        a = src.rindex("\ntemplate", 0, a) + 1
        b = src.index("\n}\n", a) + 3
        h.update(src[a:b].encode())
    return h.hexdigest()


def measured_traffic(instances: int, dtype: str, schedule: dict):
    t = STAGE_TRAFFIC
    if t["bytes_per_launch"] is None or stage_kernel_sha256() != t["kernel_sha256"]:
        return None
    if instances != t["instances"] or tuple(N_RANGE) != t["n_range"] or dtype != t["dtype"]:
        return None
    if (schedule["stage_path"], schedule["pipe_slots"], schedule["pipe_ctas_per_sm"]) != ("pipe", 2, 0):
        return None  # captured with the default schedule
    return t["bytes_per_launch"]


def workload(n_inst: int, rank: int):
    """Instances of this rank: the seeded stream of kerr_batch, rank-major shards."""
    from workloads import configs
    r = shard_range(n_inst, rank)
    allp = configs.kerr_batch(B=r.stop, T=HORIZON, dt=DT, n_min=N_RANGE[0], n_max=N_RANGE[1])
    return allp[r.start:r.stop]


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """Slowest rank's time (the job's time); a no-op for one rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def configs_batch(n: int):
    from workloads import configs
    return configs.kerr_batch(B=n, T=HORIZON, dt=DT, n_min=N_RANGE[0], n_max=N_RANGE[1])


def points_of(specs):
    """(R + G_x + G_y) grid points per instance (grid = Fock truncation)."""
    tot = 0
    for p in specs:
        n = p.N[0]
        tot += n * n + 2 * n
    return tot


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux
        return os.cpu_count() or 1


def _oracle_task(args):
    """One oracle solve (oracle.mapping.rk4_mapped, FP64) of instance `index` of the seeded
    batch for n_steps steps; returns (grid-point RK-stage updates, seconds)."""
    index, n_inst, n_steps, n_range = args
    from oracle import mapping
    from workloads import configs
    p = configs.kerr_batch(B=index + 1, T=HORIZON, dt=DT, n_min=n_range[0], n_max=n_range[1])[index]
    t0 = time.perf_counter()
    mapping.rk4_mapped(p, n_steps=n_steps)
    return points_of([p]) * 4 * n_steps, time.perf_counter() - t0


def _pool_init():
    os.environ["OMP_NUM_THREADS"] = "1"


def oracle_throughput(indices, n_range, n_steps: int, budget_s: float):
    """The FP64 oracle on every host core: a spawn process pool (one single-threaded worker
    per core) runs instances of the seeded batch in order, n_steps RK4 steps each, until about
    budget_s of wall time; returns (updates/s, cores, instances done, wall seconds)."""
    import multiprocessing as mp
    cores = host_cores()
    env0 = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env0:
        os.environ[k] = "1"  # the workers inherit single-threaded BLAS
    try:
        ctx = mp.get_context("spawn")
        done_pts, done = 0, 0
        with ctx.Pool(cores, initializer=_pool_init) as pool:
            tasks = [(i, max(indices) + 1, n_steps, tuple(n_range)) for i in indices]
            t0 = time.perf_counter()
            for pts, _ in pool.imap(_oracle_task, tasks):
                done_pts += pts
                done += 1
                if time.perf_counter() - t0 > budget_s and done >= cores:
                    break
            el = time.perf_counter() - t0
            pool.terminate()
    finally:
        for k, v in env0.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return done_pts / el, cores, done, el


def cpu_baseline(n_inst: int, budget_s: float = 15.0):
    """The FP64 oracle (oracle.mapping.rk4_mapped) on a bounded sample of the same workload:
    instances of the seeded batch taken in order, 100 RK4 steps each, on every host core."""
    n_steps = 100
    v, cores, done, el = oracle_throughput(range(min(n_inst, 4096)), N_RANGE, n_steps, budget_s)
    return {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{done} instances x {n_steps} RK4 steps (FP64, numpy, one single-threaded process per core "
                      f"on {cores} cores), {el:.1f} s"}


class Clocks:
    def __init__(self):
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        self.p = None

    def start(self, gpu: int):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


E2E_PARTS = 4


def e2e_leg(specs, opts, schedule: dict, steps: int, world: int, barrier):
    """The headline step end to end through the C ABI, every step uploading the whole state
    from pinned host memory and reading every instance's Tr(rho0 A) back: the batch as
    E2E_PARTS states on as many streams, pipelined (while one part is stepped, the next part's
    input is uploaded and the previous part's result is read back)."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    cut = [len(specs) * i // E2E_PARTS for i in range(E2E_PARTS + 1)]
    parts = [specs[cut[i]:cut[i + 1]] for i in range(E2E_PARTS)]
    sts = [bq.State([bq.problem_from_spec(p) for p in part], opts) for part in parts]
    for st in sts:
        st.set_tune(stage_path=schedule["stage_path"], pipe_slots=schedule["pipe_slots"],
                    pipe_ctas_per_sm=schedule["pipe_ctas_per_sm"])
    streams = [torch.cuda.Stream() for _ in parts]
    hosts = []
    for st in sts:
        h = torch.empty(st.state_bytes(), dtype=torch.uint8, pin_memory=True)
        st.store_state(h.data_ptr())
        hosts.append(h)
    torch.cuda.synchronize()

    outs = [torch.empty(2 * len(part), dtype=torch.float64, pin_memory=True) for part in parts]

    def run(n):
        # per step and part: upload the state, one RK4 step, Tr(rho0 A) of every instance back
        # to pinned host memory, all enqueued on the part's stream (no host wait inside)
        for _ in range(n):
            for h in range(len(parts)):
                sts[h].load_state(hosts[h].data_ptr(), stream=streams[h])
                sts[h].step(DT, 1, stream=streams[h])
                sts[h].evaluate_async(outs[h].data_ptr(), stream=streams[h])

    run(2)
    barrier()
    cur = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for sm in streams:
        sm.wait_event(e0)
    run(steps)
    for sm in streams:
        ev = torch.cuda.Event()
        ev.record(sm)
        cur.wait_event(ev)
    e1.record(cur)
    barrier()
    ms = e0.elapsed_time(e1)
    for h in range(len(parts)):
        ref = sts[h].evaluate(stream=streams[h])  # synchronising read: error word, finiteness
        assert np.array_equal(outs[h].numpy(), np.stack([ref.real, ref.imag], 1).ravel())
    pts = points_of(specs)
    return {"value": world * 4 * pts * steps / (ms / 1e3), "unit": METRIC,
            "h2d_bytes_per_step": sum(st.state_bytes() for st in sts), "d2h_bytes_per_step": 16 * len(specs),
            "how": f"{E2E_PARTS} states of a quarter of the batch each on as many streams, the upload of one part "
                   "overlapped with the other parts' steps; observables read back with bq_evaluate_async into "
                   "pinned host memory"}


def alu_peaks():
    """Measured FMA throughput of this GPU in FP32 and FP64 (bq_fma_peak: independent FMA
    chains on every SM, CUDA events, at the clocks the GPU runs), each the best of three runs
    of about 0.2 s."""
    import paper_2203_05526_gb300 as bq
    out = {}
    for dt, it in (("f32", 1 << 14), ("f64", 1 << 8)):
        v = bq.fma_peak(dt, it)
        n_fma = bq.fma_peak_count(it)
        it2 = max(1, int(it * 0.2 / (n_fma / v)))
        best = max(bq.fma_peak(dt, it2) for _ in range(3))
        out[f"{'fp32' if dt == 'f32' else 'fp64'}_fma_per_s"] = best
        out[f"{'fp32' if dt == 'f32' else 'fp64'}_tflops"] = 2 * best / 1e12
    out["how"] = "bq_fma_peak: 16 dependent FMA chains per thread, 4 CTAs of 256 threads per SM, best of 3 x ~0.2 s"
    return out


def fp64_leg(n_inst: int, peaks: dict, steps: int = 5, warmup: int = 3):
    """The headline workload in complex FP64: stage-kernel time per RK4 step, updates/s, and
    the two roofs that could bind it (HBM on 64 B per grid-point stage; the measured FP64 FMA
    rate on FLOP_PER_POINT_STAGE); GB300's FP64 pipe makes the latter bind."""
    import torch

    import paper_2203_05526_gb300 as bq
    specs = configs_batch(n_inst)
    st = bq.State([bq.problem_from_spec(p) for p in specs], bq.map_opts(method="mapped", dtype="f64", horizon=HORIZON,
                                                                            dt=DT))
    pts = points_of(specs)
    for _ in range(warmup):
        st.step(DT, 1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.step(DT, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    s_per_step = e0.elapsed_time(e1) / 1e3 / steps
    ups = 4 * pts / s_per_step
    hbm = 64 * ups / 1e9
    flops = FLOP_PER_POINT_STAGE * ups
    f64_peak = 2 * peaks.get("fp64_fma_per_s", float("nan"))
    hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    roofs = {"hbm": {"achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": hbm / hbm_peak},
             "fp64_alu": {"achieved": flops / 1e12, "peak": f64_peak / 1e12, "unit": "TFLOP/s",
                          "frac": flops / f64_peak}}
    bound = max(roofs, key=lambda k: roofs[k]["frac"])
    return {"workload": f"kerr_batch x{n_inst}, complex FP64, {steps} RK4 steps", "ms_per_step": 1e3 * s_per_step,
            "updates_per_s": ups, "stage_path": st.get_tune()["stage_path"], "roofs": roofs, "bound": bound}


def batched_leg(world: int):
    """The 4096-instance batch itself (seed 20220311, complex FP32, T = 100 ns, dt = 0.002 ns,
    50 000 RK4 steps): full solves through the persistent one-launch path (bq_solve), through
    the streamed stage kernels (bq_step, CUDA-graph replays), and the plain
    one-instance-per-launch path (each instance its own state and launches), the latter timed
    on a sample of instances and steps and scaled to the full batch."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    specs = configs.kerr_batch(B=4096, T=HORIZON, dt=DT)
    n_steps = specs[0].n_steps
    pts = points_of(specs)
    opts = bq.map_opts(method="mapped", dtype="f32", horizon=HORIZON, dt=DT)
    handles = [bq.problem_from_spec(p) for p in specs]
    out = {"workload": "kerr_batch 4096 instances, complex FP32, T=100 ns, dt=0.002 ns (50000 RK4 steps)"}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    st = bq.State(handles, opts)
    st.solve(DT, 200)  # warm-up
    st = bq.State(handles, opts)
    out["schedule"] = st.autotune(DT, trial_steps=20)  # bq_autotune: state restored afterwards
    if out["schedule"]["solve_kernel"] == "step":  # bq_solve would step: time the persistent kernel
        st.set_tune(solve_kernel="merged" if st.solve_eligible() else "program")
    out["persistent_kernel"] = st.get_tune()["solve_kernel"]
    n0 = bq.launch_count()
    t_solve = timed(lambda: st.solve(DT, n_steps))
    launches = bq.launch_count() - n0
    ev = st.evaluate()
    out["persistent"] = {"seconds": t_solve, "solves_per_s": 4096 / t_solve,
                         "updates_per_s": 4 * pts * n_steps / t_solve, "launches": launches,
                         "finite": bool(np.all(np.isfinite(ev)))}
    st2 = bq.State(handles, opts)
    st2.step(DT, 128)
    st2 = bq.State(handles, opts)
    st2.autotune(DT, trial_steps=8)
    t_step = timed(lambda: st2.step(DT, n_steps))
    out["streamed"] = {"seconds": t_step, "solves_per_s": 4096 / t_step,
                       "updates_per_s": 4 * pts * n_steps / t_step,
                       "launches_per_step": 1 if st2.get_tune()["pipe_fused"] else 4}
    out["bq_solve_path"] = out["schedule"]["solve_kernel"]  # what bq_solve runs after bq_autotune
    # one instance per launch: 16 sampled instances, 2000 steps each, scaled
    sample = list(range(0, 4096, 256))
    sample_steps = 2000
    tot = 0.0
    for i in sample:
        s1 = bq.State([handles[i]], opts)
        s1.step(DT, 64)
        tot += timed(lambda: s1.step(DT, sample_steps)) * (n_steps / sample_steps)
    per_inst = tot / len(sample)
    out["one_instance_per_launch"] = {"seconds_per_instance_solve": per_inst, "solves_per_s": 1.0 / per_inst,
                                      "sample": f"instances {sample[0]}..{sample[-1]} step 256, {sample_steps} of "
                                                f"{n_steps} steps each, scaled"}
    out["persistent_vs_one_per_launch"] = out["persistent"]["solves_per_s"] / out["one_instance_per_launch"]["solves_per_s"]
    return out


def grads_leg(n_steps=None, sched=None):
    """Gradient of P(|1,0>) at T = 200 ns for the two-mode control problem (64 complex
    piecewise-constant drive segments, K_1, K_2, g: 131 real parameters; 20 480 RK4 steps,
    complex FP64, checkpoint every 160 steps) by the discrete adjoint kernels (bq_grad)."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    p = configs.two_mode_control()
    st = bq.State([bq.problem_from_spec(p)], bq.map_opts(dtype="f64", horizon=p.T, dt=p.dt))
    if sched is None:
        tune = st.autotune_grad(p.dt, trial_steps=64, checkpoint_every=32)  # measured on the gradient itself
    else:
        st.set_tune(tile=sched[0], lanes=sched[1], gread=sched[2])
        tune = st.get_tune()
    st.grad(p.dt, 320, 160)  # warm-up (modules, workspace)
    torch.cuda.synchronize()
    steps = p.n_steps if n_steps is None else n_steps
    t0 = time.perf_counter()
    loss, g = st.grad(p.dt, steps, 160)
    el = time.perf_counter() - t0
    out = {"workload": f"two_mode_control: 2 modes x M=12, 64 pwc segments, 131 parameters, {steps} RK4 steps, "
                       "checkpoint every 160, complex FP64",
           "seconds_per_gradient": el, "grads_per_s": 1.0 / el, "loss": float(loss[0]),
           "grad_norm": float(np.linalg.norm(g)), "n_params": int(g.size), "tile": tune["tile"],
           "lanes": tune["lanes"], "gread": tune["gread"], "grad_coop": tune["grad_coop"],
           "tuned_on": "gradient" if sched is None else "fixed"}
    # the same gradient with a workspace that holds every segment's recording (GB300's HBM:
    # 4 x 20 480 states of 0.34 MB = 27.5 GB), so that no segment is recomputed
    per, nseg = bq.grad_record_bytes(st, steps, 160)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss_r, g_r = st.grad(p.dt, steps, 160, record_segments=-1)
    el_r = time.perf_counter() - t0
    out["all_segments_recorded"] = {
        "seconds_per_gradient": el_r, "grads_per_s": 1.0 / el_r, "recording_bytes": per * nseg,
        "max_rel_diff": float(np.max(np.abs(g_r - g)) / np.max(np.abs(g)))}
    if n_steps is None:
        out["batched"] = grads_batched_leg()
    return out


def grads_batched_leg(B: int = 16, steps: int = 1280):
    """Gradients of B control problems (drive amplitudes from seeds 5526 + b) in one state
    (one set of adjoint launches for the whole batch) against one problem per state (the
    plain one-instance-per-launch path), over the first `steps` RK4 steps, same arithmetic."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    probs = [configs.two_mode_control(seed=5526 + b) for b in range(B)]
    dt = probs[0].dt
    opts = bq.map_opts(dtype="f64", horizon=probs[0].T, dt=dt)
    stB = bq.State([bq.problem_from_spec(q) for q in probs], opts)
    tuneB = stB.autotune_grad(dt, trial_steps=64, checkpoint_every=32)
    stB.grad(dt, 160, 160)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lossB, gB = stB.grad(dt, steps, 160)
    tB = time.perf_counter() - t0
    t1 = 0.0
    worst = 0.0
    # one problem per state: the schedule tuned on the first such state serves all of them
    tune1 = bq.State([bq.problem_from_spec(probs[0])], opts).autotune_grad(dt, trial_steps=64, checkpoint_every=32)
    n_per = gB.size // B
    for b, q in enumerate(probs):
        st1 = bq.State([bq.problem_from_spec(q)], opts)
        st1.set_tune(tile=tune1["tile"], lanes=tune1["lanes"], gread=tune1["gread"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        l1, g1 = st1.grad(dt, steps, 160)
        t1 += time.perf_counter() - t0
        ref = gB[b * n_per:(b + 1) * n_per]
        worst = max(worst, float(np.max(np.abs(g1 - ref)) / max(float(np.max(np.abs(ref))), 1e-300)))
    return {"workload": f"{B} two_mode_control problems (seeds 5526..{5526 + B - 1}), first {steps} RK4 steps, "
                        "checkpoint every 160, complex FP64",
            "batched_grads_per_s": B / tB, "one_instance_per_launch_grads_per_s": B / t1,
            "batched_vs_one_per_launch": t1 / tB, "max_rel_diff_batched_vs_single": worst,
            "tile_batched": tuneB["tile"], "lanes_batched": tuneB["lanes"], "gread_batched": tuneB["gread"]}


def methods_leg(B: int = 1024, Ns=(10, 20, 40), steps: int = 100, acc_steps: int = 50000):
    """The paper's memory, time and accuracy comparison (Fig. 2's quantities) on this GPU:
    B driven Kerr oscillators with the secular dissipator (secular_batch draws at truncation
    N) integrated by the conventional number-basis method (N^2 elements per instance), the
    mapping with the full residual R (2N + N^2), with the residual kept as a function of x y
    only (R diagonal: 3N; the paper's observation) and with R = 0 (2N).  Complex FP32,
    schedules autotuned; device time per RK4 step of the whole batch; epsilon_r (the paper's
    relative error on the three-level block) of instance 0 after acc_steps steps against the
    conventional method at truncation N + 8 with half the time step in FP64."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    methods = (("direct", dict(method="direct")), ("mapped_full_R", dict(method="mapped")),
               ("mapped_R_diag", dict(method="mapped", r_layout="diag")),
               ("mapped_R_off", dict(method="mapped", r_layout="off")))
    rows = []
    for N in Ns:
        specs = configs.secular_batch(B=B, T=HORIZON, dt=DT, n_min=N, n_max=N)
        handles = [bq.problem_from_spec(p) for p in specs]
        # reference block of instance 0: conventional method, N + 8, dt / 2, FP64
        ref_spec = configs.secular_batch(B=1, T=HORIZON, dt=DT, n_min=N + 8, n_max=N + 8)[0]
        ref_spec.N = (N + 8,)
        ref = bq.State([bq.problem_from_spec(ref_spec)], bq.map_opts(method="direct", dtype="f64",
                                                                       horizon=HORIZON, dt=DT / 2))
        ref.step(DT / 2, 2 * acc_steps)
        bref = ref.fock_block(3, dim=3)[0]
        for name, kw in methods:
            st = bq.State(handles, bq.map_opts(dtype="f32", horizon=HORIZON, dt=DT, **kw))
            st.autotune(DT, trial_steps=4)
            st.step(DT, 8)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.step(DT, steps)
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / steps
            one = bq.State([handles[0]], bq.map_opts(dtype="f32", horizon=HORIZON, dt=DT, **kw))
            one.step(DT, acc_steps)
            blk = one.fock_block(3, dim=3)[0]
            eps = float(np.linalg.norm(blk - bref) / np.linalg.norm(bref))
            rows.append({"N": N, "method": name, "elements_per_instance": st.state_bytes() / 8 / B,
                         "state_bytes": st.state_bytes(), "us_per_step": us, "ns_per_instance_step": 1e3 * us / B,
                         "eps_r_instance0": eps})
    return {"workload": f"{B} secular_batch instances per N (kerr_batch draws with the secular dissipator, "
                        f"fixed N), complex FP32, {steps} timed RK4 steps of dt={DT} ns; eps_r of instance 0 "
                        f"after {acc_steps} steps vs the conventional method at N + 8, dt/2, FP64",
            "rows": rows}


def fig2_left_leg(modes=(1, 2), times=(2.0, 5.0, 10.0, 20.0, 40.0), target: float = 1e-4, steps_per_unit: int = 200,
                  n_max: int = 16):
    """The paper's Fig. 2 (left panels) on this GPU: the same Table I networks for one and two
    oscillators as functions of the scaled time omega_q t / pi.  For every time and method the
    smallest truncation with epsilon_r <= `target` against the conventional method at a
    larger truncation with half the time step (FP64, the same step size at every time), its
    stored elements (largest over the run: the state is allocated once) and its device time per
    RK4 step."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    ref_n = {1: 20, 2: 13}
    rows = []

    def run(p, dt, n, **kw):
        st = bq.State([bq.problem_from_spec(p)], bq.map_opts(dtype="f64", horizon=p.T, dt=dt, **kw))
        st.step(dt, n)
        torch.cuda.synchronize()
        return st

    for nm in modes:
        for tsc in times:
            steps = int(round(steps_per_unit * tsc))
            pr = configs.table_one_network(nm, ref_n[nm], scaled_time=tsc, steps=2 * steps)
            ref = run(pr, pr.dt, 2 * steps, method="direct").fock_block(3, dim=3 ** nm)[0]
            for name, kw in (("conventional", dict(method="direct")), ("mapping_R_diag", dict(r_layout="diag")),
                             ("mapping_R_off", dict(r_layout="off"))):
                found = None
                for N in range(3, min(n_max, ref_n[nm] - 1) + 1):
                    p = configs.table_one_network(nm, N, scaled_time=tsc, steps=steps)
                    st = run(p, p.dt, steps, **kw)
                    blk = st.fock_block(3, dim=3 ** nm)[0]
                    eps = float(np.linalg.norm(blk - ref) / np.linalg.norm(ref))
                    if eps <= target:
                        found = (N, p, st, eps)
                        break
                if found is None:
                    rows.append({"modes": nm, "scaled_time": tsc, "method": name, "truncation": None})
                    continue
                N, p, st, eps = found
                st.autotune(p.dt, trial_steps=10)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st.step(p.dt, 200)
                e1.record()
                torch.cuda.synchronize()
                n_sys = st.n_systems()
                rows.append({"modes": nm, "scaled_time": tsc, "method": name, "truncation": N, "eps_r": eps,
                             "systems": n_sys, "elements_per_system": st.state_bytes() / 16 / n_sys,
                             "elements_total": st.state_bytes() / 16, "us_per_step": e0.elapsed_time(e1) * 1e3 / 200})
    return {"workload": "Table I network, lab frame, secular dissipator at T_E = 0, A(0) = a_1 x ... x a_n, "
                        f"scaled times {list(times)} at {steps_per_unit} RK4 steps per unit, complex FP64; "
                        f"truncation tuned to eps_r <= {target:g}", "rows": rows}


def fig2_leg(modes=(1, 2, 3), target: float = 1e-4, steps: int = 2000, n_max: int = 12):
    """The paper's Fig. 2 (right panels) on this GPU: the Table I network of n coupled
    driven anharmonic oscillators in the lab frame (secular dissipator, A(0) = a_1 (x) ... (x)
    a_n) at the scaled time omega_q t / pi = 10.  For each method the smallest truncation
    whose epsilon_r (three-level block) against a reference (conventional method, larger
    truncation, half the time step, FP64) is at most `target`; then its stored elements
    (conventional: N^(2n); mapping: per initial condition and in total) and its device time
    per RK4 step (FP64)."""
    import numpy as np
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    ref_n = {1: 14, 2: 10, 3: 8, 4: 7}
    rows = []

    def run(p, dt, n, **kw):
        st = bq.State([bq.problem_from_spec(p)], bq.map_opts(dtype="f64", horizon=p.T, dt=dt, **kw))
        st.step(dt, n)
        torch.cuda.synchronize()
        return st

    for nm in modes:
        pr = configs.table_one_network(nm, ref_n[nm], steps=2 * steps)
        ref = run(pr, pr.dt, 2 * steps, method="direct").fock_block(3, dim=3 ** nm)[0]
        for name, kw in (("conventional", dict(method="direct")), ("mapping_R_diag", dict(r_layout="diag")),
                         ("mapping_R_off", dict(r_layout="off"))):
            found = None
            for N in range(3, n_max + 1):
                if N >= ref_n[nm]:
                    break
                p = configs.table_one_network(nm, N, steps=steps)
                st = run(p, p.dt, steps, **kw)
                blk = st.fock_block(3, dim=3 ** nm)[0]
                eps = float(np.linalg.norm(blk - ref) / np.linalg.norm(ref))
                if eps <= target:
                    found = (N, p, st, eps)
                    break
            if found is None:
                rows.append({"modes": nm, "method": name, "truncation": None})
                continue
            N, p, st, eps = found
            tune = st.autotune(p.dt, trial_steps=10)  # restores the state; keeps the fastest schedule
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.step(p.dt, 200)
            e1.record()
            torch.cuda.synchronize()
            n_sys = st.n_systems()
            per_sys = st.state_bytes() / 16 / n_sys
            rows.append({"modes": nm, "method": name, "truncation": N, "eps_r": eps, "systems": n_sys,
                         "elements_per_system": per_sys, "elements_total": st.state_bytes() / 16,
                         "conventional_elements": N ** (2 * nm), "us_per_step": e0.elapsed_time(e1) * 1e3 / 200,
                         "schedule": {k: tune[k] for k in ("stage_path", "tile", "lanes", "gread")}})
    return {"workload": f"Table I network, lab frame, secular dissipator at T_E = 0, A(0) = a_1 x ... x a_n, "
                        f"omega_q t / pi = 10 in {steps} RK4 steps, complex FP64; truncation tuned to "
                        f"eps_r <= {target:g}", "rows": rows}


def secular_leg(B: int = 32768, steps: int = 20):
    """The paper's secular dissipator (Eq. 203 / Eq. S9, zero temperature) on kerr_batch's
    instances (secular_batch: same draws, complex FP32): grid-point RK-stage updates/s of the
    stage kernel (the projector term is restricted to diagonal index pairs) and its HBM
    bandwidth on the algorithmic bytes of the headline roofline (16 array transfers per point
    and step), with the kernel's own transfer count beside it."""
    import torch

    import paper_2203_05526_gb300 as bq
    from workloads import configs
    specs = configs.secular_batch(B=B, T=HORIZON, dt=DT, n_min=N_RANGE[0], n_max=N_RANGE[1])
    st = bq.State([bq.problem_from_spec(p) for p in specs], bq.map_opts(dtype="f32", horizon=HORIZON, dt=DT))
    st.step(DT, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st.step(DT, steps)
    e1.record()
    torch.cuda.synchronize()
    s_step = e0.elapsed_time(e1) / 1e3 / steps
    pts = points_of(specs)
    achieved = 16 * 8 * pts / 4 / (s_step / 4) / 1e9
    variant = st.stage_variant()
    own = 18 if variant == "pipelined" else 19  # + the FP32 update's residual (and Kahan) transfers
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    return {"workload": f"secular_batch x{B} (kerr_batch draws, secular dissipator, T_E = 0), complex FP32, "
                        f"{steps} RK4 steps", "kernel": {"pipelined": "bq::k_stage_pipe", "single_mode": "bq::k_stage_m1",
                                               "generic": "bq::k_stage"}[variant],
            "updates_per_s": 4 * pts / s_step, "ms_per_step": 1e3 * s_step,
            "bytes_per_point_stage": 32, "kernel_transfers_per_step": own,
            "achieved_gbs": achieved, "frac_of_measured_hbm": achieved / peak}


def run_reference(args, rank, world):
    """The oracle arm: the plain FP64 CPU oracle on the same workload, on every host core (a
    spawn process pool), each step a bounded sample of instances of the seeded batch.  Under
    several ranks only rank 0 runs and prints."""
    if rank != 0:
        return
    n_steps = 20
    cores = host_cores()
    per_step = cores  # one instance per core per bench step
    for i in range(args.warmup):
        oracle_throughput(range(i * per_step, (i + 1) * per_step), N_RANGE, n_steps, 0.0)
    v, _, done, el = oracle_throughput(range(args.warmup * per_step, (args.warmup + args.steps) * per_step), N_RANGE,
                                       n_steps, 1e30)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"kerr_batch x{args.instances} (driven damped Kerr, seed 20220311)",
                                           "instances": args.instances, "dt_ns": DT},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} instances x {n_steps} RK4 steps per step, one single-threaded "
                                       f"process per core"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def launch_replicas(args) -> int:
    """`bench.py --gpus N` without a launcher: start N ranks on this node (one GPU each, the
    environment torchrun would give them, rendezvous at 127.0.0.1) and return the first
    non-zero exit status (rank 0 prints the JSON line)."""
    import socket
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    procs = []
    for r in range(args.gpus):
        env = {**os.environ, "RANK": str(r), "WORLD_SIZE": str(args.gpus), "LOCAL_RANK": str(r),
               "LOCAL_WORLD_SIZE": str(args.gpus), "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)}
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), *sys.argv[1:]], env=env))
    rc = 0
    for p in procs:
        p.wait()
        rc = rc or p.returncode
    return rc


def main():
    global N_RANGE
    args = parse()
    N_RANGE = (int(args.n_range[0]), int(args.n_range[1]))
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(launch_replicas(args))
    rank, world, local = dist_env()
    if world != args.gpus:
        sys.exit(f"bench.py: WORLD_SIZE={world} but --gpus {args.gpus}")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2203_05526_gb300 as bq
    from paper_2203_05526_gb300 import build
    build.build()
    if args.only_fig2:
        print(json.dumps({"only_fig2": True, "right": fig2_leg(modes=(1, 2, 3, 4)), "left": fig2_left_leg()}))
        return
    if args.only_grad:
        sched = None if args.grad_tune is None else [int(v) for v in args.grad_tune.split(",")]
        print(json.dumps({"only_grad": True, **grads_leg(args.grad_steps, sched)}))
        return
    if args.only_solve:
        specs = configs_batch(args.instances)
        st = bq.State([bq.problem_from_spec(p) for p in specs], bq.map_opts(dtype=args.dtype, horizon=HORIZON, dt=DT))
        st.solve(DT, 10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.solve(DT, args.solve_steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        print(json.dumps({"only_solve": True, "instances": args.instances, "steps": args.solve_steps, "seconds": el,
                          "updates_per_s": 4 * points_of(specs) * args.solve_steps / el}))
        return
    specs = workload(args.instances, rank)
    handles = [bq.problem_from_spec(p) for p in specs]
    opts = bq.map_opts(method="mapped", dtype=args.dtype, horizon=HORIZON, dt=DT)
    state = bq.State(handles, opts)
    # bq_autotune picks bq_step's schedule (the state is restored afterwards)
    schedule = state.get_tune() if args.no_autotune else state.autotune(DT, trial_steps=6)
    pts = points_of(specs)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------------------
    for _ in range(args.warmup):
        state.step(DT, 1)
        state.evaluate()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # every step's Tr(rho0 A) of all instances goes to pinned host memory (bq_evaluate_async:
    # enqueued on the stream, so the host keeps the GPU fed instead of waiting for each read)
    obs_host = [torch.empty(2 * len(specs), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    clk = Clocks()
    clk.start(local)
    barrier()
    n_launch0 = bq.launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        state.step(DT, 1)
        ev[i][1].record(stream)
        state.evaluate_async(obs_host[i % 2].data_ptr(), stream)
    t1.record(stream)
    barrier()
    obs = state.evaluate()  # synchronising read: checks the device error word and finiteness
    assert np.array_equal(obs_host[(args.steps - 1) % 2].numpy(), np.stack([obs.real, obs.imag], 1).ravel())
    launches = bq.launch_count() - n_launch0
    clocks = clk.stop()
    ms = t0.elapsed_time(t1)
    stage_ms = sum(a.elapsed_time(b) for a, b in ev)
    ms = max_over_ranks(ms, world, device="cuda")
    assert np.all(np.isfinite(obs))
    upd_per_step = 4 * pts
    value = world * upd_per_step * args.steps / (ms / 1e3)

    # roofline of the fused stage kernel on the algorithmic bytes of classical RK4 streamed
    # stage by stage: 16 array transfers of one complex element per grid point and step
    # (stage 1: read y, write u and the stage sum; stages 2-3: read u, y and the sum, write u and
    # the sum; stage 4: read u and the sum, write y), 4 per stage launch: 32 B in FP32, 64 B in
    # FP64.  The kernel itself moves 18 (the rounding residual that keeps the FP32 state update
    # exact is read and written once per step, and stage 4 reads the state once more to add the
    # step's increment to it): reported beside it.
    csz = 8 if args.dtype == "f32" else 16
    # the pipelined path runs the four stages of a step in one launch (k_steps_pipe); the other
    # paths launch once per stage
    variant = state.stage_variant()
    fused = variant == "pipelined" and state.get_tune()["pipe_fused"] == 1
    stages_per_launch = 4 if fused else 1
    bytes_per_launch = stages_per_launch * 4 * csz * pts
    kernel_bytes_per_launch = stages_per_launch * 18 * csz * pts / 4
    launch_s = stage_ms / 1e3 / (4 * args.steps / stages_per_launch)
    achieved = bytes_per_launch / launch_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:  # noqa: BLE001
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(args.instances, args.dtype, schedule) if fused else None,
            "kernel": "bq::k_steps_pipe" if fused else {"pipelined": "bq::k_stage_pipe", "single_mode": "bq::k_stage_m1",
                                                          "generic": "bq::k_stage"}[variant],
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "stages_per_launch": stages_per_launch, "bytes_per_launch": bytes_per_launch, "bytes_per_point_stage": 4 * csz,
            "kernel_bytes_per_launch": kernel_bytes_per_launch, "kernel_transfers_per_step": 18,
            "avg_launch_us": launch_s * 1e6}

    # ---- end to end through the C ABI: state from pinned host memory, observables back ---
    # The batch is split into E2E_PARTS states on as many streams: while one part is stepped,
    # the next part's input is uploaded (and the previous part's observables are read back), so
    # the host-to-device copies hide behind the stage kernels.
    nbytes = state.state_bytes()
    e2e = e2e_leg(specs, opts, schedule, args.steps, world, barrier)
    del state

    # the 4096-instance full solves and the gradient are single-GPU legs (rank 0 of a 1-GPU run)
    peaks_alu = alu_peaks() if world == 1 else None
    fp64 = None
    if not args.no_batched and world == 1 and args.dtype == "f32":
        fp64 = fp64_leg(args.instances, peaks_alu)
    batched = None
    if not args.no_batched and world == 1:
        batched = batched_leg(world)
        f32_peak = 2 * peaks_alu["fp32_fma_per_s"]
        p = batched["persistent"]
        p["alu_roofline"] = {"bound": "alu", "achieved": FLOP_PER_POINT_STAGE * p["updates_per_s"] / 1e12,
                             "peak": f32_peak / 1e12, "unit": "TFLOP/s",
                             "frac": FLOP_PER_POINT_STAGE * p["updates_per_s"] / f32_peak,
                             "peak_source": "measured (bq_fma_peak, FP32)"}
    grads = None
    if not args.no_grads and world == 1:
        grads = grads_leg()
    methods = None
    secular = None
    fig2 = None
    if not args.no_batched and world == 1:
        methods = methods_leg()
        secular = secular_leg()
        fig2 = fig2_leg()  # the left panels (time dependence): --only-fig2

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.instances)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c" + args.dtype,
                "data": "synthetic (seeded kerr_batch distribution)",
                "config": {"workload": f"kerr_batch x{args.instances}: driven damped Kerr oscillators, "
                                       f"mapped method (G_x, G_y, full R), one RK4 step of dt={DT} ns + "
                                       "Tr(rho0 A) per instance per step",
                           "instances_per_gpu": args.instances, "n_range": list(N_RANGE), "grid_points_per_gpu": pts,
                           "schedule": {k: schedule[k] for k in ("stage_path", "pipe_slots", "pipe_ctas_per_sm",
                                                                 "n_candidates", "step_us")},
                           "state_bytes_per_array": nbytes, "l2": "inputs larger than L2 (5 arrays x "
                           f"{nbytes / 1e6:.0f} MB vs 129 MB)", "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "alu_peaks": peaks_alu, "fp64": fp64, "batched": batched, "grads": grads, "methods": methods, "secular": secular, "fig2": fig2, "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
