"""Throughput of the pseudo-spectral Navier-Stokes step on GB300.

Workload (one "step" = one Lawson IF-RK4 step of the whole hot path):
  3D incompressible NS, 512^3, FP32 state and FFTs, random-phase solenoidal
  initial velocity with E(k) ~ k^4 exp(-2 (k/4)^2) (mean energy 0.5, seed 0),
  nu = 2e-3, dt = 1e-3 (the 512^3 configuration; 20 steps per job).
Metric: Mpoint * RK4-steps / s = N^3 * steps / seconds / 1e6 (whole job over
all ranks).  Under torchrun every rank advances its own independent replica
(the single-box problem does not shard without an all-to-all), so per-rank
work is fixed and scaling is weak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the baseline this project is
measured against) on the host cores, rank 0 only, on the same 512^3 workload
(time-bounded: the line states how many steps ran).  The GPU line carries
err_vs_fp64: the relative L2 error after 10 steps against the oracle of the
FP32, tensor-core and FP64 forms (64^3 instance of the recipe) and of the
ensemble (one member per grid size), each beside its stated bound.
The line also carries `tensor_core`: the same workload with the x-line
transforms on the tensor cores (precision NS_FP32_TC, split-BF16 GEMMs),
beside the FP32 headline; `--precision tc` times that mode alone (profiling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 512
NU, DT = 2e-3, 1e-3
JOB_STEPS = 20
UNIT = "Mpoint*steps/s"


def metric_name(n=None, tc=False):
    n = N_GRID if n is None else n
    return f"Mpoint*RK4-steps/s at 3D {n}^3 " + ("FP32 (tensor-core x pass)" if tc else "FP32")


def workload(n=None, tc=False):
    n = N_GRID if n is None else n
    return (f"3D incompressible NS {n}^3 " + ("FP32 with the x-line transforms on the tensor cores" if tc else "FP32")
            + ", random-phase solenoidal IC E(k)~k^4 exp(-2(k/4)^2), E=0.5, seed 0, "
            "nu=2e-3, dt=1e-3, Lawson IF-RK4, 2/3 dealiasing")


def l2_note(n=None, elem=8):
    """State and pass-buffer sizes of the n^3 run against the 129 MB L2."""
    n = N_GRID if n is None else n
    kc = (n - 1) // 3
    c, h = 2 * kc + 1, kc + 1
    hs = -(-h * elem // 128) * 128 // elem
    state = 3 * c * c * hs * elem / 1e9
    bufs = (6 * n * c * hs + 6 * n * n * hs) * elem / 1e9
    return (f"inputs larger than L2: state {state:.2f} GB, pass buffers {bufs:.1f} GB vs 129 MB L2 "
            "(no flush needed)")
# Algorithmic bytes of one 512^3 FP32 step for the fused three-phase model
# (truncated spectrum, middle-axis passes counted once): 252.8 B/point.
MODEL_BYTES_PER_POINT = 252.8


def flop_model(n):
    """Dense-FFT flop counts (2.5 n log2 n per real transform of length n):
    per point of a step, nine real 3D transforms per RK stage, four stages;
    per x-pass launch, nine real x-line transforms per (z, y) line plus the
    cross product (9 flops per point)."""
    import math

    lg = math.log2(n)
    return 4 * 9 * 2.5 * 3 * lg, n * n * (9 * 2.5 * n * lg + 9 * n)


# wall-clock bound of the reference arm's timed oracle steps (seconds)
REF_BUDGET_S = 90.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int, device) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, points: int, steps: int, ms: float) -> float:
    """Whole-job Mpoint*steps/s: every rank advances its own replica of `points`
    grid points by `steps` steps in `ms` milliseconds (weak scaling)."""
    return ws * points * steps / (ms / 1e3) / 1e6


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        self.index = ids[local_rank] if local_rank < len(ids) and ids[local_rank].isdigit() else str(local_rank)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", self.index], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# the sources that define the 3D FP32 pass kernels (their launch shapes included)
PASS_KERNEL_SOURCES = ("ns_fft.cuh", "ns_internal.h", "ns_k3_f32.cu", "ns_kernels.cuh")


def pass_kernel_digest() -> str:
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1807_01769_gb300", "csrc")
    for f in PASS_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def traffic_from_profiles(kernel: str):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if the
    pass-kernel sources are unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = pass_kernel_digest()
    for line in open(path):
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("n") == str(N_GRID) and kv.get("source_sha") == digest:
            return int(kv["dram_bytes_per_launch"])
    return None


def flops_entry(ms_step, prof, fma_peak):
    """Flop efficiency beside the HBM roofline: the dense-FFT model against the
    measured FP32 FMA rate of the GPU."""
    per_pt, xpass_flops = flop_model(N_GRID)
    step_tf = per_pt * N_GRID ** 3 / (ms_step / 1e3) / 1e12
    out = {"model_flop_per_point": per_pt, "achieved_tflops": step_tf, "peak_tflops": fma_peak,
           "peak_kind": "measured FP32 FMA rate (ns_fp32_fma_peak)", "frac": step_tf / fma_peak,
           "note": "dense-FFT count, 2.5 n log2 n per real transform; the pruned transforms do fewer"}
    if "xpass" in prof and prof["xpass"][1] > 0:
        xs = prof["xpass"][0] / prof["xpass"][1] / 1e3
        out["xpass_tflops"] = xpass_flops / xs / 1e12
        out["xpass_frac"] = out["xpass_tflops"] / fma_peak
    return out


def cpu_baseline(n=None, steps=1):
    """The FP64 oracle as it stands, on this host's cores: a bounded sample,
    `steps` RK4 steps of the bench recipe on the bench grid itself (one 512^3
    step holds about 25 GB of host memory and takes ~40 s on 16 Grace cores)."""
    import oracle
    from paper_1807_01769_gb300 import inputs

    n = N_GRID if n is None else n
    u0 = inputs.random_velocity_3d(n, seed=0, k0=4.0, a=2.0, energy=0.5)
    t0 = time.perf_counter()
    oracle.step(3, n, NU, DT, steps, u0)
    t = time.perf_counter() - t0
    return {"value": n ** 3 * steps / t / 1e6, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{steps} Lawson IF-RK4 step(s) of the bench recipe at {n}^3 in FP64 ({t:.1f} s), "
                      f"the same grid as the GPU line"}


def _rel_l2(a, b):
    import numpy as np

    w = np.full(b.shape[-1], 2.0)
    w[0] = 1.0
    return float(np.sqrt(np.sum(w * np.abs(a - b) ** 2) / np.sum(w * np.abs(b) ** 2)))


# error bounds each precision states after 10 steps against the FP64 oracle
ERR_TOL = {"fp32": 1e-5, "fp32_tc": 1e-3, "fp64": 1e-11, "ensemble_fp32": 1e-5}


def err_vs_fp64(steps=10, n=64):
    """Relative L2 error (half-spectrum weights, i.e. the physical L2 error by
    Parseval) after `steps` steps against the FP64 oracle, outside the timed
    region: the 3D forms on the n^3 instance of the bench recipe (same seed,
    nu, dt), the ensemble on one member of each of its grid sizes (2D recipe of
    the ensemble line, seeds = member indices)."""
    import oracle
    from paper_1807_01769_gb300 import inputs, ns

    out = {}
    u0 = inputs.random_velocity_3d(n, seed=0, k0=4.0, a=2.0, energy=0.5)
    ref = oracle.step(3, n, NU, DT, steps, u0)
    for name, prec in (("fp32", ns.NS_FP32), ("fp32_tc", ns.NS_FP32_TC), ("fp64", ns.NS_FP64)):
        with ns.Solver(3, n, prec, nu=NU, dt=DT) as s:
            s.set_state_spectral(u0)
            s.step(steps)
            err = _rel_l2(s.get_state_spectral(), ref)
        out[name] = {"rel_l2": err, "tol": ERR_TOL[name], "ok": err <= ERR_TOL[name], "grid": f"{n}^3",
                     "steps": steps}
    sizes = inputs.ensemble_sizes(64)
    members = [sizes.index(m) for m in (128, 256, 512) if m in sizes]
    ens = []
    with ns.Ensemble([sizes[m] for m in members], ns.NS_FP32, nu=5e-4, dt=5e-4, autotune=False) as e:
        w0 = [inputs.random_vorticity_2d(sizes[m], seed=m, k0=8.0, a=2.0, energy=0.5) for m in members]
        for j, w in enumerate(w0):
            e.set_state_spectral(j, w)
        e.step(steps)
        for j, m in enumerate(members):
            nm = sizes[m]
            err = _rel_l2(e.get_state_spectral(j), oracle.step(2, nm, 5e-4, 5e-4, steps, w0[j]))
            ens.append({"member": m, "grid": f"{nm}^2", "rel_l2": err})
    worst = max(x["rel_l2"] for x in ens)
    out["ensemble_fp32"] = {"rel_l2": worst, "tol": ERR_TOL["ensemble_fp32"], "ok": worst <= ERR_TOL["ensemble_fp32"],
                            "steps": steps, "members": ens}
    out["note"] = (f"{steps} steps vs the FP64 oracle; 3D forms on the {n}^3 instance of the bench recipe, the "
                   "ensemble on one member of each size")
    return out


ENSEMBLE_WORKLOAD = ("64 independent 2D NS runs (vorticity form), sizes drawn uniformly from {128^2, 256^2, 512^2} "
                     "(splitmix64(1000+i)), FP32, random-phase spectrum peaked at k=8 (E~k^4 exp(-2(k/8)^2)), "
                     "seeds 0..63, nu=dt=5e-4")


def ensemble_bench(steps=50):
    """Batched 2D ensemble (one persistent launch per pass over all members,
    autotuned schedule, one CUDA graph per step) against the plain form: the
    same 64 runs each advanced by its own ns_step graph on the same stream."""
    import torch

    from paper_1807_01769_gb300 import inputs, ns

    sizes = inputs.ensemble_sizes(64)
    u0 = [inputs.random_vorticity_2d(n, seed=m, k0=8.0, a=2.0, energy=0.5) for m, n in enumerate(sizes)]
    pts = sum(n * n for n in sizes)
    stream = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ns.Ensemble(sizes, ns.NS_FP32, nu=5e-4, dt=5e-4, autotune=True) as e:
        e.set_stream(stream.cuda_stream)
        for m, u in enumerate(u0):
            e.set_state_spectral(m, u)
        e.step(3)
        e.sync()
        ev0.record(stream)
        e.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        e.sync()
        ms = ev0.elapsed_time(ev1) / steps
        sched = e.schedule()
        tiles = e.tiles()
        fused, fused_max = e.fused()
        # the other form for the record: one cooperative launch per stage at the
        # most resident blocks, or (if that was chosen) the two-launch form
        if fused:
            e.set_tiles(256, 8)
        else:
            e.set_fused(fused_max)
        e.step(3)
        ev0.record(stream)
        e.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        e.sync()
        ms_other = ev0.elapsed_time(ev1) / steps
    solvers = [ns.Solver(2, n, ns.NS_FP32, nu=5e-4, dt=5e-4) for n in sizes]
    for s, u in zip(solvers, u0):
        s.set_stream(stream.cuda_stream)
        s.set_state_spectral(u)
        s.step(3)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        for s in solvers:
            s.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_plain = ev0.elapsed_time(ev1) / steps
    for s in solvers:
        s.close()
    return {"workload": ENSEMBLE_WORKLOAD, "metric": "Mpoint*RK4-steps/s", "steps": steps,
            "value": pts / (ms / 1e3) / 1e6, "ms_per_step": ms, "plain_value": pts / (ms_plain / 1e3) / 1e6,
            "plain_ms_per_step": ms_plain, "speedup_vs_plain": ms_plain / ms,
            "one_launch_per_stage_ms_per_step" if not fused else "two_launches_per_stage_ms_per_step": ms_other,
            "schedule": {"y_block_threads": tiles[0], "x_block_warps": tiles[1],
                         "one_launch_per_stage_blocks_per_sm": fused,
                         "x_blocks_per_sm": sched[0], "y_blocks_per_sm": sched[1],
                         "task_order": ["member-major", "round-robin"][sched[2]]}}


# The grids the paper times (Performance section: sequential and Beskow runs),
# with its best published rate for each in Mpoint*steps/s (CPU; context only).
PAPER_SHAPES = [
    (2, 512, "fp64", 4.85), (2, 512, "fp32", 4.85),
    (2, 1024, "fp64", 45.6), (2, 1024, "fp32", 45.6),
    (2, 2048, "fp64", 82.2), (2, 2048, "fp32", 82.2),
    (3, 128, "fp64", 77.7), (3, 128, "fp32", 77.7),
    (3, 1024, "fp32", 493.7),
]


def paper_shapes(target_s=0.25):
    """Mpoint*RK4-steps/s of the GPU path on the paper's grid sizes (random
    initial fields of the 2D and 3D recipes, nu = 1e-3, dt = 1e-3), CUDA events
    on a dedicated stream after two warm-up steps."""
    import torch
    from paper_1807_01769_gb300 import inputs, ns

    out = []
    stream = torch.cuda.Stream()
    for dim, n, prec, paper in PAPER_SHAPES:
        p = ns.NS_FP64 if prec == "fp64" else ns.NS_FP32
        u0 = (inputs.random_vorticity_2d(n, seed=0, k0=8.0, a=1.0, energy=0.5) if dim == 2
              else inputs.random_velocity_3d(n, seed=0, k0=4.0, a=2.0, energy=0.5))
        with ns.Solver(dim, n, p, nu=1e-3, dt=1e-3) as s:
            s.set_stream(stream.cuda_stream)
            s.set_state_spectral(u0)
            s.step(2)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            s.step(1)
            ev1.record(stream)
            torch.cuda.synchronize()
            k = max(3, min(500, int(target_s * 1e3 / max(ev0.elapsed_time(ev1), 1e-3))))
            ev0.record(stream)
            s.step(k)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / k
            e, _ = s.diagnostics()
        out.append({"grid": f"{n}^{dim}", "dtype": prec, "steps": k, "ms_per_step": ms,
                    "value": n ** dim / (ms / 1e3) / 1e6, "paper_best_cpu": paper, "energy_after": e})
    return {"metric": "Mpoint*RK4-steps/s", "note": "paper_best_cpu: the paper's best CPU rate for the grid "
            "(sequential for 2D 512^2, Beskow MPI runs otherwise), for context", "runs": out}


def tensor_core_bench(u0, steps=20, warm=3):
    """The same workload with the x-line transforms on the tensor cores
    (NS_FP32_TC: split-BF16 GEMMs, FP32 accumulation), beside the FP32 path:
    step time, x pass per launch (CUDA events), and the energy and enstrophy
    after warm + steps steps relative to an FP32 run of the same steps."""
    import torch
    from paper_1807_01769_gb300 import ns

    stream = torch.cuda.Stream()
    with ns.Solver(3, N_GRID, ns.NS_FP32, nu=NU, dt=DT) as s:
        s.set_stream(stream.cuda_stream)
        s.set_state_spectral(u0)
        s.step(warm + steps)
        e32, om32 = s.diagnostics()
    with ns.Solver(3, N_GRID, ns.NS_FP32_TC, nu=NU, dt=DT) as s:
        s.set_stream(stream.cuda_stream)
        s.set_state_spectral(u0)
        s.step(warm)
        s.sync()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        e, om = s.diagnostics()
        prof = s.profile_step(3)
    x = prof.get("xpass", (0.0, 0, 0))
    return {"precision": "NS_FP32_TC", "steps": steps, "ms_per_step": ms, "value": N_GRID ** 3 / (ms / 1e3) / 1e6,
            "xpass_ms_per_launch": x[0] / x[1] if x[1] else None,
            "energy_rel_diff_vs_fp32": abs(e - e32) / e32,
            "enstrophy_rel_diff_vs_fp32": abs(om - om32) / om32,
            "note": "not the headline: products carry ~1e-5 relative error (BF16 hi+lo operands)"}


def run_reference(args):
    """The oracle on the bench workload itself (512^3, FP64, host cores): one
    512^3 RK4 step takes ~40 s on 16 Grace cores, so the run is bounded by
    time: warm-up steps and timed steps stop once REF_BUDGET_S seconds have
    gone into each (at least one timed step); the line states how many ran."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1807_01769_gb300 import inputs

    n = N_GRID
    u = inputs.random_velocity_3d(n, seed=0, k0=4.0, a=2.0, energy=0.5)
    t0 = time.perf_counter()
    warm = 0
    while warm < args.warmup and time.perf_counter() - t0 < REF_BUDGET_S / 4:
        u = oracle.step(3, n, NU, DT, 1, u)
        warm += 1
    timed = 0
    t0 = time.perf_counter()
    while timed < max(args.steps, 1) and (timed == 0 or time.perf_counter() - t0 < REF_BUDGET_S):
        u = oracle.step(3, n, NU, DT, 1, u)
        timed += 1
    t = time.perf_counter() - t0
    v = n ** 3 * timed / t / 1e6
    sample = (f"{timed} of the {args.steps} requested Lawson IF-RK4 steps of the bench workload at {n}^3 in FP64 "
              f"timed after {warm} warm-up step(s) (time-bounded at {REF_BUDGET_S:.0f} s)")
    line = {"impl": "reference", "metric": metric_name(n), "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": timed, "warmup": warm, "requested_steps": args.steps, "requested_warmup": args.warmup,
            "ms_per_step": t / timed * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(n), "n": n, "l2": l2_note(n)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if args.gpus != ws and ws > 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE={ws}", file=sys.stderr)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    from paper_1807_01769_gb300 import inputs, ns

    u0 = inputs.random_velocity_3d(N_GRID, seed=0, k0=4.0, a=2.0, energy=0.5)
    prec = ns.NS_FP32_TC if args.precision == "tc" else ns.NS_FP32
    s = ns.Solver(3, N_GRID, prec, nu=NU, dt=DT)
    # a dedicated (non-default) torch stream: the library launches on it and
    # the CUDA events below are recorded on it
    stream = torch.cuda.Stream()
    s.set_stream(stream.cuda_stream)
    s.set_state_spectral(u0)

    # warm-up (builds the step graph)
    s.step(max(args.warmup, 3))
    s.sync()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, ws, "cuda")
    e, om = s.diagnostics()
    if not (np.isfinite(e) and np.isfinite(om)):
        raise RuntimeError("non-finite state after the timed steps")

    # per-kernel CUDA-event timing (instrumented launches, same stream)
    prof = s.profile_step(3)
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    dom_ms, dom_n, dom_bytes = prof[dom]
    dom_avg_s = dom_ms / dom_n / 1e3
    hbm, peak_kind = peaks()
    achieved = dom_bytes / dom_avg_s / 1e9
    traffic = traffic_from_profiles(dom) if prec == ns.NS_FP32 else None
    fma_peak = ns.fp32_fma_peak(local)  # TFLOP/s, measured on this GPU

    # end to end through the C ABI with pinned host buffers: upload the initial
    # state, advance one job (JOB_STEPS steps), read back state and spectrum
    spec_bytes = s.sizes["state_doubles"] * 8
    h_in = torch.from_numpy(u0.view(np.float64).reshape(-1)).pin_memory()
    h_out = torch.empty(s.sizes["state_doubles"], dtype=torch.float64).pin_memory()
    e2e_reps = max(1, args.e2e_reps)
    # one untimed job first: the first copies from freshly pinned buffers pay
    # a one-time mapping cost (about 16 ms each way at 512^3)
    s.set_state_spectral_ptr(h_in.data_ptr())
    s.step(JOB_STEPS)
    s.get_state_spectral_ptr(h_out.data_ptr())
    s.energy_spectrum()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        s.set_state_spectral_ptr(h_in.data_ptr())
        s.step(JOB_STEPS)
        s.get_state_spectral_ptr(h_out.data_ptr())
        spec = s.energy_spectrum()
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, ws, "cuda")
    launches_per_step = sum(v[1] for k, v in prof.items()) // 3

    if rank == 0:
        pts = N_GRID ** 3
        value = job_value(ws, pts, args.steps, ms_max)
        step_bytes = MODEL_BYTES_PER_POINT * pts
        line = {
            "metric": metric_name(tc=args.precision == "tc"), "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == ns.NS_FP32 else "f32+bf16x3",
            "data": "synthetic",
            "config": {"workload": workload(tc=args.precision == "tc"), "n": N_GRID, "precision": args.precision,
                       "parallelism": f"replicas x{ws}",
                       "l2": l2_note(), "job_steps": JOB_STEPS},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                         "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_avg_s * 1e3},
            "step_roofline": {"model_bytes_per_point": MODEL_BYTES_PER_POINT,
                              "achieved_gbs": step_bytes / (ms_max / args.steps / 1e3) / 1e9,
                              "frac": step_bytes / (ms_max / args.steps / 1e3) / 1e9 / hbm},
            "flops": flops_entry(ms_max / args.steps, prof, fma_peak),
            "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches_per_step": v[1] / 3,
                            "algorithmic_gbs": v[2] / (v[0] / v[1] / 1e3) / 1e9}
                        for k, v in prof.items() if v[1] > 0},
            "clocks": clk,
            "e2e": {"value": job_value(ws, pts, JOB_STEPS * e2e_reps, e2e_s * 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": spec_bytes / JOB_STEPS,
                    "d2h_bytes_per_step": (spec_bytes + spec.nbytes) / JOB_STEPS,
                    "job": f"H2D of the FP64 initial spectrum (pinned), {JOB_STEPS} steps, D2H of the state and "
                           f"spectrum; {e2e_reps} jobs after one untimed job"},
            "gpu_launches": launches_per_step * args.steps,
            "energy_after": e, "enstrophy_after": om,
        }
        if ws == 1 and not args.no_err:
            line["err_vs_fp64"] = err_vs_fp64()
        if ws == 1 and not args.no_ensemble:
            line["ensemble"] = ensemble_bench()
        if ws == 1 and not args.no_paper_shapes:
            line["paper_shapes"] = paper_shapes()
        if ws == 1 and prec == ns.NS_FP32 and not args.no_tc:
            try:  # a side measurement: it must never cost the headline line
                line["tensor_core"] = tensor_core_bench(u0)
            except Exception as exc:  # noqa: BLE001
                line["tensor_core"] = {"precision": "NS_FP32_TC", "error": f"{type(exc).__name__}: {exc}"}
        # the oracle last, after every GPU measurement: its 25 GB of host
        # memory, freed just before, slowed the pinned copies of the
        # end-to-end jobs that followed it (uploads 4.8 -> ~40 ms)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-reps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched 2D ensemble measurement")
    ap.add_argument("--no-paper-shapes", action="store_true", help="skip the paper-grid measurements")
    ap.add_argument("--n", type=int, default=512, help="grid size override (profiling of smaller cases only)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc"],
                    help="tc: the x-line transforms on the tensor cores (profiling; the headline is fp32)")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core comparison")
    ap.add_argument("--no-err", action="store_true", help="skip the 10-step error against the FP64 oracle")
    args = ap.parse_args()
    global N_GRID
    N_GRID = args.n
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
