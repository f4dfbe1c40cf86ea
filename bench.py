#!/usr/bin/env python
"""Throughput of the 3D elastic staggered-grid forward loop on one GB300.

One bench *step* is one full forward simulation of the 256^3 workload: 2000
time steps of the velocity pass, source injection, receiver sampling and
stress pass with a 20-cell C-PML, on a 5-layer + Gaussian-correlated +-5 %
synthetic model with a double-couple source (5 Hz Ricker at 2 km depth) and
16 x 16 receivers.  Metric: Gcell-updates/s (one cell-update = all 9 fields
of one cell advanced one time step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  Under torchrun (N > 1) every rank runs an
independent replica of the workload (the path has no exchange step), the
timing is the max over ranks and `value` counts the cells of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s per FP32 elastic step, % of HBM roofline; adjoint grad time / fwd"
UNIT = "Gcell-updates/s"
WORKLOAD = ("256^3 grid, dx=20 m, 2000 steps, 20-cell C-PML, 5 layers vp 2000-6000 m/s "
            "+ Gaussian-correlated +-5% (200 m), Gardner rho, double couple (30,60,90) "
            "5 Hz Ricker at 2 km, 16x16 receivers")
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=256, help="cube side (default 256)")
    ap.add_argument("--nt", type=int, default=2000, help="time steps per bench step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint-gradient / forward time ratio")
    ap.add_argument("--adj-n", type=int, default=192)
    ap.add_argument("--adj-nt", type=int, default=1500)
    ap.add_argument("--boundary", choices=("cpml", "sponge", "none"), default="cpml",
                    help="absorbing edge of the main loop (the benchmark workload: cpml; "
                         "the others serve profiling captures)")
    ap.add_argument("--tile", choices=("auto", "32x8", "32x4", "32x16", "fused"), default="auto",
                    help="tile shape of the main loop (auto: the tuner's choice)")
    ap.add_argument("--storage", choices=("f32", "bf16", "f16"), default="f32",
                    help="wavefield storage of the main workload (FP32 arithmetic)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the timing sweep over the paper's 11 grid levels")
    ap.add_argument("--sweep-nt", type=int, default=100,
                    help="time steps timed per level of the sweep")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-shot comparison")
    ap.add_argument("--batch-shots", type=int, default=48,
                    help="shots of the 48-shot batched workload run forward (first k)")
    ap.add_argument("--batch-grad-shots", type=int, default=48,
                    help="shots of it run forward + gradient (first k; one call runs "
                         "them in waves whose gradient state fits the GPU)")
    ap.add_argument("--no-free-surface", action="store_true",
                    help="skip the free-surface (vacuum formulation) timing")
    ap.add_argument("--fs-nt", type=int, default=200,
                    help="time steps timed with and without the free surface")
    ap.add_argument("--no-coarse", action="store_true",
                    help="skip the coarse-medium-grid timing")
    ap.add_argument("--no-fwi", action="store_true",
                    help="skip the multi-shot inversion-iteration timing")
    ap.add_argument("--fwi-shots", type=int, default=8)
    ap.add_argument("--no-storage", action="store_true",
                    help="skip the FP32 / BF16 / FP16 storage comparison")
    ap.add_argument("--storage-nt", type=int, default=40,
                    help="time steps timed per storage type on the large grid")
    ap.add_argument("--crop-nt", type=int, default=1000,
                    help="time steps of the 128^3 crop run against the oracle")
    return ap.parse_args()


# --- distributed plumbing ----------------------------------------------------

def dist_setup(want: int):
    """Rank, world and local device from the torchrun environment; NCCL
    process group on GPUs (gloo when no GPU is present, e.g. CPU tests)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values (each rank's timed region)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, steps: int, ms: float, world: int) -> float:
    """Whole-job throughput: the units all ranks processed (replicas, the
    same work on every rank) over the slowest rank's time."""
    return world * units_per_rank * steps / (ms / 1e3)


# --- clocks ------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={CLOCK_QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r[2] > 150.0] or rows
        reasons = sorted({REASONS[i] for r in load for i, v in enumerate(r[3])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load),
                "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(load), "power_w_max": max(r[2] for r in rows),
                "reasons": reasons}


def section(fn, *a):
    """Run one of the secondary sections after the headline measurement; if
    it raises, record the error in its place (and on stderr) so that the
    JSON line with the headline number is still printed."""
    try:
        return fn(*a)
    except Exception as e:                       # noqa: BLE001 -- reported, not hidden
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"[:400]}


# --- roofline bookkeeping ----------------------------------------------------

def algorithmic_bytes(prob, es: int = 4):
    """Minimal DRAM bytes per launch of each pass, for wavefields stored in
    `es` bytes (the medium is FP32):
    velocity: read 6 sigma + rho, read+write 3 v           = 12 es + 4 B / cell
    stress:   read 3 v + lambda + mu, read+write 6 sigma   = 15 es + 8 B / cell
    (FP32: 52 and 68 B).  C-PML: each pass reads and writes 3 FP32 memory
    variables per damped direction of every slab cell (24 B per
    cell-direction and pass).  The whole-step minimum reads and writes the 9
    fields once and reads the medium once: 18 es + 12 B (84 B in FP32)."""
    n = prob.nx * prob.ny * prob.nz
    W = prob.width if prob.boundary == "cpml" else 0
    slab = 2 * W * (prob.ny * prob.nz + prob.nx * prob.nz + prob.nx * prob.ny)
    return {"velocity": (12 * es + 4) * n + 24 * slab, "stress": (15 * es + 8) * n + 24 * slab,
            "step_min": (18 * es + 12) * n + 48 * slab, "step": (18 * es + 12) * n + 48 * slab,
            "slab_cell_dirs": slab}


def kernel_source_sha() -> str:
    """Hash of the stencil kernels' source, the headers it includes and the
    build flags (everything the traffic figure's kernels are compiled from);
    any edit there voids the committed figure."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_2112_15071_gb300")
    for f in (os.path.join(pkg, "csrc", "ews_stencil.cu"), os.path.join(pkg, "csrc", "ews_fused.cu"),
              os.path.join(pkg, "csrc", "ews_internal.cuh"),
              os.path.join(pkg, "csrc", "ews_ops.cuh"), os.path.join(ROOT, "include", "ews.h"),
              os.path.join(pkg, "_build.py")):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload_tag: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    prof = os.path.join(ROOT, "profiles")
    if not os.path.isdir(prof):
        return None
    sha = kernel_source_sha()
    pat = re.compile(r"bench-traffic:\s*kernel=(\S+)\s+workload=(\S+)\s+sha=(\S+)\s+"
                     r"bytes_per_launch=([0-9.eE+]+)")
    for f in sorted(os.listdir(prof)):
        if not f.endswith((".md", ".txt")):
            continue
        for m in pat.finditer(open(os.path.join(prof, f)).read()):
            if m.group(1) == kernel and m.group(2) == workload_tag and m.group(3) == sha:
                return float(m.group(4))
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --- CPU baseline: the FP64 oracle as it stands ------------------------------

def cpu_oracle_rate(prob, seconds: float):
    """Time the oracle on the host cores on a bounded sample of the workload
    (the full grid, a number of time steps sized to ~`seconds`)."""
    from oracle import oracle
    oracle.build()
    s = oracle.OracleSim(prob.nx, prob.ny, prob.nz, prob.spacing)
    s.set_medium_vel(prob.vp, prob.vs, prob.rho)
    s.set_boundary(prob.boundary, prob.width, prob.dt, prob.f0)
    s.forward(2, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp, prob.wavelet,
              prob.rec_pos)                      # first touch of the oracle's arrays
    t0 = time.perf_counter()
    s.forward(2, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp, prob.wavelet,
              prob.rec_pos)
    per = (time.perf_counter() - t0) / 2
    nsteps = max(2, min(prob.nt - 2, int(seconds / max(per, 1e-6))))
    t0 = time.perf_counter()
    s.forward(nsteps, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp, prob.wavelet,
              prob.rec_pos)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": prob.ncell * nsteps / el / 1e9, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"FP64 oracle, full {prob.nx}^3 grid with C-PML, first {nsteps} of "
                      f"{prob.nt} time steps ({el:.1f} s)"}


# --- our arm ------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_2112_15071_gb300 import ews, synth

    prob = synth.config2(n=args.n, nt=args.nt)
    prob.boundary = args.boundary
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sim = ews.simulation_for(prob, storage=args.storage)
    if args.tile != "auto":
        sim.set_tile_shape(args.tile)
    sim.set_stream(stream.cuda_stream)
    seis = torch.zeros((3, sim.nrec, prob.nt), device=dev)
    for _ in range(args.warmup):
        sim.run(prob.nt, prob.dt, seis)
    torch.cuda.synchronize()
    sim.profile(reset=True)

    # timed region: the time loop as one captured CUDA graph per run
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        sim.run(prob.nt, prob.dt, seis)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(t_start.elapsed_time(t_end), world)
    _, klaunch = sim.profile(reset=True)
    cells = prob.ncell * prob.nt
    value = aggregate_rate(cells, args.steps, ms, world) / 1e9

    # per-kernel durations: the same runs with CUDA events between launches
    # (direct launches instead of the graph), on the launching stream
    sim.set_profiling(True)
    for _ in range(max(1, min(args.steps, 2))):
        sim.run(prob.nt, prob.dt, seis)
    torch.cuda.synchronize()
    kms, kl_prof = sim.profile(reset=True)
    sim.set_profiling(False)

    # dominant kernel and its roofline
    names = ews.KERNEL_NAMES
    dom = int(np.argmax(kms[:len(names)]))
    alg = algorithmic_bytes(prob, 4 if args.storage == "f32" else 2)
    avg_ms = kms[dom] / max(kl_prof[dom], 1)
    dom_bytes = alg.get(names[dom], 0)
    peak, peak_kind = peaks()
    achieved = dom_bytes / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    tag = f"{prob.nx}cube_{args.boundary}" + ("" if args.storage == "f32" else "_" + args.storage)
    kfunc = {"points": "k_post_stress", "step": "k_fused"}.get(names[dom], f"k_{names[dom]}")
    traffic = committed_traffic(kfunc, tag)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "kernel": kfunc, "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": dom_bytes,
            "avg_launch_ms": round(avg_ms, 5)}
    step_ms = ms / args.steps
    # whole time step against the fused minimum (84 B per cell-update plus
    # the C-PML memory variables), per GPU
    whole_gbs = alg["step_min"] * prob.nt / (step_ms / 1e3) / 1e9
    whole = {"algorithmic_bytes_per_time_step": alg["step_min"],
             "achieved_gbs": round(whole_gbs, 1), "frac": round(whole_gbs / peak, 4)}
    # the same without the C-PML terms: Gcell/s x (9 fields read + written
    # + 3 medium arrays read) / peak
    es = 4 if args.storage == "f32" else 2
    min_cell = 18 * es + 12
    gcells_dev = prob.nx * prob.ny * prob.nz * prob.nt / (step_ms / 1e3) / 1e9
    whole["bytes_per_cell_fields_medium"] = min_cell
    whole["frac_fields_medium"] = round(gcells_dev * min_cell / peak, 4)
    kernel_share = {names[k]: round(kms[k] / max(kms.sum(), 1e-12), 4)
                    for k in range(len(names)) if kl_prof[k]}

    # end to end through the public API with host buffers (pinned)
    vp = torch.from_numpy(prob.vp).pin_memory().numpy()
    vs = torch.from_numpy(prob.vs).pin_memory().numpy()
    rho = torch.from_numpy(prob.rho).pin_memory().numpy()
    seis_host = torch.zeros((3, sim.nrec, prob.nt), dtype=torch.float32).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 3))
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_model_vel(vp, vs, rho)
        sim.run(prob.nt, prob.dt, seis_host)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * cells * e2e_steps / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": int(3 * prob.vp.nbytes),
           "d2h_bytes_per_step": int(seis_host.nbytes),
           "steps": e2e_steps, "api": "ews_set_model_vel + ews_run (host buffers)"}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded layered + random model)",
        "config": {"workload": WORKLOAD if args.boundary == "cpml" else
                   WORKLOAD.replace("20-cell C-PML", "20-cell sponge" if args.boundary == "sponge"
                                    else "no absorbing edge"),
                   "grid": [prob.nx, prob.ny, prob.nz], "nt": prob.nt,
                   "dx_m": prob.spacing[0], "boundary": args.boundary, "width": prob.width,
                   "storage": args.storage, "tile_shape": sim.tile_shape,
                   "receivers": int(sim.nrec), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (9 fields + 3 medium arrays = 768 MiB "
                         "resident, 129 MB L2)",
                   "launch": "time loop captured as one CUDA graph per run; kernel times from "
                             "event-bracketed direct launches of the same runs"},
        "roofline": roof, "whole_step": whole, "kernel_share": kernel_share,
        "gpu_launches": int(klaunch.sum()) * world,
        "e2e": e2e, "clocks": clk,
    }
    if not args.no_adjoint:
        out["adjoint"] = section(adjoint_ratio, args, local)
    if not args.no_storage:
        out["storage"] = section(storage_report, args, local, rank == 0 and world == 1)
    if not args.no_batch:
        out["batch"] = section(batch_report, args, local)
    if not args.no_sweep:
        out["paper_sweep"] = section(paper_sweep, args, local)
    if not args.no_free_surface:
        out["free_surface"] = section(free_surface_report, args, local)
    if not args.no_coarse:
        out["coarse_medium"] = section(coarse_report, args, local)
    if not args.no_fwi:
        out["fwi_iteration"] = section(fwi_report, args, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = section(cpu_oracle_rate, prob, args.cpu_seconds)
    sim.close()
    return out


def adjoint_ratio(args, local):
    """Adjoint workload: 192^3, dx = 15 m, 1500 steps, sponge 20, explosion,
    20 x 20 receivers, L2 misfit against data from the model with a 10 %
    sphere, checkpoints every 50 steps.  Times one forward run and one
    gradient (forward with checkpoints + segment recompute + adjoint)."""
    import torch
    from paper_2112_15071_gb300 import ews, synth
    true, start = synth.config4(n=args.adj_n, nt=args.adj_nt)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sim_t = ews.simulation_for(true)
    sim_t.set_stream(stream.cuda_stream)
    obs = torch.zeros((3, sim_t.nrec, true.nt), device=dev)
    sim_t.run(true.nt, true.dt, obs)
    sim_t.close()
    sim = ews.simulation_for(start)
    sim.set_stream(stream.cuda_stream)
    seis = torch.zeros_like(obs)
    g = torch.zeros((3, start.nz, start.ny, start.nx), device=dev)

    def timed(fn):
        fn()                                     # warm-up (allocations, plan)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    fwd_ms = timed(lambda: sim.run(start.nt, start.dt, seis))
    mis = [0.0]

    def grad():
        mis[0] = ews.ews_gradient(sim.handle, start.nt, start.dt, obs, g[0], g[1], g[2], 50)

    grad_ms = timed(grad)                    # default: history resident as far as it fits
    hist_gb = (start.nt + 1) * 3 * 4 * start.ncell / 1e9
    free_gb = torch.cuda.mem_get_info(dev)[0] / 1e9
    sim.set_history_budget(0)                # every segment recomputed from its checkpoint
    grad_rec_ms = timed(grad)
    g32 = g.clone()
    ck = {}
    for stor in ("bf16", "f16"):             # 16-bit checkpoints, same recomputation
        sim.set_checkpoint_storage(stor)
        ms = timed(grad)
        err = [float(torch.linalg.vector_norm(g[q] - g32[q]) / torch.linalg.vector_norm(g32[q]))
               for q in range(3)]
        ck[stor] = {"gradient_ms": round(ms, 2), "ratio": round(ms / fwd_ms, 3),
                    "rel_l2_vs_f32_checkpoints": [float(f"{e:.3g}") for e in err]}
    sim.set_checkpoint_storage("f32")
    ck_gb = (start.nt // 50) * 9 * 4 * start.ncell / 1e9
    sim.set_history_budget(-1)
    sim.close()
    torch.cuda.empty_cache()
    return {"workload": f"{start.nx}^3 dx={start.spacing[0]} m, {start.nt} steps, sponge "
                        f"{start.width}, explosion 6 Hz, {start.rec_pos.shape[0]} receivers, "
                        "L2 misfit vs 10% sphere model, checkpoints every 50",
            "forward_ms": round(fwd_ms, 2), "gradient_ms": round(grad_ms, 2),
            "ratio": round(grad_ms / fwd_ms, 3), "misfit": mis[0],
            "history": f"automatic budget (half the free HBM): the {hist_gb:.1f} GB velocity "
                       "history of all steps stays resident when it fits; checkpoints every 50 "
                       "steps are still taken",
            "free_gb_after": round(free_gb, 1),
            "recompute_all": {"gradient_ms": round(grad_rec_ms, 2),
                              "ratio": round(grad_rec_ms / fwd_ms, 3),
                              "history": "one 50-step segment; every earlier segment "
                                         "recomputed from its checkpoint",
                              "checkpoints_gb_f32": round(ck_gb, 2),
                              "checkpoints_16bit": ck}}


def storage_report(args, local, with_oracle: bool):
    """Large forward case (1024 x 1024 x 512, dx = 50 m, sponge 20, point
    force 2 Hz at 10 km, 32 x 32 receivers): throughput of the same loop with
    the wavefields stored in FP32, BF16 and FP16, and the seismogram error of
    each against the FP64 oracle on the 128^3 crop of the same recipe."""
    import numpy as np
    import torch
    from paper_2112_15071_gb300 import ews, synth
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    nt = args.storage_nt
    prob = synth.config3(nt=nt, device=dev)
    peak, peak_kind = peaks()
    es = {"f32": 4, "bf16": 2, "f16": 2}
    out = {"workload": f"{prob.nx}x{prob.ny}x{prob.nz} dx=50 m, sponge 20, layered + random "
                       "(device-generated), vertical force 2 Hz at 10 km, 32x32 receivers",
           "timed_steps": nt, "peak_gbs": peak, "peak_kind": peak_kind}
    for st in ("f32", "bf16", "f16"):
        sim = ews.simulation_for(prob, storage=st)
        sim.set_stream(stream.cuda_stream)
        seis = torch.zeros((3, sim.nrec, nt), device=dev)
        sim.run(nt, prob.dt, seis)                   # warm-up
        torch.cuda.synchronize()
        sim.profile(reset=True)
        sim.set_profiling(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.run(nt, prob.dt, seis)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        kms, kl = sim.profile(reset=True)
        sim.set_profiling(False)
        alg = algorithmic_bytes(prob, es[st])
        v_ms = kms[ews.EWS_KERNEL_VELOCITY] / max(kl[ews.EWS_KERNEL_VELOCITY], 1)
        s_ms = kms[ews.EWS_KERNEL_STRESS] / max(kl[ews.EWS_KERNEL_STRESS], 1)
        step_ms = ms / nt
        # the tuned tile shape against the 32 x 8 tiles of the other passes
        tuned = sim.tile_shape
        sim.set_tile_shape("32x8")
        sim.run(nt, prob.dt, seis)                   # warm-up (graph capture)
        a.record(stream)
        sim.run(nt, prob.dt, seis)
        b.record(stream)
        torch.cuda.synchronize()
        ms8 = a.elapsed_time(b)
        out[st] = {"gcells": round(prob.ncell * nt / (ms / 1e3) / 1e9, 3),
                   "tile_shape": tuned,
                   "gcells_32x8_tiles": round(prob.ncell * nt / (ms8 / 1e3) / 1e9, 3),
                   "ms_per_time_step": round(step_ms, 4),
                   "velocity_frac": round(alg["velocity"] / (v_ms / 1e3) / 1e9 / peak, 4)
                   if v_ms > 0 else None,
                   "stress_frac": round(alg["stress"] / (s_ms / 1e3) / 1e9 / peak, 4)
                   if s_ms > 0 else None,
                   "whole_step_frac": round(alg["step_min"] / (step_ms / 1e3) / 1e9 / peak, 4),
                   "algorithmic_bytes_per_cell": 18 * es[st] + 12,
                   "field_scales": [float(x) for x in sim.field_scales()]}
        if st == "f32":
            # the fused step (both passes in one launch, 84 B per cell) on the
            # same loop, against the two-pass kernels above
            sim.set_tile_shape("fused")
            sim.run(nt, prob.dt, seis)               # warm-up (graph capture)
            a.record(stream)
            sim.run(nt, prob.dt, seis)
            b.record(stream)
            torch.cuda.synchronize()
            msf = a.elapsed_time(b)
            sim.profile(reset=True)
            sim.set_profiling(True)
            sim.run(nt, prob.dt, seis)
            torch.cuda.synchronize()
            kf, klf = sim.profile(reset=True)
            sim.set_profiling(False)
            f_ms = kf[ews.EWS_KERNEL_STEP] / max(klf[ews.EWS_KERNEL_STEP], 1)
            out[st]["fused_step"] = {
                "tile_shape": sim.tile_shape,
                "gcells": round(prob.ncell * nt / (msf / 1e3) / 1e9, 3),
                "step_launch_ms": round(f_ms, 4),
                "frac": round(alg["step"] / (f_ms / 1e3) / 1e9 / peak, 4) if f_ms > 0 else None,
                "note": "frac = 84 B per cell / launch time / peak; the launch is bound by "
                        "instruction issue (the velocity of a 2-cell ring per tile is "
                        "recomputed), not by DRAM"}
        sim.close()
        del seis
    del prob
    torch.cuda.empty_cache()
    if with_oracle:
        from oracle import oracle
        oracle.build()
        crop = synth.config3_crop(nt=args.crop_nt)
        t0 = time.perf_counter()
        want = oracle.run_problem(crop)
        t_or = time.perf_counter() - t0
        err = {"crop": f"{crop.nx}^3, same recipe, force at k={int(crop.src_pos[2] / 50)}, "
                       f"{crop.rec_pos.shape[0]} receivers", "nt": crop.nt,
               "metric": "relative L2 of all seismograms vs the FP64 oracle",
               "oracle_seconds": round(t_or, 1)}
        for st in ("f32", "bf16", "f16"):
            sim = ews.simulation_for(crop, storage=st)
            got = sim.run(crop.nt, crop.dt)
            err[st] = float(np.linalg.norm(got.astype(np.float64) - want) / np.linalg.norm(want))
            sim.close()
        out["error_vs_oracle"] = err
    return out


def batch_report(args, local):
    """Batched shots (48-shot recipe: cubes 96..224, 800..1600 steps, 5..15 Hz,
    own layered + random model each, sponge 16, explosion at nz/3, 8 x 8
    receivers): the forward of the first --batch-shots shots, and forward plus
    L2 gradient (data from a +5 % sphere variant) of the first
    --batch-grad-shots, each as persistent launches in one graph and as one shot after
    another.  Aggregate Gcell-updates/s counts cells x steps of every shot
    over the wall time of the whole job."""
    import torch
    from paper_2112_15071_gb300 import ews, synth
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    probs = synth.config5_shots(48, device=dev)[:args.batch_shots]
    gprobs = probs[:args.batch_grad_shots]
    sims = [ews.simulation_for(p) for p in probs]
    seis = [torch.zeros((3, s.nrec, p.nt), device=dev) for s, p in zip(sims, probs)]
    # observed data of the gradient shots: the anomaly variants, batched
    obs = [torch.zeros_like(x) for x in seis[:len(gprobs)]]
    vsims = []
    for p in gprobs:
        v = ews.simulation_for(p)
        v.set_model_vel(*synth.sphere_anomaly_device(p.vp, p.vs, p.spacing))
        vsims.append(v)
    ews.ews_batch([{"sim": v, "nt": p.nt, "dt": p.dt, "seis": o}
                   for v, p, o in zip(vsims, gprobs, obs)], stream_handle=stream.cuda_stream)
    for v in vsims:
        v.close()
    grads = [torch.zeros((3, p.nz, p.ny, p.nx), device=dev) for p in gprobs]
    # Both modes recompute every checkpoint segment (history budget 0): run
    # alone, each shot could keep its whole history resident, which a batch
    # of shots sharing the GPU cannot; this compares the scheduling alone.
    for s in sims[:len(gprobs)]:
        s.set_history_budget(0)

    def job(mode, gradient):
        shots = []
        n = len(gprobs) if gradient else len(probs)
        for i in range(n):
            d = {"sim": sims[i], "nt": probs[i].nt, "dt": probs[i].dt, "seis": seis[i]}
            if gradient:
                g = grads[i]
                d.update(observed=obs[i], g_lam=g[0], g_mu=g[1], g_rho=g[2])
            shots.append(d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ews.ews_batch(shots, mode=mode, ckpt_every=50, stream_handle=stream.cuda_stream)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def cells_of(ps):
        return sum(p.ncell * p.nt for p in ps)

    out = {"workload": "48-shot recipe: cubes 96..224, 800..1600 steps, sponge 16, explosion, "
                       "64 receivers, device-generated models",
           "forward_shots": len(probs), "gradient_shots": len(gprobs),
           "gradient_history": "checkpoints every 50 steps, every segment recomputed (budget 0)",
           "gradient_memory": "one ews_batch call: the shots' gradient state does not fit "
                              "at once, so the call runs them in waves that do (halving on "
                              "EWS_ENOMEM); the one-by-one mode releases earlier shots' state "
                              "when it needs the room"}
    for name, gradient, ps in (("forward", False, probs), ("forward_gradient", True, gprobs)):
        if not gradient:                         # warm-up: autotune, graph captures
            job(ews.EWS_BATCH_PERSISTENT, gradient)
            job(ews.EWS_BATCH_SEQUENTIAL, gradient)
        tp = job(ews.EWS_BATCH_PERSISTENT, gradient)
        if gradient:                             # the last wave's gradient state
            for s in sims[:len(gprobs)]:
                s.release_workspace()
        ts = job(ews.EWS_BATCH_SEQUENTIAL, gradient)
        c = cells_of(ps)
        out[name] = {"cell_steps": c, "persistent_s": round(tp, 3), "one_by_one_s": round(ts, 3),
                     "persistent_gcells": round(c / tp / 1e9, 3),
                     "one_by_one_gcells": round(c / ts / 1e9, 3),
                     "speedup": round(ts / tp, 3)}
        if gradient:
            for s in sims[:len(gprobs)]:
                s.release_workspace()
    sizes = sorted({p.nx for p in probs})
    out["tuned_zchunk"] = {f"{n}^3": ews.ews_batch_tuned_zchunk(
        next(s.grid for s, p in zip(sims, probs) if p.nx == n), 1, False) for n in sizes}
    for s in sims:
        s.close()
    torch.cuda.empty_cache()
    return out


# The paper's GL timings (Sec. 4, total-time table divided by cells x steps):
# Mcell-updates/s per level on its integrated Vega GPU.  Context only.
PAPER_GPU_MCELLS = [74, 111, 127, 99, 58, 105, 97, 99, 112, 79, 77]


def paper_sweep(args, local):
    """The 11 grid levels of the paper's level-of-detail table with its 1D
    crustal model and moment tensor: Gcell-updates/s of --sweep-nt steps per
    level (time only), beside the paper's own GL figures for context."""
    import torch
    from paper_2112_15071_gb300 import ews, synth
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for lv in range(len(synth.PAPER_LEVELS)):
        p = synth.paper_level(lv, nt=args.sweep_nt)
        sim = ews.simulation_for(p)
        sim.set_stream(stream.cuda_stream)
        seis = torch.zeros((3, sim.nrec, p.nt), device=dev)
        sim.run(p.nt, p.dt, seis)                     # warm-up (graph capture)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.run(p.nt, p.dt, seis)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        g = p.ncell * p.nt / (ms / 1e3) / 1e9
        rows.append({"level": lv, "grid": [p.nx, p.ny, p.nz], "ms_per_step": round(ms / p.nt, 4),
                     "gcells": round(g, 3), "tile_shape": sim.tile_shape,
                     "paper_gl_mcells": PAPER_GPU_MCELLS[lv],
                     "x_paper": round(g * 1e3 / PAPER_GPU_MCELLS[lv], 1)})
        sim.close()
    return {"workload": "paper level table (Sec. 3.2.1): grids, spacings and dt as printed, 1D "
                        "crustal model, Eq. 7 moment tensor, sponge, 8 receivers; "
                        f"{args.sweep_nt} timed steps per level",
            "paper_hardware": "AMD Ryzen 7 4700U integrated Vega GPU, OpenGL (context only)",
            "levels": rows}


def free_surface_report(args, local):
    """The main workload with a vacuum free surface on the plane below the
    top damping zone (ks = W; the paper's surface boundary, Sec. 2.5) and
    the receivers on it, timed beside the same workload without it."""
    import torch
    from paper_2112_15071_gb300 import ews, synth
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    rows = {}
    for fs in (False, True):
        p = synth.config2(n=args.n, nt=args.fs_nt)
        if fs:
            ks = p.width
            p.free_surface = (ks, 1e-3)
            p.rec_pos = p.rec_pos.copy()
            p.rec_pos[:, 2] = (ks - 0.5) * p.spacing[2]
        sim = ews.simulation_for(p)
        sim.set_stream(stream.cuda_stream)
        seis = torch.zeros((3, sim.nrec, p.nt), device=dev)
        sim.run(p.nt, p.dt, seis)                     # warm-up (graph capture)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.run(p.nt, p.dt, seis)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        rows["surface" if fs else "plain"] = {
            "gcells": round(p.ncell * p.nt / (ms / 1e3) / 1e9, 3),
            "ms_per_step": round(ms / p.nt, 4)}
        sim.close()
    rows["ratio"] = round(rows["surface"]["gcells"] / rows["plain"]["gcells"], 4)
    rows["workload"] = (f"{args.n}^3 C-PML workload, {args.fs_nt} timed steps; surface at "
                        "ks = W (vacuum eps = 1e-3 above), receivers on the surface plane")
    return rows


def coarse_report(args, local):
    """The main workload with its medium on a grid 4x coarser per axis (the
    paper's small medium textures, Sec. 2.2.1), sampled in the passes,
    timed beside the same workload with the wavefield-grid medium."""
    import torch
    from paper_2112_15071_gb300 import ews, synth
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    rows = {}
    m = max(1, args.n // 4)
    for coarse in (False, True):
        p = synth.config2(n=args.n, nt=args.fs_nt)
        if coarse:
            synth.with_coarse_medium(p, (m, m, m))
        sim = ews.simulation_for(p)
        sim.set_stream(stream.cuda_stream)
        seis = torch.zeros((3, sim.nrec, p.nt), device=dev)
        sim.run(p.nt, p.dt, seis)                     # warm-up (graph capture)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.run(p.nt, p.dt, seis)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        rows["coarse" if coarse else "plain"] = {
            "gcells": round(p.ncell * p.nt / (ms / 1e3) / 1e9, 3),
            "ms_per_step": round(ms / p.nt, 4)}
        sim.close()
    rows["ratio"] = round(rows["coarse"]["gcells"] / rows["plain"]["gcells"], 4)
    rows["workload"] = (f"{args.n}^3 C-PML workload, {args.fs_nt} timed steps; medium on a "
                        f"{m}^3 grid (same recipe) sampled trilinearly at the staggered points")
    return rows


def fwi_report(args, local):
    """One multi-shot inversion iteration (ews_fwi_iteration) on the adjoint
    case's recipe at 128^3 (layers + random + 10 % sphere as the true model,
    smoothed layers as the start), --fwi-shots explosions on a grid at
    k = W + 10, 600 steps: batched gradients, their sum, the scaled
    direction and the parabolic line search.  Reported: the iteration's
    time, that time in units of one batched forward of all shots, and the
    misfit before and after."""
    import numpy as np
    import torch
    from paper_2112_15071_gb300 import ews, synth
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    true, start = synth.config4(n=128, nt=600)
    ns = args.fwi_shots
    h = start.spacing[0]
    w = start.width
    xs = np.linspace(w + 8, start.nx - w - 8, 4) * h
    ys = np.linspace(w + 8, start.ny - w - 8, max(1, (ns + 3) // 4)) * h
    srcs = [np.array([x, y, (w + 10) * h]) for y in ys for x in xs][:ns]

    def sims_for(p):
        out = []
        for s in srcs:
            sim = ews.Simulation(p.nx, p.ny, p.nz, p.spacing, boundary=p.boundary, width=p.width)
            sim.set_model_vel(p.vp, p.vs, p.rho)
            sim.set_source(p.src_kind, s, p.src_comp, p.wavelet)
            sim.set_receivers(p.rec_pos)
            out.append(sim)
        return out

    tsims = sims_for(true)
    obs = [torch.zeros((3, start.rec_pos.shape[0], start.nt), device=dev) for _ in srcs]
    ews.ews_batch([{"sim": t, "nt": start.nt, "dt": start.dt, "seis": o}
                   for t, o in zip(tsims, obs)], stream_handle=stream.cuda_stream)
    for t in tsims:
        t.close()
    sims = sims_for(start)
    seis = [torch.zeros_like(o) for o in obs]
    fwd = [{"sim": s, "nt": start.nt, "dt": start.dt, "seis": x} for s, x in zip(sims, seis)]
    ews.ews_batch(fwd, stream_handle=stream.cuda_stream)           # warm-up, tuning
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ews.ews_batch(fwd, stream_handle=stream.cuda_stream)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    lam, mu, rho = (torch.from_numpy(a).to(dev) for a in start.lame())
    shots = [{"sim": s, "nt": start.nt, "dt": start.dt, "observed": o} for s, o in zip(sims, obs)]
    # warm-up on a copy of the model (every shot's gradient state gets allocated)
    ews.ews_fwi_iteration(shots, lam.clone(), mu.clone(), rho.clone(), max_rel_step=0.02,
                          ckpt_every=50, stream_handle=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    j0, j1, a = ews.ews_fwi_iteration(shots, lam, mu, rho, max_rel_step=0.02, ckpt_every=50,
                                      stream_handle=stream.cuda_stream)
    torch.cuda.synchronize()
    t_it = time.perf_counter() - t0
    for s in sims:
        s.close()
    torch.cuda.empty_cache()
    return {"workload": f"{ns} explosions on the adjoint recipe at 128^3 (dx {h} m), {start.nt} "
                        "steps, sponge, 10 % sphere hidden in layers + random; start = smoothed layers",
            "iteration_s": round(t_it, 3), "batched_forward_s": round(t_fwd, 3),
            "forward_equivalents": round(t_it / t_fwd, 2), "misfit_before": j0,
            "misfit_after": j1, "accepted_step": a}


# --- reference arm: the FP64 oracle on the host cores -------------------------

def run_reference(args, world, rank):
    from paper_2112_15071_gb300 import synth
    from oracle import oracle
    prob = synth.config2(n=args.n, nt=args.nt)
    oracle.build()
    s = oracle.OracleSim(prob.nx, prob.ny, prob.nz, prob.spacing)
    s.set_medium_vel(prob.vp, prob.vs, prob.rho)
    s.set_boundary(prob.boundary, prob.width, prob.dt, prob.f0)
    # each step: a bounded sample of the workload (first few time steps of
    # the full grid), so the whole run stays within a few minutes
    t0 = time.perf_counter()
    s.forward(1, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp, prob.wavelet,
              prob.rec_pos)
    per = time.perf_counter() - t0
    budget = 120.0 / max(args.steps + args.warmup, 1)
    sample = max(1, min(20, int(budget / max(per, 1e-6))))
    for _ in range(args.warmup):
        s.forward(sample, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp,
                  prob.wavelet, prob.rec_pos)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.forward(sample, prob.dt, prob.src_kind, prob.src_pos, prob.src_comp,
                  prob.wavelet, prob.rec_pos)
    el = time.perf_counter() - t0
    value = prob.ncell * sample * args.steps / el / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"FP64 oracle on host cores, full {prob.nx}^3 grid with C-PML, {sample} of "
            f"{prob.nt} time steps per bench step")
    return {"metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded layered + random model)", "impl": "reference",
            "config": {"workload": WORKLOAD, "grid": [prob.nx, prob.ny, prob.nz],
                       "nt": prob.nt, "sample_steps": sample},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, world, rank)), flush=True)
        return 0
    world, rank, local = dist_setup(args.gpus)
    out = run_ours(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
