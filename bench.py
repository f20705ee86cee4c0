#!/usr/bin/env python3
"""Benchmark of the batched PBD-R substep on one GB300 (or N, one per rank).

Workload: 4096 independent scenes, each with 1-32 rigid bodies of
{27, 64, 125, 343} particles (log-uniform body count, uniform sizes), seeded
random poses and velocities, r = 0.05 m, mu = 0.5, dt = 1/240 s, 10 solver
iterations: about 5 M particles.  One step = one PBD-R substep of every scene
(integration, neighbour build, 10 iterations), issued as one batched
pbdr_step call.  Metric: particle-iterations per second.

Printed (rank 0, one JSON line): the batched throughput (CUDA events on the
launching stream, inputs resident in HBM and larger than L2), the end-to-end
throughput through the C ABI with pinned host buffers copied in and out every
step, the one-scene-per-launch throughput on a sample of the same scenes,
p50/p99 substep latency, the dominant kernel's roofline fraction, SM clocks
sampled during the timed region, and the FP64 CPU oracle timed on the host
cores (cpu_baseline).  ``--impl reference`` times that oracle alone on the
same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PBD-R particle-iters/s batched vs per-scene launch; p50/p99 step latency"
UNIT = "particle-iters/s"
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pbdr", choices=["pbdr", "reference"])
    ap.add_argument("--scenes", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--per-scene-sample", type=int, default=256)
    ap.add_argument("--per-scene-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--e2e-split", type=int, default=4,
                    help="contexts (each on its own stream) the end-to-end run splits the batch "
                         "over, so that one part's host copies overlap another part's substep")
    ap.add_argument("--cpu-scenes", type=int, default=256)
    ap.add_argument("--cpu-substeps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample-scenes", type=int, default=256)
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson arrival trace of the serving run (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0,
                    help="Poisson arrival rate of the serving run (the serving workload's 2000/s)")
    ap.add_argument("--serve-pool", type=int, default=256,
                    help="distinct seeded requests the trace draws from")
    ap.add_argument("--serve-budget-gb", type=int, default=120)
    ap.add_argument("--path", choices=["resident", "streaming"], default="resident",
                    help="timed path: scene-resident kernel where scenes fit (default) or the "
                         "streaming form for every scene")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default launch shapes instead of tuned ones")
    ap.add_argument("--grad-steps", type=int, default=200,
                    help="substeps of the differentiated 16-body run (0: skip)")
    ap.add_argument("--dense-scenes", type=int, default=152,
                    help="scenes of the contact-dense secondary line (0: skip)")
    ap.add_argument("--dense-steps", type=int, default=50)
    ap.add_argument("--strong", action="store_true",
                    help="under torchrun: split ONE batch (the seed's) over the ranks by "
                         "longest-processing-time on particle counts (strong scaling) instead of "
                         "giving every rank its own batch (weak scaling)")
    ap.add_argument("--settle", type=int, default=240,
                    help="substeps run before the warm-up so that bodies have landed and touch")
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    return a


def workload_config(scs, args, extra=None):
    n = sum(s.num_particles for s in scs)
    b = sum(s.num_bodies for s in scs)
    cfg = {
        "workload": (f"batched: {args.scenes} scenes x 1-32 rigid bodies of {{27,64,125,343}} "
                     f"particles, seed {args.seed}, r=0.05 m, mu=0.5, dt=1/240 s, 10 iterations"),
        "scenes": len(scs), "particles": n, "bodies": b, "iterations": 10, "dt": 1.0 / 240.0,
        "step": "one PBD-R substep of all scenes in one batched pbdr_step",
        "path": getattr(args, "path", "resident"),
        "state": (f"after {args.settle} settling substeps ({args.settle / 240.0:.2f} s simulated) "
                  "from the seeded start, so bodies rest on the ground and on each other"),
        "l2": "inputs larger than L2 (state ~%d MB >> 129 MB)" % (n * 80 // (1 << 20)),
        "parallelism": "scene batch per GPU",
    }
    if extra:
        cfg.update(extra)
    return cfg


def make_workload(args, seed):
    from paper_2603_14634_gb300 import scenes
    # ranks of one node share the host cores
    local = max(1, int(os.environ.get("LOCAL_WORLD_SIZE", "1")))
    return scenes.batched_scenes(args.scenes, seed=seed,
                                 workers=max(1, min((os.cpu_count() or 1) // local, 32)))


# ---------------------------------------------------------------------------
# CPU oracle timings (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_scenes(scs, settle, threads):
    """The FP64 oracle's copies of the scenes, advanced `settle` substeps
    (untimed: the state the GPU arm times is the one after its settling)."""
    from oracle import oracle as O
    O.build()
    objs = [O.OracleScene(s) for s in scs]
    if settle > 0:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda o: o.substep(settle), objs))
    return objs


def oracle_time(objs, scs, substeps, threads):
    """Times the oracle advancing its scenes `substeps` further, spread over
    `threads` host threads (ctypes releases the GIL).
    Returns (particle-iters/s, seconds, particle-iters)."""
    work = sum(s.num_particles * s.iterations for s in scs) * substeps
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda o: o.substep(substeps), objs))
    dt = time.perf_counter() - t0
    return work / dt, dt, work


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
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
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------

def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


# the sources each timed kernel is compiled from
KERNEL_SOURCES = {
    "k_scene_substep": ("pbdr_fused.cu", "pbdr_math.cuh", "pbdr_internal.cuh"),
    "k_iterate": ("pbdr_kernels.cu", "pbdr_math.cuh", "pbdr_internal.cuh"),
}


def kernel_source_sha(kernel):
    """hash of the CUDA sources of one kernel (a changed kernel voids its
    committed ncu traffic figure)"""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2603_14634_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_figure(kernel, key="dram_bytes_per_unit"):
    """A per-unit figure (DRAM bytes, warp instructions) of a kernel from the
    committed ncu summary, if it was taken on the current kernel sources."""
    sha = kernel_source_sha(kernel)
    for path in glob.glob(os.path.join(ROOT, "profiles", f"*{kernel}*.md")):
        txt = open(path).read()
        m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
        m_val = re.search(key + r":\s*([0-9.]+)", txt)
        if m_sha and m_val and m_sha.group(1) == sha:
            return float(m_val.group(1))
    return None


def ncu_traffic(kernel):
    return ncu_figure(kernel, "dram_bytes_per_unit")


# FP32 operations of the method per particle, counted from the arithmetic of
# the scene-resident kernel (an FMA counts 2): per solver iteration the
# contact pass without contacts (ground test, X_bsm, the 12 shape-matching
# sums) 37, the goal pass (V_bsm, goals, X_asm, V_asm, the 18 sums of the
# momentum step) 117, the momentum correction 27; per substep the
# integration 12.  Contacts, the per-body rotation and momentum solves and
# the neighbour build are not counted.
FLOPS_PER_PARTICLE_ITERATION = 37 + 117 + 27
FLOPS_PER_PARTICLE_SUBSTEP = 12
FP32_LANES_PER_SM = 128


def alu_roofline(iterations, particles, sec_per_step, n_sm, sm_mhz):
    """Counted FP32 throughput of one substep against the FP32 peak of the
    SMs (lanes x 2 flop x clock)."""
    flops_per_unit = FLOPS_PER_PARTICLE_ITERATION * iterations + FLOPS_PER_PARTICLE_SUBSTEP
    achieved = flops_per_unit * particles / sec_per_step
    peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6
    return {"bound": "alu", "achieved": round(achieved / 1e12, 3), "peak": round(peak / 1e12, 2),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "flops_per_unit": round(flops_per_unit, 1), "unit_of_work": "particle-substep",
            "what": "counted FP32 operations of the method (iteration passes and integration; "
                    "contacts, per-body solves and neighbour build not counted) against "
                    "SMs x 128 FP32 lanes x 2 x max SM clock"}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_pbdr(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2603_14634_gb300.binding import Context

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    if args.strong:   # strong scaling: this rank's LPT share of one batch
        from paper_2603_14634_gb300.shard import lpt_partition
        scs_job = make_workload(args, args.seed)
        mine = lpt_partition([s.num_particles for s in scs_job], world)[rank]
        scs = [scs_job[i] for i in mine]
    else:             # weak scaling: own batch per rank
        scs = make_workload(args, args.seed + rank)
        scs_job = scs
    ctx = Context(local_rank)
    if args.no_autotune:
        from paper_2603_14634_gb300.binding import OPT_AUTOTUNE
        ctx.set_option(OPT_AUTOTUNE, 0)
    elif args.settle > 0:   # shapes tuned on the settled state that is timed (first warm-up step)
        from paper_2603_14634_gb300.binding import OPT_TUNE_AFTER
        ctx.set_option(OPT_TUNE_AFTER, args.settle)
    if args.path == "streaming":
        ctx.set_path(streaming=True)
    ids = [ctx.create_scene(s) for s in scs]
    plan_cfg = None
    n_particles = sum(s.num_particles for s in scs)
    work_per_step = sum(s.num_particles * s.iterations for s in scs)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    def barrier():
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        if args.settle > 0:
            ctx.step(ids, args.settle, sh)
        for _ in range(args.warmup):
            ctx.step(ids, 1, sh)
        stream.synchronize()
        kbar = ctx.neighbor_total(ids, sh) / max(n_particles, 1)
        launches_per_step = ctx.last_launch_count()
        plan_cfg = [c for c in ctx.plan_config(ids) if c["scenes"]]

        # ---- timed region: K batched substeps, inputs resident in HBM ----
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        # cudaProfilerStart/Stop bracket the timed region, so that a profiler
        # started with collection off sees exactly its launches
        torch.cuda.profiler.start()
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            ctx.step(ids, 1, sh)
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        barrier()
        clk = clocks.stop() if clocks else None
        ms_total = t_start.elapsed_time(t_end)
        lat = sorted(a.elapsed_time(b) for a, b in ev)
        # per-stage CUDA events on the launching stream over a run of the same
        # substeps right after the timed region (stage events replace the
        # graph replay, so they are not inside the timed region itself)
        prof_steps = max(3, min(args.steps, 50))
        ctx.set_profiling(True)
        ctx.read_profile()
        ctx.step(ids, prof_steps, sh)
        prof = ctx.read_profile()
        ctx.set_profiling(False)

    ms_max = ms_total
    total_work = work_per_step * args.steps
    if dist is not None:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
        w = torch.tensor([float(total_work)], device="cuda")
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        total_work = float(w.item())
    value = total_work / (ms_max * 1e-3)

    # ---- end to end through the C ABI with pinned host buffers ----
    # The batch is split over `e2e_split` contexts, each driven on its own
    # stream: every step of every part writes its inputs from pinned host
    # memory, steps, and reads its results back (asynchronously, completed
    # before the part's next write on the same stream), so one part's copies
    # overlap another part's substep.  The parts start from the settled state
    # of the timed batch.
    pos_h = torch.empty((n_particles, 3), dtype=torch.float32, pin_memory=True).numpy()
    vel_h = torch.empty((n_particles, 3), dtype=torch.float32, pin_memory=True).numpy()
    with torch.cuda.stream(stream):
        ctx.read_states(ids, pos_h, vel_h, sh)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    split = max(1, min(args.e2e_split, len(scs)))
    bounds = [len(scs) * k // split for k in range(split + 1)]
    poff = np.concatenate([[0], np.cumsum([s.num_particles for s in scs])])
    parts = []
    for k in range(split):
        a, b = bounds[k], bounds[k + 1]
        c = Context(local_rank)
        if args.no_autotune:
            from paper_2603_14634_gb300.binding import OPT_AUTOTUNE
            c.set_option(OPT_AUTOTUNE, 0)
        if args.path == "streaming":
            c.set_path(streaming=True)
        pids = [c.create_scene(s) for s in scs[a:b]]
        sl = slice(int(poff[a]), int(poff[b]))
        err = torch.zeros(b - a, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        parts.append((c, pids, sl, err, torch.cuda.Stream()))
    for c, pids, sl, err, st in parts:   # the settled state; past tuning and graph capture
        c.write_states(pids, pos_h[sl], vel_h[sl], st.cuda_stream)
        c.step(pids, 130, st.cuda_stream)
        c.write_states(pids, pos_h[sl], vel_h[sl], st.cuda_stream)
    torch.cuda.synchronize()

    def e2e_round():
        for c, pids, sl, err, st in parts:
            c.write_states(pids, pos_h[sl], vel_h[sl], st.cuda_stream)
            c.step(pids, 1, st.cuda_stream)
            c.read_states_async(pids, pos_h[sl], vel_h[sl], err, st.cuda_stream)
    for k in range(2):
        e2e_round()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        e2e_round()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_err = int(sum(int(np.count_nonzero(p[3])) for p in parts))
    for p in parts:
        p[0].close()
    e2e_work = float(work_per_step * e2e_steps)
    job_particles, job_scenes = n_particles, len(ids)   # summed over the ranks below
    if dist is not None:   # slowest rank's time, all ranks' work (each rank has its own batch)
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
        w = torch.tensor([e2e_work, float(n_particles), float(len(ids))], device="cuda", dtype=torch.float64)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
        e2e_work, job_particles, job_scenes = float(w[0]), int(w[1]), int(w[2])
    e2e_value = e2e_work / e2e_s

    # ---- the streaming form (one launch per stage and per iteration) ----
    ctx.set_path(streaming=True)
    with torch.cuda.stream(stream):
        ctx.step(ids, 2, sh)
        torch.cuda.synchronize()
        a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_stream_steps = max(3, min(20, args.steps))
        a0.record(stream)
        ctx.step(ids, n_stream_steps, sh)
        b0.record(stream)
        torch.cuda.synchronize()
        streaming_value = work_per_step * n_stream_steps / (a0.elapsed_time(b0) * 1e-3)
    ctx.set_path(streaming=args.path == "streaming")

    # ---- one scene per launch on a sample of the same scenes ----
    sample = ids[:: max(1, len(ids) // max(1, args.per_scene_sample))][: args.per_scene_sample]
    s_work = sum(scs[i].num_particles * scs[i].iterations for i in sample)
    with torch.cuda.stream(stream):
        for sid in sample:
            ctx.step([sid], 1, sh)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.per_scene_steps):
            for sid in sample:
                ctx.step([sid], 1, sh)
        b.record(stream)
        torch.cuda.synchronize()
        ps_ms = a.elapsed_time(b)
    per_scene_value = s_work * args.per_scene_steps / (ps_ms * 1e-3)
    # the batched path on the same sample, for a like-for-like ratio
    with torch.cuda.stream(stream):
        ctx.step(sample, 1, sh)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.per_scene_steps):
            ctx.step(sample, 1, sh)
        b.record(stream)
        torch.cuda.synchronize()
        bs_ms = a.elapsed_time(b)
    batched_sample_value = s_work * args.per_scene_steps / (bs_ms * 1e-3)

    shards = None
    if dist is not None:
        from paper_2603_14634_gb300.shard import gather_to_rank0
        shards = gather_to_rank0({"rank": rank, "scenes": len(ids), "particles": n_particles,
                                  "timed_ms": round(ms_total, 3)}, dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    # ---- roofline of the dominant kernel ----
    peak, peak_src = hbm_peak()
    dom = max(prof, key=lambda k: prof[k][0])
    d_ms, d_launches = prof[dom]
    if dom == "scene_resident":
        # k_scene_substep: one launch per size class per substep; compulsory
        # HBM bytes per particle-substep: read X, V, Q (48 B), write X, V
        # (32 B), write the neighbour lists (4 + 4 kbar B)
        kernel = "k_scene_substep"
        bytes_per_unit = 84.0 + 4.0 * kbar
        units = n_particles
        unit_name = "particle-substep"
        sec_per_step = d_ms * 1e-3 / prof_steps
        achieved = bytes_per_unit * units / sec_per_step / 1e9
        avg_launch_us = d_ms * 1e3 / max(d_launches, 1)
    else:
        # k_iterate: one launch per solver iteration; bytes per
        # particle-iteration: read X, V, Q (48 B), the list count and entries
        # (4 + 4 kbar B), write X, V (32 B)
        kernel = "k_iterate"
        bytes_per_unit = 84.0 + 4.0 * kbar
        units = n_particles
        unit_name = "particle-iteration"
        avg_launch_s = d_ms * 1e-3 / max(d_launches, 1)
        achieved = bytes_per_unit * units / avg_launch_s / 1e9
        avg_launch_us = avg_launch_s * 1e6
    tr = ncu_traffic(kernel)
    roofline = {
        "bound": "hbm", "kernel": kernel, "achieved": round(achieved, 1), "peak": peak,
        "unit": "GB/s", "frac": round(achieved / peak, 4),
        "traffic": None if tr is None else round(tr * units),
        "algorithmic_bytes": f"{bytes_per_unit:.2f} per {unit_name}", "kbar": round(kbar, 4),
        "avg_launch_us": round(avg_launch_us, 2), "peak_source": peak_src,
        "stage_ms_per_step": {k: round(v[0] / prof_steps, 4) for k, v in prof.items()},
        "stage_timing": f"CUDA events per stage over {prof_steps} substeps after the timed region",
    }
    # the bound this latency-bound kernel actually meets: instruction issue
    # (152 SMs x 4 schedulers x 1 warp instruction per cycle at the sampled
    # SM clock), against the warp instructions per unit ncu counted
    wi = ncu_figure(kernel, "warp_instructions_per_unit")
    issue = None
    if wi is not None and dom == "scene_resident":
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
        peak_issue = n_sm * 4 * sm_mhz * 1e6
        ach_issue = wi * units / sec_per_step
        issue = {"bound": "issue", "achieved": round(ach_issue / 1e9, 1), "peak": round(peak_issue / 1e9, 1),
                 "unit": "G warp-instructions/s", "frac": round(ach_issue / peak_issue, 4),
                 "warp_instructions_per_unit": wi, "source": "ncu smsp__inst_executed.sum of the committed capture"}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True, "scaling": "strong" if args.strong else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(scs_job, args, {"parallelism": (
            "one batch split over the ranks (LPT by particle count), one GPU per rank"
            if args.strong else "scene batch per GPU")} if world > 1 else None),
        "p50_step_ms": round(lat[len(lat) // 2], 4),
        "p99_step_ms": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 4),
        "per_scene_launch": {
            "value": round(per_scene_value, 1), "unit": UNIT, "sample_scenes": len(sample),
            "batched_same_sample": round(batched_sample_value, 1),
            "batched_over_per_scene": round(batched_sample_value / per_scene_value, 2)},
        "streaming_form": {"value": round(streaming_value, 1), "unit": UNIT,
                           "what": "same batch, one launch per stage and per solver iteration"
                                   + (" (rank 0's GPU)" if world > 1 else "")},
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                "h2d_bytes_per_step": int(job_particles * 24),
                "d2h_bytes_per_step": int(job_particles * 24 + 4 * job_scenes), "steps": e2e_steps,
                "path": "pbdr_write_states + pbdr_step + pbdr_read_states_async from and to pinned host "
                        "buffers, every step; the batch split over %d contexts on their own streams, so "
                        "that one part's copies overlap another's substep" % split,
                "scenes_with_error_bits": e2e_err},
        "gpu_launches": int(launches_per_step * args.steps),
        "launch_config": {"graph_per_substep": True, "autotuned_classes": plan_cfg},
        "roofline": roofline,
        "clocks": clk,
    }
    if shards is not None:
        line["shards"] = shards
    if issue is not None:
        line["roofline_issue"] = issue
    if dom == "scene_resident":
        line["roofline_alu"] = alu_roofline(
            work_per_step / max(n_particles, 1), n_particles, sec_per_step,
            torch.cuda.get_device_properties(local_rank).multi_processor_count,
            (clk or {}).get("sm_max_mhz") or 2070.0)
    # the same throughput priced by the streaming form's byte model (state
    # streamed every iteration: 100 + 4 kbar B per particle-iteration plus
    # (184 + 4 kbar) / K per substep), which the fused kernel keeps on chip;
    # the compulsory-byte figure above is the kernel's own roofline
    K = work_per_step / max(n_particles, 1)
    b_model = 100.0 + 4.0 * kbar + (184.0 + 4.0 * kbar) / K
    line["streaming_model_equivalent"] = {
        "bytes_per_particle_iteration": round(b_model, 2),
        "equivalent_GBps": round(b_model * value / world / 1e9, 1), "peak": peak,
        "frac": round(b_model * value / world / 1e9 / peak, 4),
        "what": "per-GPU throughput x bytes a state-streaming substep would move (not DRAM traffic)",
    }
    if world == 1 and args.dense_scenes > 0 and args.dense_steps > 0:
        line["contact_dense"] = run_contact_dense(args, local_rank, peak)
    if world == 1 and args.serve_seconds > 0:
        line["serving"] = run_serving(args, local_rank)
    if world == 1 and args.grad_steps > 0:
        line["gradient"] = run_gradient(args, local_rank)
    if world == 1 and not args.no_cpu_baseline:
        cpu_scs = scs[: args.cpu_scenes]
        thr = host_cores()
        objs = oracle_scenes(cpu_scs, args.settle, thr)
        v, secs, work = oracle_time(objs, cpu_scs, args.cpu_substeps, thr)
        line["cpu_baseline"] = {
            "value": round(v, 1), "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": (f"first {len(cpu_scs)} scenes of the workload, settled {args.settle} substeps "
                       f"by the oracle as the GPU arm's batch is, then {args.cpu_substeps} timed "
                       f"substeps; FP64 C oracle, one scene per host thread "
                       f"({work} particle-iters in {secs:.1f} s)")}
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_contact_dense(args, local_rank, peak):
    """Secondary line with particle-particle contact everywhere: a batch of
    stacked blocks (125 bodies of 4^3 each, 8000 particles, faces one
    particle diameter apart, K = 20), timed after settling, so that the
    contact gather is inside a timed number."""
    import torch
    from paper_2603_14634_gb300 import scenes
    from paper_2603_14634_gb300.binding import Context
    scs = scenes.stacked_block_scenes(args.dense_scenes, seed=args.seed + 5000,
                                      workers=max(1, min(os.cpu_count() or 1, 32)))
    n = sum(s.num_particles for s in scs)
    work = sum(s.num_particles * s.iterations for s in scs)
    K = scs[0].iterations
    out = {"what": "stacked blocks of 125 bodies of 4^3 (8000 particles each) resting on the "
                   "ground with touching faces, K = 20, one batched pbdr_step per substep",
           "scenes": len(scs), "particles": n, "iterations": K, "settle_substeps": 24}
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    with Context(local_rank) as ctx, torch.cuda.stream(stream):
        ids = [ctx.create_scene(s) for s in scs]
        for path in ("resident", "streaming"):
            ctx.set_path(streaming=path == "streaming")
            ctx.step(ids, 24 if path == "resident" else 2, sh)
            stream.synchronize()
            kbar = ctx.neighbor_total(ids, sh) / n
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.dense_steps):
                ctx.step(ids, 1, sh)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b) / args.dense_steps
            _, _, err = ctx.read_states(ids, stream=sh)
            value = work / (ms * 1e-3)
            b_model = 100.0 + 4.0 * kbar + (184.0 + 4.0 * kbar) / K
            rec = {"value": round(value, 1), "unit": UNIT, "ms_per_step": round(ms, 4),
                   "kbar": round(kbar, 3), "scenes_with_error_bits": int((err != 0).sum()),
                   "streaming_model_frac": round(b_model * value / 1e9 / peak, 4),
                   "compulsory_frac": round((84.0 + 4.0 * kbar) * n / (ms * 1e-3) / 1e9 / peak, 4)}
            out[path] = rec
    out["note"] = ("streaming_model_frac prices the throughput at 100 + 4 kbar + (184 + 4 kbar)/K B "
                   "per particle-iteration, compulsory_frac at 84 + 4 kbar B per particle-substep, "
                   "both against the measured HBM copy bandwidth")
    return out


def run_gradient(args, local_rank):
    """Differentiation: d(final body centres of mass)/d(initial rigid
    velocities v_b, omega_b) of 16 bodies of 5^3 sliding on the ground
    (4x4 grid, 0.6 m pitch, mu = 0.5, K = 10, dt = 1/240), by forward-mode
    tangents: the 96 directions run as 96 copies of the scene in one
    batched tangent step."""
    import numpy as np
    import torch
    from paper_2603_14634_gb300 import diff
    from paper_2603_14634_gb300.binding import Context
    sc = diff.c5_scene(seed=args.seed)
    v = np.stack([sc.vel[s].astype(np.float64).mean(0) for s in diff.body_slices(sc)])
    w = np.zeros_like(v)
    wts = np.ones((sc.num_bodies, 3))
    with Context(local_rank) as c:
        diff.final_com_and_jacobian(c, sc, v, w, 3)        # warm: build, allocate
        diff.com_gradient_reverse(c, sc, v, w, 3, wts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, J = diff.final_com_and_jacobian(c, sc, v, w, args.grad_steps, with_mu=True)
        secs = time.perf_counter() - t0
        t0 = time.perf_counter()
        diff.com_gradient_reverse(c, sc, v, w, args.grad_steps, wts, checkpoint_every=20, with_mu=True)
        secs_rev = time.perf_counter() - t0
    dirs = J.shape[1]
    return {
        "what": "d(final body CoMs)/d(initial v_b, omega_b, friction mu), 16 bodies of 5^3: full Jacobian by forward-mode tangents (all directions batched), and one gradient by the reverse-mode adjoint (checkpoints every 20 substeps)",
        "outputs": int(J.shape[0]), "directions": int(dirs), "substeps": args.grad_steps,
        "jacobian_ms": round(secs * 1e3, 2),
        "tangent_particle_iters_per_s": round(dirs * sc.num_particles * sc.iterations * args.grad_steps / secs, 1),
        "adjoint_gradient_ms": round(secs_rev * 1e3, 2),
        "timing": "wall clock around each whole call (scene setup, seeds, steps, read-back)",
    }


def run_serving(args, local_rank):
    """Serving: Poisson arrivals of scene requests (1e3-2e5 particles, bodies
    of 64-512 particles, 1-100 substeps each) drawn from a seeded pool,
    admitted by an HBM budget and served by continuous batching."""
    import numpy as np
    import torch
    from paper_2603_14634_gb300 import scenes
    from paper_2603_14634_gb300.serve import Server, poisson_trace
    rng = np.random.default_rng(args.seed + 1000)
    pool = [scenes.serving_request(rng)[0] for _ in range(args.serve_pool)]
    arrivals = poisson_trace(args.serve_rate, args.serve_seconds, seed=args.seed)
    pick = rng.integers(0, len(pool), size=len(arrivals))
    steps = rng.integers(1, 101, size=len(arrivals))
    stream = torch.cuda.Stream()
    errs = [0]

    def delivered(rid, pos, vel, err):   # results are delivered, not kept (20k requests)
        errs[0] += 1 if err else 0
    srv = Server(hbm_budget_bytes=args.serve_budget_gb << 30, device=local_rank,
                 stream=stream.cuda_stream, on_result=delivered)
    offered = 0
    for t, k, st in zip(arrivals, pick, steps):
        srv.submit(pool[k], int(st), arrival=float(t))
        offered += pool[k].num_particles * pool[k].iterations * int(st)
    with torch.cuda.stream(stream):
        stats = srv.run(realtime=True)
    errs = errs[0]
    return {
        "requests": stats["requests"], "arrival_rate_hz": args.serve_rate,
        "trace_s": args.serve_seconds, "budget_gb": args.serve_budget_gb,
        "request_latency_ms_p50": round(stats["latency_ms_p50"], 3),
        "request_latency_ms_p99": round(stats["latency_ms_p99"], 3),
        "tick_ms_p50": round(stats["tick_ms_p50"], 3), "tick_ms_p99": round(stats["tick_ms_p99"], 3),
        "offered_particle_iters_per_s": round(offered / args.serve_seconds, 1),
        "achieved_particle_iters_per_s": round(stats["achieved_particle_iters_per_s"], 1),
        "wall_s": round(stats["wall_s"], 3), "requests_with_error_bits": errs,
        "ms_per_tick_split": {k: round(v, 3) for k, v in stats["host_ms_per_tick"].items()},
        "what": "continuous batching: admit between substeps by HBM budget, one batched substep of all resident requests per tick, retire and free finished ones",
    }


def run_reference(args, rank):
    """The reference arm: the FP64 oracle as it stands on the host cores;
    each step advances a bounded sample of the workload by one substep."""
    if rank != 0:
        return None
    scs = make_workload(args, args.seed)
    sample = scs[: args.ref_sample_scenes]
    thr = host_cores()
    objs = oracle_scenes(sample, args.settle, thr)   # the state the GPU arm times
    for _ in range(args.warmup):
        oracle_time(objs, sample, 1, thr)
    times = []
    work = 0
    for _ in range(args.steps):
        v, secs, w = oracle_time(objs, sample, 1, thr)
        times.append(secs)
        work += w
    total = sum(times)
    value = work / total
    cpu = {"value": round(value, 1), "unit": UNIT, "cores": thr, "kind": "oracle",
           "sample": (f"first {len(sample)} scenes of the workload, settled {args.settle} substeps by "
                      f"the oracle as the GPU arm's batch is, then one substep per step, FP64 C oracle")}
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(scs, args, {"reference_sample_scenes": len(sample)}),
        "cpu_baseline": cpu,
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        from paper_2603_14634_gb300 import build as B
        if rank == 0 or world == 1:
            B.build()
        else:   # rank 0 builds (the link is an atomic rename); the others wait for it
            t0 = time.time()
            while not B.up_to_date():
                if time.time() - t0 > 900:
                    raise RuntimeError("the library built by rank 0 did not appear")
                time.sleep(0.5)
        line = run_pbdr(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
