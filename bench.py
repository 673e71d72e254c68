#!/usr/bin/env python3
"""Throughput benchmark of the refined VLBM on B300 (FP64).

Workload: the adaptive shock-bubble -- a Mach 1.22 planar shock running into
a circular light-gas bubble (density ratio 0.14, radius 1/8 of the domain
height) on [0, 2] x [0, 1], gamma = 1.4, FP64 -- on a 2048 x 1024 coarse
grid with up to three levels of ratio 2, regridded every 4 coarse steps from
the normalised density-gradient indicator with the conservative split and
merge operators, its totals audited exactly across every regrid.  One step
is one coarse step of the whole hierarchy (one level-0 step, two level-1
steps, four level-2 steps, reconstruction and reflux at every interface);
the regrid that follows every fourth step of the run, and its two audits,
are inside the timed region.

Metric: MLUPS (cell updates per second, every active cell of every level
counted once per level step, counted on the device at the layout each step
ran on) and the roofline fraction of the dominant kernel (the level sweep),
which on B300 is bounded by the FP64 pipe.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With N > 1 (torchrun) every rank runs an independent replica (the workload
does not shard; no collective is on the data path) and `value` is the
whole-job aggregate.  `--impl reference` times the oracle (the plain FP64 CPU
rendering of the method) on the host cores, on the same workload and metric.
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_35529_b300 import inputs as I  # noqa: E402

WORKLOAD = ("AMR shock-bubble: Mach 1.22 shock into a bubble of density ratio 0.14 (radius 1/8 of the height), "
            "2048x1024 coarse, 3 levels of ratio 2, regrid every 4 coarse steps (normalised density gradient, "
            "tol 0.02, buffer 2, split/merge), exact audit before and after every regrid, FP64")
METRIC = "MLUPS (FP64, 1 B300)"
# FP64 arithmetic of one cell update in the canonical collision (FMA = 2
# flops, the one reciprocal = 1): 12 adds (moments), 1 reciprocal, 14 flux
# operations of which one is fused (15 flops), 4 products (beta/2) W, 32
# fused multiply-adds (relaxation).
FLOPS_PER_LUP = 12 + 1 + 15 + 4 + 64
# algorithmic bytes of one cell update: 16 populations read + 16 written
BYTES_PER_LUP = 256
# FP64-pipe operations of one cell update (the reciprocal runs on the
# integer pipes)
FP64_OPS_PER_LUP = 62
# DRAM traffic of the persistent task kernel per cell update on this
# workload type: dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of a task-kernel launch (four coarse steps, three CTAs per SM) of
# the 1024 x 512 coarse shock-bubble with three adaptive levels, divided by
# the launch's cell updates (the launch shape changes occupancy, not the
# bytes moved); valid while the kernel source is the one captured
# (TASK_SOURCE_SHA of csrc/vlbm_kernels.cu), else the line reports traffic
# as null.
TASK_DRAM_BYTES_PER_LUP = 195.8
TASK_SOURCE_SHA = "924ac9fe68b50a1c"


def kernel_source_sha():
    with open(os.path.join(ROOT, "paper_2609_35529_b300", "csrc", "vlbm_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def peaks():
    p = {"hbm_gbs": 6469.6, "sm_max_mhz": 2032.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p.update({k: m[k] for k in ("hbm_gbs", "sm_max_mhz") if k in m})
        p["source"] = "measured"
    except Exception:
        pass
    # FP64 pipe: 2 FP64 FMA per clock per SM (64 lanes / 32 clocks), 148 SMs
    p["fp64_tflops"] = 2 * 2 * 148 * p["sm_max_mhz"] * 1e6 / 1e12
    return p


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the sampler is running before the timed region starts
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_time(x, pg, device="cpu"):
    """The whole job's time: the maximum over ranks (identity on one rank)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_mlups(lups_per_step, steps, world, ms):
    """Whole-job throughput: every rank ran `steps` coarse steps of its own
    replica (weak scaling), in at most `ms` milliseconds."""
    return world * lups_per_step * steps / (ms * 1e-3) / 1e6


def run_steps(h, n, state, every):
    """n coarse steps of the run, regridding after every `every`-th step of
    the run (state["step"] counts the run's steps)."""
    while n > 0:
        k = min(n, every - state["step"] % every)
        h.advance(k)
        state["step"] += k
        n -= k
        if state["step"] % every == 0:
            h.regrid()


# --------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------

def oracle_setup(case):
    from oracle import oracle as O
    o = O.Hierarchy(case.nx0, case.ny0, case.nlev, 2, case.bc, case.gamma, case.c, case.beta, case.inflow)
    o.set_layout(None)
    o.set_state(0, case.W[0])
    for _ in range(case.nlev - 1):
        o.regrid_tagged(case.amr["tol"], case.amr["buffer"], 8)
    return o


def oracle_lups_per_step(o, nlev):
    act = o.active_masks()
    return sum(int(act[l].sum()) << l for l in range(nlev))


def oracle_cycles(o, case, steps, budget_s, state):
    """Up to `steps` coarse steps of the oracle with the run's regrids,
    stopping once budget_s seconds have passed; returns (lups, steps done,
    seconds)."""
    every = case.amr["every"]
    lups, done, t0 = 0, 0, time.perf_counter()
    while done < steps:
        k = min(steps - done, every - state["step"] % every)
        lups += oracle_lups_per_step(o, case.nlev) * k
        o.advance(k)
        state["step"] += k
        done += k
        if state["step"] % every == 0:
            o.regrid_tagged(case.amr["tol"], case.amr["buffer"], 8)
        if time.perf_counter() - t0 >= budget_s:
            break
    return lups, done, time.perf_counter() - t0


def _replica(args):
    """One oracle replica (a process of its own): set up, then one regrid
    cycle of the workload timed."""
    steps, q = args
    case = I.shockbubble()
    o = oracle_setup(case)
    lups, done, el = oracle_cycles(o, case, steps, 1e9, {"step": 0})
    q.put((lups, el))


def mem_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except Exception:
        pass
    return 0


def cpu_baseline(seconds):
    """The oracle on the host: one thread on one regrid cycle (4 coarse steps
    and the regrid) of the workload after its set-up, then as many
    concurrent single-thread replicas of the same sample as the cores and
    the host memory allow (each replica is a process of its own; the oracle
    itself is single-threaded)."""
    case = I.shockbubble()
    every = case.amr["every"]
    o = oracle_setup(case)
    lups, done, el = oracle_cycles(o, case, every, seconds, {"step": 0})
    one = {"value": round(lups / el / 1e6, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"{done} coarse steps of the workload and the regrid after them ({el:.1f} s, one thread), "
                     f"after the initial layout"}
    del o
    cores = os.cpu_count() or 1
    per = 13 * (1 << 30)  # host memory of one oracle instance of this workload (dense levels)
    reps = max(1, min(cores, 64, int(0.6 * mem_available_bytes() / per)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica, args=((every, q),)) for _ in range(reps)]
    for p in procs:
        p.start()
    res = [q.get() for _ in procs]
    for p in procs:
        p.join()
    agg = sum(r[0] for r in res) / max(r[1] for r in res) / 1e6
    one["all_cores"] = {"value": round(agg, 3), "unit": "MLUPS", "cores": reps, "nproc": cores,
                        "sample": f"{reps} concurrent single-thread replicas of the same sample "
                                  f"(limited by host memory: ~13 GB each)" if reps < cores else
                                  f"{reps} concurrent single-thread replicas of the same sample"}
    one["nproc"] = cores
    return one


def run_reference(args, budget_s=90.0):
    """The reference arm: the oracle, as it stands, on the host cores, on the
    same workload and metric: the initial layout, min(W, 1) warm-up steps,
    then up to K coarse steps with the run's regrids (a bounded sample: at
    most budget_s seconds of timed steps)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = I.shockbubble()
    o = oracle_setup(case)
    state = {"step": 0}
    oracle_cycles(o, case, min(args.warmup, 1), 1e9, state)
    lups, done, el = oracle_cycles(o, case, args.steps, budget_s, state)
    v = lups / el / 1e6
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / max(done, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "coarse": [case.nx0, case.ny0], "levels": case.nlev,
                       "regrid_every": case.amr["every"], "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": 1, "nproc": cores, "kind": "oracle",
                             "sample": f"{done} of {args.steps} coarse steps of the workload with their regrids "
                                       f"(time budget {budget_s:.0f} s), one thread"},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# extra workloads (context for the headline; static layouts)
# --------------------------------------------------------------------------

def static_rate(V, case, stream, steps=256, schedule=1, graph_steps=16):
    h = V.Hierarchy.from_case(case, stream=stream)
    h.set_tuning(schedule=schedule, graph_steps=graph_steps)
    h.advance(graph_steps)
    h.sync()
    l0 = h.lups_done()
    t0 = time.perf_counter()
    h.advance(steps)
    h.sync()
    el = time.perf_counter() - t0
    v = (h.lups_done() - l0) / el / 1e6
    h.close()
    return round(v, 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--schedule", type=int, default=-1,
                    help="0 per-phase, 1 persistent; -1 (default) lets the autotuner pick")
    ap.add_argument("--no-extras", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    dev = torch.cuda.current_device()
    from paper_2609_35529_b300 import autotune, build, vlbm as V
    build.build()

    case = I.shockbubble()
    every = case.amr["every"]
    stream = torch.cuda.Stream()

    def make():
        h = V.Hierarchy.from_case(case, stream=stream)
        for _ in range(case.nlev - 1):
            h.regrid()
        return h

    # launch shape: the project's autotuner on scratch hierarchies of the
    # same workload (regrid cycles), or a fixed schedule
    if args.schedule < 0:
        tune, trials = autotune.tune_adaptive(make, every, cycles=16, prepare=lambda g: g.set_regrid_audit(True))
    else:
        tune = {"variant": 1, "schedule": args.schedule, "max_ctas": 0, "graph_steps": every, "persist_after": 0}
        trials = {}
    torch.cuda.empty_cache()
    h = make()
    h.set_tuning(**tune)
    h.set_regrid_audit(True)
    state = {"step": 0}
    run_steps(h, max(3, args.warmup), state, every)
    h.sync()
    h.regrid_audits()  # drop the warm-up rows
    info0 = h.info()

    # timed: exactly K coarse steps; an iteration is the steps up to the
    # next regrid point of the run and that regrid (with its audits); the
    # working set (11 GB) is far larger than the 126 MB L2, so no flush
    marks = torch.zeros(2 + args.steps, dtype=torch.int64).pin_memory()
    chunks = []
    left, s = args.steps, state["step"]
    while left > 0:
        k = min(left, every - s % every)
        chunks.append(k)
        s += k
        left -= k
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    k0 = h.kernels_launched()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        with torch.cuda.stream(stream):
            h.lups_mark(marks.data_ptr())
            for i, k in enumerate(chunks):
                ev[i][0].record(stream)
                run_steps(h, k, state, every)
                ev[i][1].record(stream)
                h.lups_mark(marks.data_ptr() + 8 * (i + 1))
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    launches = h.kernels_launched() - k0
    it_ms = [a.elapsed_time(b) for a, b in ev]
    ms = ev[0][0].elapsed_time(ev[-1][1])
    m = marks.numpy()
    it_lups = [int(m[i + 1] - m[i]) for i in range(len(chunks))]
    lups = int(m[len(chunks)] - m[0])
    if pg:
        pg.barrier()
    ms = job_time(ms, pg, "cuda")
    value = job_mlups(lups, 1, world, ms)
    # conservation across the timed regrids
    rows = h.regrid_audits()
    if len(rows):
        drift = float(np.max(np.abs(rows[:, 8:12] - rows[:, 0:4]) / np.maximum(rows[:, 4:8], 1e-300)))
    else:
        drift = None
    info1 = h.info()

    # roofline of the dominant kernel of the timed schedule, on the layout of
    # the end of the timed steps (no regrid in between, so no task-list
    # build): schedule 1 -- the persistent task kernel, each launch (one
    # graph of `every` coarse steps) timed with CUDA events on the
    # hierarchy's stream; schedule 0 -- the level sweeps of eager per-phase
    # launches (vlbm_profile, CUDA events on the same stream)
    pk = peaks()
    traffic_per_lup = None
    if tune["schedule"] == 1:
        kname = "task_kernel"
        per_step = info1["lups_per_step"]
        with torch.cuda.stream(stream):
            h.advance(every)
            tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(16)]
            for a, b in tev:
                a.record(stream)
                h.advance(every)
                b.record(stream)
        torch.cuda.synchronize()
        launch_ms = statistics.median(a.elapsed_time(b) for a, b in tev)
        cells = per_step * every
        n_launches = len(tev)
        if TASK_DRAM_BYTES_PER_LUP is not None and TASK_SOURCE_SHA == kernel_source_sha():
            traffic_per_lup = TASK_DRAM_BYTES_PER_LUP
    else:
        kname = "sweep_kernel"
        prof = h.profile(8)
        sweep = [r for r in prof if r["kind"] == "sweep"]
        n_launches = sum(r["launches"] for r in sweep)
        launch_ms = sum(r["ms"] for r in sweep) / n_launches
        cells = sum(r["cells"] for r in sweep) / n_launches
    achieved_tflops = FLOPS_PER_LUP * cells / (launch_ms * 1e-3) / 1e12
    hbm_gbs = BYTES_PER_LUP * cells / (launch_ms * 1e-3) / 1e9
    traffic = round(traffic_per_lup * cells) if traffic_per_lup is not None else None
    roof = {"bound": "alu", "achieved": round(achieved_tflops, 4), "peak": round(pk["fp64_tflops"], 4),
            "unit": "TFLOP/s", "frac": round(achieved_tflops / pk["fp64_tflops"], 4), "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu capture per cell update x the launch's cell updates)",
            "kernel": kname, "avg_launch_ms": round(launch_ms, 5), "cells_per_launch": round(cells),
            "launches_timed": n_launches, "flops_per_lup": FLOPS_PER_LUP,
            "peak_basis": "2 FP64 FMA/clk/SM x 148 SMs x sm_max_mhz x 2 flops (no FP64 figure in MEASURED_PEAKS)",
            "hbm": {"achieved": round(hbm_gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": round(hbm_gbs / pk["hbm_gbs"], 4), "peak_source": pk["source"]},
            "fp64_pipe": {"ops_per_lup": FP64_OPS_PER_LUP,
                          "achieved_gops": round(FP64_OPS_PER_LUP * cells / (launch_ms * 1e-3) / 1e9, 1),
                          "peak_gops_nominal": round(2 * 148 * pk["sm_max_mhz"] * 1e6 / 1e9, 1),
                          "frac_of_nominal": round(FP64_OPS_PER_LUP * cells / (launch_ms * 1e-3)
                                                   / (2 * 148 * pk["sm_max_mhz"] * 1e6), 4)}}
    h.close()
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers: the initial state
    # from pinned host memory, the initial layout and K coarse steps with
    # their regrids, every level's final W read back into pinned host memory
    Wh = torch.from_numpy(np.ascontiguousarray(case.W[0])).pin_memory().numpy()
    shapes = [(4, case.ny0 << l, case.nx0 << l) for l in range(case.nlev)]
    Wr = [torch.empty(sh, dtype=torch.float64).pin_memory().numpy() for sh in shapes]
    h2 = V.Hierarchy(case.nx0, case.ny0, case.nlev, case.bc, case.gamma, case.c, case.beta, dx0=case.dx0,
                     inflow=case.inflow, tag_tol=case.amr["tol"], tag_buffer=case.amr["buffer"], stream=stream)
    h2.set_tuning(**tune)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2.set_state(0, Wh)
    for _ in range(case.nlev - 1):
        h2.regrid()
    st2 = {"step": 0}
    run_steps(h2, args.steps, st2, every)
    for l in range(case.nlev):
        h2.get_conserved(l, out=Wr[l], valid=False)
    e2e_s = time.perf_counter() - t0
    e2e_lups = h2.lups_done()
    h2.close()
    e2e_s = job_time(e2e_s, pg, "cuda")
    wbytes = Wh.nbytes
    rbytes = sum(w.nbytes for w in Wr)
    e2e = {"value": round(world * e2e_lups / e2e_s / 1e6, 3), "unit": "MLUPS",
           "h2d_bytes_per_step": wbytes / args.steps, "d2h_bytes_per_step": rbytes / args.steps,
           "note": f"{args.steps} coarse steps through the C ABI from a fresh hierarchy: vlbm_set_state from pinned "
                   f"host W, the initial layout ({case.nlev - 1} tag-driven regrids), the steps with their regrids, "
                   f"every level's final W read back into pinned host memory; wall clock"}

    extras = None
    if not args.no_extras:
        extras = {"vortex_512_patch_static_mlups": static_rate(V, I.vortex(N=512), stream),
                  "laxliu3_1024_three_levels_static_mlups": static_rate(V, I.riemann3(N=1024, nlev=3), stream)}

    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            cpu = cpu_baseline(args.cpu_seconds)
        its = [l / (t * 1e-3) / 1e6 for l, t in zip(it_lups, it_ms) if t > 0]
        line = {"metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (closed-form initial state)",
                "config": {"workload": WORKLOAD, "coarse": [case.nx0, case.ny0], "levels": case.nlev,
                           "regrid_every": every, "timed_steps": [state["step"] - args.steps, state["step"]],
                           "lups_per_step_at_start": info0["lups_per_step"],
                           "lups_per_step_at_end": info1["lups_per_step"],
                           "active_cells_at_end": info1["active_cells"], "c": case.c, "beta": case.beta,
                           "l2": "not flushed: the working set (about 11 GB) is far larger than the 126 MB L2",
                           "tuning": tune, "tuning_trials_mlups": {str(k): round(v, 1) for k, v in trials.items()},
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "iterations": {"n": len(its), "steps_each": chunks[0] if chunks else 0,
                               "best_mlups": round(max(its), 1) if its else None,
                               "median_mlups": round(statistics.median(its), 1) if its else None},
                "conservation": {"max_rel_change_across_regrid": drift, "regrids_audited": int(len(rows))},
                "extras": extras, "clocks": clk.summary()}
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
