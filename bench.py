#!/usr/bin/env python3
"""Throughput benchmark of the refined VLBM on B300 (FP64).

Workload: the isentropic-vortex configuration -- periodic [0,10]^2, vortex
strength 5, free stream (1,1), gamma = 1.4, FP64 -- at the largest size of
its convergence series: 512 x 512 coarse cells with a ratio-2 patch over the
central 256 x 256 coarse cells (25 % of the area), time ratio 2.  One step is
one coarse step of the whole hierarchy: the level-0 sweep, two level-1
sweeps (fused collide + push-stream + mean-preserving coarse-to-fine
reconstruction), the reflux close and the end-of-step bookkeeping.

Metric: MLUPS (cell updates per second, counting every active cell of every
level once per level step) and the fraction of the roofline of the dominant
kernel (the level sweep), which on B300 is bounded by the FP64 pipe.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

With N > 1 (torchrun) every rank runs an independent replica (the workload
does not shard; no collective is on the data path) and `value` is the
whole-job aggregate.  `--impl reference` times the oracle (the plain FP64 CPU
rendering of the method) on the host cores, on the same workload and metric.
"""
import argparse
import json
import math
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

WORKLOAD = "isentropic vortex 512^2 coarse + central ratio-2 patch (2 levels), periodic, FP64"
METRIC = "MLUPS (FP64, 1 B300)"
# FP64 arithmetic of one cell update in the canonical collision (FMA = 2
# flops, the one division = 1): 12 adds (moments), 1 division, 14 flux
# operations of which one is fused (15 flops), 4 products (beta/2) W,
# 32 fused multiply-adds (relaxation).
FLOPS_PER_LUP = 12 + 1 + 15 + 4 + 64
# algorithmic bytes of one cell update: 16 populations read + 16 written
BYTES_PER_LUP = 256
# FP64-pipe operations of one cell update: the 62 arithmetic operations (the
# reciprocal 1/rho runs on the integer pipes); ncu counts 33.0 DFMA + 16.1
# DADD + 13.0 DMUL thread-instructions per cell update in the task kernel
FP64_OPS_PER_LUP = 62
# DRAM traffic of the task kernel per cell update: dram__bytes_read.sum +
# dram__bytes_write.sum of a launch of 64 coarse steps (variant 1, audit off,
# 512 MB L2 flush before each launch), ncu --nvtx capture of this bench's
# roofline launches (profiles/task_kernel_vortex512.md): 3.612e9 + 6.525e9 B
# per 46 137 344 cell updates.  Valid for the kernel as captured (integer-pipe
# reciprocal, audit tasks); to be measured again whenever the kernel changes.
TASK_KERNEL_DRAM_BYTES_PER_LUP = 219.7
TRAFFIC_VARIANT = 1


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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def oracle_rate(case, seconds):
    """The oracle (plain FP64 CPU code, one thread) on `case`: coarse steps
    until `seconds` of CPU time have passed.  Returns (MLUPS, steps, wall)."""
    from oracle import oracle as O
    o = O.Hierarchy(case.nx0, case.ny0, case.nlev, 2, case.bc, case.gamma, case.c, case.beta, case.inflow)
    o.set_layout(case.refs if case.nlev > 1 else None)
    for l in range(case.nlev):
        o.set_state(l, case.W[l])
    lups = case.lups_per_step()
    n, t0 = 0, time.perf_counter()
    while True:
        o.advance(1)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return lups * n / el / 1e6, n, el


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


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, budget_s=90.0):
    """The oracle on the host cores.  Each timed step is one coarse step of
    the workload; the run stops after `budget_s` seconds of timed steps (a
    bounded sample of the K requested) so that it ends within minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = I.vortex(N=512, steps=args.steps)
    lups = case.lups_per_step()
    from oracle import oracle as O
    o = O.Hierarchy(case.nx0, case.ny0, case.nlev, 2, case.bc, case.gamma, case.c, case.beta)
    o.set_layout(case.refs)
    for l in range(case.nlev):
        o.set_state(l, case.W[l])
    for _ in range(min(args.warmup, 1)):
        o.advance(1)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        o.advance(1)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    v = lups * done / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / done * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lups_per_step": lups, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"{done} of {args.steps} coarse steps of the workload (time budget "
                                       f"{budget_s:.0f} s), one thread"},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--variant", type=int, default=-1,
                    help="sweep variant; -1 (default) lets the autotuner pick variant, schedule and steps per launch")
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
    from paper_2609_35529_b300 import build, vlbm as V
    build.build()

    case = I.vortex(N=512, steps=args.steps)
    stream = torch.cuda.Stream()
    g = V.Hierarchy.from_case(case, stream=stream)
    if args.variant >= 0:
        g.set_tuning(variant=args.variant)
    else:
        # launch shape from the project's autotuner, timed on a scratch
        # hierarchy of the same configuration (the persistent schedule is
        # required for the per-step audit)
        from paper_2609_35529_b300 import autotune
        cands = [c for c in autotune.DEFAULT_CANDIDATES if c["schedule"] == 1]
        autotune.tune(lambda: V.Hierarchy.from_case(case, stream=stream), target=g, candidates=cands, steps=128)
    # every step includes the exact conservation audit
    g.set_step_totals(True)
    tune = g.get_tuning()
    chunk = max(1, tune["graph_steps"])
    info = g.info()
    lups = info["lups_per_step"]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # warm-up (also builds the task lists and instantiates the CUDA graphs)
    for _ in range(max(3, args.warmup)):
        g.advance(1)
    g.advance(chunk)
    g.sync()
    g.step_totals()  # drop the warm-up rows

    # timed: iterations of `chunk` coarse steps (one graph launch each), the
    # L2 flushed between iterations
    iters = max(1, args.steps // chunk)
    steps = iters * chunk
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets ncu select these launches (--nvtx-include timed/)
        with torch.cuda.stream(stream):
            for i in range(iters):
                flush.fill_(float(i))  # > L2 between timed iterations
                ev[i][0].record(stream)
                g.advance(chunk)
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    g.sync()
    rows = g.step_totals(cap=steps)
    drift = float(np.max(np.abs(rows[:, :4] - rows[0, :4]) / rows[0, 4:])) if len(rows) else None
    it_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(it_ms)
    if pg:
        pg.barrier()
    ms = job_time(ms, pg, "cuda")
    value = job_mlups(lups, steps, world, ms)

    # roofline of the dominant kernel, the persistent task kernel (all
    # sweeps and closes of `chunk` coarse steps in one launch): timed alone
    # -- the same launches with the per-step audit off, so that the graph
    # holds just the kernel (and its 8-byte counter reset) -- with CUDA
    # events on the library's stream, L2 flushed between launches
    pk = peaks()
    g.set_step_totals(False)
    g.advance(chunk)
    nk = min(iters, 64)
    evk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nk)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("roofline")  # lets ncu select these launches (--nvtx-include roofline/)
    with torch.cuda.stream(stream):
        for i in range(nk):
            flush.fill_(float(i))
            evk[i][0].record(stream)
            g.advance(chunk)
            evk[i][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    g.sync()
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in evk)
    audit_share = 1.0 - launch_ms / statistics.mean(it_ms)
    cells = lups * chunk
    achieved_tflops = FLOPS_PER_LUP * cells / (launch_ms * 1e-3) / 1e12
    hbm_gbs = BYTES_PER_LUP * cells / (launch_ms * 1e-3) / 1e9
    kernel = "task_kernel" if tune["schedule"] == 1 else "sweep_kernel"
    # the per-phase sweep kernel measured alone (eager launches with events)
    prof = g.profile(min(steps, 64))
    sweep = [r for r in prof if r["kind"] == "sweep"]
    sw_ms = sum(r["ms"] for r in sweep)
    sw_cells = sum(r["cells"] for r in sweep)
    traffic = None
    if tune["schedule"] == 1 and tune["variant"] == TRAFFIC_VARIANT:
        traffic = round(TASK_KERNEL_DRAM_BYTES_PER_LUP * cells)  # bytes per launch
    roof = {"bound": "alu", "achieved": round(achieved_tflops, 4), "peak": round(pk["fp64_tflops"], 4),
            "unit": "TFLOP/s", "frac": round(achieved_tflops / pk["fp64_tflops"], 4), "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu capture scaled by cell updates)",
            "kernel": kernel, "avg_launch_ms": round(launch_ms, 5), "cells_per_launch": cells,
            "flops_per_lup": FLOPS_PER_LUP, "peak_basis": "2 FP64 FMA/clk/SM x 148 SMs x sm_max_mhz",
            "hbm": {"achieved": round(hbm_gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": round(hbm_gbs / pk["hbm_gbs"], 4), "peak_source": pk["source"]},
            "sweep_kernel_alone_mlups": round(sw_cells / sw_ms / 1e3, 1),
            "audit_share_of_step": round(audit_share, 4),
            "fp64_pipe": {"ops_per_lup": FP64_OPS_PER_LUP,
                          "achieved_gops": round(FP64_OPS_PER_LUP * cells / (launch_ms * 1e-3) / 1e9, 1),
                          "peak_gops_nominal": round(2 * 148 * pk["sm_max_mhz"] * 1e6 / 1e9, 1),
                          "frac_of_nominal": round(FP64_OPS_PER_LUP * cells / (launch_ms * 1e-3)
                                                   / (2 * 148 * pk["sm_max_mhz"] * 1e6), 4)}}
    # schedule 1: the task kernel (sweeps and audit reductions) and the
    # kernel that rounds each step's audit totals
    launches_per_iter = 2 if tune["schedule"] == 1 else None
    if launches_per_iter is None:
        launches_per_iter = sum(r["launches"] for r in prof) / min(steps, 64) * chunk

    # end to end through the public API with host buffers: the initial state
    # from pinned host memory, every step's conservation totals read back to
    # the host (one copy per launch of `chunk` steps), the final state read
    # back.
    Wh = [torch.from_numpy(np.ascontiguousarray(w)).pin_memory().numpy() for w in case.W]
    # the results land in pinned host buffers too (allocated before timing)
    Wr = [torch.empty(w.shape, dtype=torch.float64).pin_memory().numpy() for w in case.W]
    h2 = V.Hierarchy(case.nx0, case.ny0, case.nlev, case.bc, case.gamma, case.c, case.beta, dx0=case.dx0,
                     stream=stream)
    h2.regrid_masks(case.refs)
    h2.set_step_totals(True)
    for l in range(case.nlev):
        h2.set_state(l, Wh[l])
    h2.advance(chunk)
    h2.step_totals()
    torch.cuda.synchronize()
    n_e2e = min(steps, 2048)
    t0 = time.perf_counter()
    for l in range(case.nlev):
        h2.set_state(l, Wh[l])
    got = 0
    for _ in range(n_e2e // chunk):
        h2.advance(chunk)
        got += len(h2.step_totals())
    Wout = [h2.get_conserved(l, out=Wr[l], valid=False)[0] for l in range(case.nlev)]
    e2e_s = time.perf_counter() - t0
    assert got == (n_e2e // chunk) * chunk
    n_e2e = (n_e2e // chunk) * chunk
    e2e_s = job_time(e2e_s, pg, "cuda")
    wbytes = sum(w.nbytes for w in case.W)
    e2e = {"value": round(job_mlups(lups, n_e2e, world, e2e_s * 1e3), 3), "unit": "MLUPS",
           "h2d_bytes_per_step": wbytes / n_e2e, "d2h_bytes_per_step": 64 + wbytes / n_e2e,
           "note": f"{n_e2e} steps through the C ABI: vlbm_set_state from pinned host W, vlbm_advance in "
                   f"launches of {chunk} steps, each step's conservation totals (64 B) read to the host "
                   f"after every launch, final W of every level read back into pinned host memory"}

    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            mlups, nst, el = oracle_rate(case, args.cpu_seconds)
            cpu = {"value": round(mlups, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                   "sample": f"{nst} coarse steps of the same workload ({el:.1f} s, one thread)"}
        line = {"metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
                "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (closed-form initial state)",
                "config": {"workload": WORKLOAD, "coarse": [case.nx0, case.ny0], "levels": case.nlev,
                           "lups_per_step": lups, "c": case.c, "beta": case.beta,
                           "l2": f"flushed between timed iterations of {chunk} coarse steps (512 MB write)",
                           "tuning": tune,
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(round(launches_per_iter * iters)),
                # per timed iteration (`chunk` coarse steps, L2 flushed before each)
                "iterations": {"n": iters, "steps_each": chunk,
                               "best_mlups": round(lups * chunk / (min(it_ms) * 1e-3) / 1e6, 1),
                               "median_mlups": round(lups * chunk / (statistics.median(it_ms) * 1e-3) / 1e6, 1)},
                "conservation": {"max_rel_drift_over_timed_steps": drift, "audited_steps": len(rows)},
                "clocks": clk.summary()}
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
