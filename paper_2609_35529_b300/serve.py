"""Continuous-batching request loop over the VLBM engine.

Requests (2-D Riemann quadrant problems or isentropic vortices of different
sizes and refinement layouts) arrive by a seeded Poisson process.  The loop
admits arrived requests, in arrival order, while the engine's device-memory
budget and a cap on the residents' cell updates per coarse step allow
(setting each one up on its own high-priority stream, overlapping the
queued work), lets the engine advance every resident request by up to 16
coarse steps per call (each step: one launch per level phase covering the
tiles of every resident), and returns each result to the host once its last
step has completed; freed memory admits the next requests.  The same arrival
trace can be served one request at a time (each request alone on the GPU,
with the auto schedule) for comparison, and every request's result is
checked bit for bit against its run alone.

Times are wall-clock from a request's arrival to its result on the host.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I
from . import vlbm as V


@dataclass
class Request:
    rid: int
    arrival: float
    kind: str          # "riemann" or "vortex"
    N: int             # coarse cells per side
    nlev: int
    adaptive: bool
    steps: int
    seed: int
    case: object = None
    result: object = None
    done_at: float = None
    lups: int = 0
    lups_done: int = 0
    bytes_est: int = 0
    digest: dict = field(default_factory=dict)  # run name -> bit-pattern digest of the final W


def digest(W, act):
    """A 64-bit digest of the bit patterns of W on the meaningful cells: equal
    results give equal digests, and a change of any bit changes it (save
    for a 2^-64 chance).  Whole-array operations only, so that it runs in a
    worker thread beside the serving loop."""
    v = np.ascontiguousarray(W).view(np.uint64)
    if v.size == 0:
        return 0
    with np.errstate(over="ignore"):
        # SplitMix64's finaliser (Steele, Lea & Flood 2014) of value + position
        z = v + np.arange(v.size, dtype=np.uint64).reshape(v.shape) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
        z *= act.astype(np.uint64)[None]  # cells without meaning give 0
    return int(np.bitwise_xor.reduce(z, axis=None)) ^ int(z.sum(dtype=np.uint64))


# The alone-vs-mix digests are taken after a run's timed region: during
# it the results are only kept (a reference to the array already read), so
# that verification does not count as serving time.
def _verify(r, run, W, act):
    r.digest[run] = (W, act)


def _finish_verification(reqs, run):
    for r in reqs:
        v = r.digest.get(run)
        if isinstance(v, tuple):
            r.digest[run] = digest(*v)


def _digests(r):
    return r.digest


def level_bytes(nx0, ny0, nlev):
    """Device bytes of a hierarchy: two FP64 population buffers (16 planes)
    and two 16-bit flag planes per level over the level's index space."""
    tot = 0
    for l in range(nlev):
        nx, ny = nx0 << l, ny0 << l
        pitch = (nx + 15) & ~15
        tot += pitch * ny * (2 * 16 * 8 + 2 * 2)
    return tot


def random_quadrants(rng):
    s = {}
    for q in ("NE", "NW", "SW", "SE"):
        s[q] = (float(rng.uniform(0.5, 2.0)), float(rng.uniform(-0.5, 0.5)),
                float(rng.uniform(-0.5, 0.5)), float(rng.uniform(0.5, 2.0)))
    return s


def make_case(req):
    rng = np.random.default_rng(req.seed)
    if req.kind == "riemann":
        states = random_quadrants(rng)
        widths = [0.08, 0.04, 0.02][: req.nlev - 1]
        cs = I.riemann3(N=req.N, nlev=req.nlev, t_end=0.1, beta=0.7, widths=widths, states=states,
                        fine_state=False)
        if req.adaptive and req.nlev > 1:
            cs.refs = I.empty_refs(req.N, req.N, req.nlev)
            cs.amr = {"tol": 0.02, "buffer": 2, "every": 4}
    else:
        cs = I.vortex(N=req.N, beta=1.0, periods=0.1, patch=req.nlev > 1, fine_state=False)
        if req.nlev > 2:
            # a third level over the vortex core
            n = req.N
            cs.refs = I.box_refs(n, n, 3, [(0, n // 4, n // 4, n // 2, n // 2)])
            cs.refs[1][3 * n // 4: 5 * n // 4, 3 * n // 4: 5 * n // 4] = 1
            cs.nlev = 3
    cs.steps = req.steps if req.steps else cs.steps
    return cs


def make_requests(n=512, seed=20261202, rate=None, nmin=128, nmax=1024):
    """Seeded request trace: kind 1/2 Riemann, 1/2 vortex; side length
    log-uniform in [nmin, nmax] rounded to 32 cells; 1-3 levels; half of the
    multi-level Riemann requests adaptive.  Arrival times are filled in by
    `schedule` once the rate is known."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        kind = "riemann" if rng.random() < 0.5 else "vortex"
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / 32.0)) * 32
        N = max(nmin, min(nmax, N))
        nlev = int(rng.integers(1, 4))
        adaptive = kind == "riemann" and nlev > 1 and rng.random() < 0.5
        r = Request(i, 0.0, kind, N, nlev, adaptive, 0, int(rng.integers(1 << 30)))
        cs = make_case(r)
        r.steps = cs.steps
        r.bytes_est = level_bytes(N, N, cs.nlev)
        r.lups = cs.lups_per_step() * cs.steps
        reqs.append(r)
    return reqs


def schedule(reqs, rate, seed=20261202):
    """Poisson arrivals at `rate` requests per second."""
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1.0 / rate)
        r.arrival = t
    return reqs


class Payloads:
    """A request's payload -- its configuration and level-0 initial state --
    is what a client would send with it.  A background thread prepares the
    payloads of the trace in arrival order, at most `ahead` beyond the
    oldest one not yet taken, so that building the closed-form states with
    numpy stays out of the serving loop in both serving modes."""

    def __init__(self, reqs, ahead=48):
        import threading
        self.order = sorted(reqs, key=lambda r: r.arrival)
        self.ready = {}
        self.taken = 0
        self.cv = threading.Condition()
        self.ahead = ahead
        self.stop = False
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        for i, r in enumerate(self.order):
            with self.cv:
                while not self.stop and i >= self.taken + self.ahead:
                    self.cv.wait()
                if self.stop:
                    return
            cs = make_case(r)
            with self.cv:
                self.ready[r.rid] = cs
                self.cv.notify_all()

    def take(self, r):
        with self.cv:
            while r.rid not in self.ready:
                self.cv.wait()
            self.taken += 1
            self.cv.notify_all()
            return self.ready.pop(r.rid)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.th.join()


def _start(r, stream, cs=None):
    """Creates the request's hierarchy from its payload (the case; built here
    when not given): level-0 state from the closed form, finer levels by the
    conservative split (Eqs. 26-27) of a regrid to the request's static
    layout, or by tag-driven regrids when adaptive."""
    cs = cs if cs is not None else make_case(r)
    h = V.Hierarchy(cs.nx0, cs.ny0, cs.nlev, cs.bc, cs.gamma, cs.c, cs.beta, dx0=cs.dx0,
                    tag_tol=(cs.amr or {}).get("tol", 0.0), tag_buffer=(cs.amr or {}).get("buffer", 0),
                    stream=stream)
    # auto schedule: a request advanced alone takes per-phase launches while
    # its layout is young (adaptive requests regrid every 4 steps) and the
    # persistent task kernel once a layout has lived long enough
    h.set_tuning(schedule=2)
    h.set_state(0, cs.W[0])
    if r.adaptive:
        for _ in range(cs.nlev - 1):
            h.regrid()
    elif cs.nlev > 1:
        h.regrid_masks(cs.refs)
    return h, cs


def serve_one_at_a_time(reqs, stream=None, verify=False):
    """Each request alone on the GPU, in arrival order."""
    pending = sorted(reqs, key=lambda r: r.arrival)
    for r in reqs:
        r.lups_done = 0
    pay = Payloads(reqs)
    t0 = time.perf_counter()
    total_lups = 0
    for r in pending:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        h, cs = _start(r, stream, pay.take(r))
        left = cs.steps
        every = 4 if r.adaptive else 0
        while left > 0:
            n = min(left, every) if every else left
            r.lups_done += n * h.info()["lups_per_step"]
            h.advance(n)
            left -= n
            if every and left > 0:
                h.regrid()
        W, act = h.get_conserved(0)
        r.done_at = time.perf_counter() - t0
        if verify:
            _verify(r, "alone", W, act)
        total_lups += r.lups_done
        h.close()
    wall = time.perf_counter() - t0
    pay.close()
    if verify:
        _finish_verification(reqs, "alone")
    tts = np.array([r.done_at - r.arrival for r in reqs])
    return tts, total_lups / wall / 1e6, wall


def alone_vs_mix(reqs):
    ds = [_digests(r) for r in reqs]
    both = [d for d in ds if "alone" in d and "batched" in d]
    return {"compared": len(both), "bitwise_equal": sum(1 for d in both if d["alone"] == d["batched"])}


def main(argv=None):
    """Runs the benchmark and prints its JSON summary."""
    import json
    out, _ = run(argv)
    print(json.dumps(out))
    return out


def run(argv=None):
    """The serving benchmark.  Returns (summary, requests); the requests of
    the --keep-sample smallest ones still hold their batched results
    (`Request.result`, per-level populations) for a caller that checks them."""
    import argparse
    ap = argparse.ArgumentParser(description="continuous-batching VLBM serving benchmark")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--seed", type=int, default=20261202)
    ap.add_argument("--load", type=float, default=0.75, help="arrival rate as a fraction of batched capacity")
    ap.add_argument("--mem-gb", type=float, default=160.0)
    ap.add_argument("--keep-sample", type=int, default=0,
                    help="keep the batched results of this many of the smallest requests")
    ap.add_argument("--nmax", type=int, default=1024)
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--capacity-one", action="store_true",
                    help="also measure the one-at-a-time capacity (whole trace offered at t = 0)")
    ap.add_argument("--capacity-only", action="store_true",
                    help="stop after the capacity measurements (no latency runs)")
    ap.add_argument("--work-cap", type=float, default=24.0,
                    help="admission cap on the residents' cell updates per coarse step, in millions (0: none)")
    ap.add_argument("--engine-schedule", type=int, default=0,
                    help="0: shared per-phase launches; 1: one persistent launch per engine call (phase-major)")
    args = ap.parse_args(argv)
    import sys
    log = (lambda *a: print(*a, file=sys.stderr, flush=True)) if args.verbose else (lambda *a: None)
    import torch
    stream = torch.cuda.Stream()
    # requests are set up on a high-priority stream: their small kernels are
    # scheduled before the engine's next queued launch
    setup = torch.cuda.Stream(priority=-8)
    t0 = time.perf_counter()
    reqs = make_requests(args.requests, args.seed, nmax=args.nmax)
    total = sum(r.lups for r in reqs)
    budget = int(args.mem_gb * (1 << 30))
    log(f"trace: {len(reqs)} requests, {total / 1e9:.1f} GLUP nominal, built in {time.perf_counter() - t0:.1f} s")
    # capacity: the whole trace offered at once (all arrivals at t = 0)
    for r in reqs:
        r.arrival = 0.0
    wcap = args.work_cap * 1e6
    _, cap_mlups, cap_wall = serve_batched(reqs, budget, stream=stream, setup_stream=setup, work_cap=wcap,
                                           schedule=args.engine_schedule)
    log(f"capacity: {cap_mlups:.1f} MLUPS, {cap_wall:.1f} s, {serve_batched.breakdown}")
    cap1 = None
    if args.capacity_one:
        _, cap1, cap1_wall = serve_one_at_a_time(reqs, stream=stream)
        log(f"capacity one at a time: {cap1:.1f} MLUPS, {cap1_wall:.1f} s")
    if args.capacity_only:
        out = {"requests": len(reqs), "total_lups": total, "capacity_mlups": round(cap_mlups, 1),
               "capacity_one_at_a_time_mlups": round(cap1, 1) if cap1 else None,
               "capacity_breakdown": serve_batched.breakdown}
        return out, reqs
    rate = args.load * len(reqs) / cap_wall
    schedule(reqs, rate, args.seed)
    sample = set(r.rid for r in sorted(reqs, key=lambda r: r.lups)[: args.keep_sample])
    tts_b, ml_b, wall_b = serve_batched(reqs, budget, stream, sample, setup_stream=setup, verify=True, work_cap=wcap,
                                        schedule=args.engine_schedule)
    breakdown = serve_batched.breakdown
    log(f"batched: {ml_b:.1f} MLUPS, {wall_b:.1f} s, {breakdown}")
    kept = {r.rid: r.result for r in reqs if r.rid in sample}
    tts_1, ml_1, wall_1 = serve_one_at_a_time(reqs, stream=stream, verify=True)
    log(f"one at a time: {ml_1:.1f} MLUPS, {wall_1:.1f} s")
    out = {"requests": len(reqs), "total_lups": total, "capacity_mlups": round(cap_mlups, 1),
           "capacity_one_at_a_time_mlups": round(cap1, 1) if cap1 else None,
           "rate_per_s": round(rate, 3), "load": args.load, "work_cap_mlup_per_step": args.work_cap,
           "engine_schedule": args.engine_schedule,
           "batched": {"mlups": round(ml_b, 1), "p50_s": float(np.percentile(tts_b, 50)),
                       "p99_s": float(np.percentile(tts_b, 99)), "wall_s": wall_b, "breakdown": breakdown},
           "one_at_a_time": {"mlups": round(ml_1, 1), "p50_s": float(np.percentile(tts_1, 50)),
                             "p99_s": float(np.percentile(tts_1, 99)), "wall_s": wall_1},
           # every request's level-0 W (active and averaged-down cells) in the
           # batched run against the same request served alone
           "alone_vs_mix": alone_vs_mix(reqs)}
    for r in reqs:
        r.result = kept.get(r.rid)
    return out, reqs


# coarse steps queued per engine call: the GPU works through them while the
# host admits the requests that arrived meanwhile
MAX_STEPS = 16


def serve_batched(reqs, budget, stream=None, keep_ids=(), setup_stream=None, verify=False, work_cap=0,
                  schedule=0):
    """Continuous batching over the engine.  New requests are set up on their
    own stream (`setup_stream`) so that their set-up overlaps the engine's
    queued steps.  work_cap > 0 admits a request only while the residents'
    cell updates per coarse step stay within it (beyond the point where the
    GPU is busy, more residents only share it more thinly, which delays the
    long requests); the others wait in arrival order.  Returns per-request
    time-to-solution (s), the aggregate MLUPS and the wall time; the final
    populations of the requests in keep_ids are kept in `result`."""
    eng = V.Engine(budget, stream=stream, schedule=schedule)
    pending = sorted(reqs, key=lambda r: r.arrival)
    for r in reqs:
        r.lups_done = 0
        r.case = None
    live = {}
    used = 0
    work = 0.0
    nxt = 0
    pay = Payloads(reqs)
    t0 = time.perf_counter()
    total_lups = 0
    spent = {"start_s": 0.0, "step_s": 0.0, "finish_s": 0.0}  # host wall time by part of the loop
    # events on the engine's stream around every engine call: the time the
    # stream spends between one call's queued work and the next call's is
    # GPU time the host did not fill (other streams' work aside)
    import torch
    tstream = stream if isinstance(stream, torch.cuda.Stream) else None
    marks = [] if tstream is not None else None
    host_ms = {}  # library host time (vlbm_host_times) summed over the requests
    while nxt < len(pending) or live:
        # 1. queue steps of the residents first: the GPU works through them
        #    while the host sets up the requests that arrived meanwhile
        if live:
            ta = time.perf_counter()
            if marks is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(tstream)
            done, _ = eng.advance(MAX_STEPS)
            if marks is not None:
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record(tstream)
                marks.append((e0, e1))
            tb = time.perf_counter()
            spent["step_s"] += tb - ta
            for slot in done:
                r, h = live.pop(slot)
                r.lups_done = eng.slot_stats(slot)[1]
                W, act = h.get_conserved(0)
                r.done_at = time.perf_counter() - t0
                if verify:
                    _verify(r, "batched", W, act)
                if r.rid in keep_ids:
                    r.result = [h.get_populations(l) for l in range(h.nlev)]
                total_lups += r.lups_done
                eng.release(slot)
                for k, v in h.host_times().items():
                    host_ms[k] = host_ms.get(k, 0.0) + v
                h.close()
                used -= r.bytes_est
                work -= r.lups / max(1, r.steps)
            spent["finish_s"] += time.perf_counter() - tb
        # 2. admit arrived requests while the memory budget allows (a few per
        #    round, so that the queue of steps is refilled in between)
        now = time.perf_counter() - t0
        admitted = 0
        while nxt < len(pending) and pending[nxt].arrival <= now and admitted < 4:
            r = pending[nxt]
            if live and used + r.bytes_est > budget:
                break
            if live and work_cap > 0 and work + r.lups / max(1, r.steps) > work_cap:
                break
            ta = time.perf_counter()
            if r.case is None:
                r.case = pay.take(r)
            h, cs = _start(r, setup_stream if setup_stream is not None else stream, r.case)
            slot = eng.admit(h, cs.steps, 4 if r.adaptive else 0)
            spent["start_s"] += time.perf_counter() - ta
            if slot is None:  # over the engine's byte budget: retry later, payload kept
                h.close()
                break
            r.case = None
            live[slot] = (r, h)
            used += r.bytes_est
            work += r.lups / max(1, r.steps)
            nxt += 1
            admitted += 1
        if not live and nxt < len(pending):
            time.sleep(max(0.0, min(0.002, pending[nxt].arrival - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    idle = None
    if marks:
        torch.cuda.synchronize()
        idle = {"engine_calls": len(marks), "engine_host_ms": eng.host_times(),
                "stream_gap_s": sum(max(0.0, a[1].elapsed_time(b[0])) for a, b in zip(marks, marks[1:])) / 1e3,
                "stream_busy_s": sum(max(0.0, a.elapsed_time(b)) for a, b in marks) / 1e3}
    eng.close()
    pay.close()
    if verify:
        _finish_verification(reqs, "batched")
    tts = np.array([r.done_at - r.arrival for r in reqs])
    serve_batched.breakdown = {"loop": spent, "library_host_ms": host_ms, "engine_stream": idle}
    return tts, total_lups / wall / 1e6, wall


if __name__ == "__main__":
    main()
