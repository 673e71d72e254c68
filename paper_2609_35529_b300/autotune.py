"""Autotuner for the sweep launch: picks, per hierarchy signature, the
compiled sweep variant, the schedule (one launch per phase, or the
persistent task kernel), the task granularity of the persistent kernel
(whole 8 x 8 tiles per thread group, or half tiles per warp), the coarse
steps per graph launch and the grid cap (one CTA per four tiles, or a grid
of resident CTAs looping over the tiles), by timing candidates on a scratch
hierarchy of the same configuration (made by a caller-supplied factory and
destroyed afterwards), so tuning never touches the simulation it is for.
tune() times static runs; tune_adaptive() times cycles of coarse steps and
regrids, where a layout lives only a few steps and the persistent schedule
pays for a task list at every regrid.

The signature is what the cost depends on: the level sizes, the active
cells per level, beta and whether the sensor-driven relaxation is on.
Results are cached in memory and, optionally, in a JSON file.
"""
import json
import os
import time

import numpy as np

from . import vlbm as V

DEFAULT_CANDIDATES = [
    {"variant": 1, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 1, "schedule": 1, "graph_steps": 16, "max_ctas": 0},
    {"variant": 1, "schedule": 1, "graph_steps": 32, "max_ctas": 0},
    {"variant": 1, "schedule": 1, "graph_steps": 64, "max_ctas": 0},
    {"variant": 1, "schedule": 1, "graph_steps": 4, "max_ctas": 0},
    {"variant": 0, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 2, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 3, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 3, "schedule": 1, "graph_steps": 16, "max_ctas": 0},
    {"variant": 1, "schedule": 0, "graph_steps": 8, "max_ctas": 0},
    {"variant": 0, "schedule": 0, "graph_steps": 8, "max_ctas": 0},
]

_cache = {}


# With the sensor-driven relaxation the sweep carries the sensor's filters
# and its two passes are tasks of their own: the launch shapes rank
# differently (more resident CTAs pay for the spills).
SENSOR_CANDIDATES = [
    {"variant": 1, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 2, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 3, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 1, "schedule": 0, "graph_steps": 8, "max_ctas": 0},
]


def signature(h):
    info = h.info()
    return "|".join([",".join(map(str, info["nx"])), ",".join(map(str, info["ny"])),
                     ",".join(map(str, info["active_cells"])), "om-1" if info["beta"] == 1.0 else "om",
                     "sensor" if getattr(h, "sensor_on", False) else "const"])


def measure(h, cand, steps):
    """MLUPS of `steps` coarse steps under candidate settings (after a
    warm-up launch that builds the task lists and graphs)."""
    h.set_tuning(**cand)
    g = cand["graph_steps"]
    h.advance(g)
    h.sync()
    n = max(g, (steps // g) * g)
    t0 = time.perf_counter()
    h.advance(n)
    h.sync()
    el = time.perf_counter() - t0
    return h.info()["lups_per_step"] * n / el / 1e6


def tune(make, target=None, steps=64, candidates=None, cache_file=None, verbose=False):
    """Times the candidates on a scratch hierarchy from make() and installs the
    fastest valid one on `target` (when given).  Returns (best settings,
    {candidate index: MLUPS}); a cached signature skips the trials."""
    probe = make()
    sig = signature(probe)
    if cache_file and not _cache and os.path.exists(cache_file):
        with open(cache_file) as fh:
            _cache.update(json.load(fh))
    results = {}
    if sig in _cache:
        best = _cache[sig]
    else:
        cands = candidates or DEFAULT_CANDIDATES
        for i, c in enumerate(cands):
            try:
                results[i] = measure(probe, c, steps)
            except V.VlbmError:
                continue
            if verbose:
                print(f"autotune {sig}: {c} -> {results[i]:.1f} MLUPS", flush=True)
        best = cands[max(results, key=results.get)]
        _cache[sig] = best
        if cache_file:
            with open(cache_file, "w") as fh:
                json.dump(_cache, fh, indent=1)
    probe.close()
    if target is not None:
        target.set_tuning(**best)
    return best, results


ADAPTIVE_CANDIDATES = [
    {"variant": 1, "schedule": 1, "max_ctas": 0},
    {"variant": 0, "schedule": 1, "max_ctas": 0},
    {"variant": 2, "schedule": 1, "max_ctas": 0},
    {"variant": 3, "schedule": 1, "max_ctas": 0},
    {"variant": 1, "schedule": 0, "max_ctas": 0},
    {"variant": 0, "schedule": 0, "max_ctas": 0},
]


def tune_adaptive(make, every, target=None, cycles=8, candidates=None, verbose=False, prepare=None):
    """Times candidates on adaptive runs: a fresh scratch hierarchy from
    make() per candidate (with its initial layout; prepare(h), when given,
    sets it up like the run it is for, e.g. with regrid audits), two warm-up
    cycles, then `cycles` cycles of `every` coarse steps and a tag-driven
    regrid, counted with the device's cell-update counter.  The first
    candidate is run once more, untimed, before the trials, so that
    first-use costs (module loads, pool growth) count against none of them.
    Installs the fastest on `target` (with `every` coarse steps per graph
    launch).  Returns (settings, {candidate index: MLUPS})."""
    cands = candidates or ADAPTIVE_CANDIDATES
    results = {}
    for i, c in [(-1, cands[0])] + list(enumerate(cands)):
        probe = make()
        if prepare is not None:
            prepare(probe)
        try:
            probe.set_tuning(graph_steps=every, persist_after=0, **c)
            for _ in range(2):
                probe.advance(every)
                probe.regrid()
            probe.sync()
            l0 = probe.lups_done()
            t0 = time.perf_counter()
            for _ in range(cycles):
                probe.advance(every)
                probe.regrid()
            probe.sync()
            el = time.perf_counter() - t0
            if i < 0:
                continue
            results[i] = (probe.lups_done() - l0) / el / 1e6
        except V.VlbmError:
            continue
        finally:
            probe.close()
        if verbose:
            print(f"autotune adaptive: {c} -> {results[i]:.1f} MLUPS", flush=True)
    best = dict(cands[max(results, key=results.get)], graph_steps=every, persist_after=0)
    if target is not None:
        target.set_tuning(**best)
    return best, results
