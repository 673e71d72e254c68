"""Autotuner for the sweep launch: picks, per hierarchy signature, the
compiled sweep variant, the schedule (one launch per phase, or the
persistent task kernel), the coarse steps per graph launch and the grid cap,
by timing candidates on a scratch hierarchy of the same configuration (made
by a caller-supplied factory and destroyed afterwards), so tuning never
touches the simulation it is for.

The signature is what the cost depends on: the level sizes, the active
cells per level and whether 1 - 2 beta == -1 (some variants need it).
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
    {"variant": 10, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 13, "schedule": 1, "graph_steps": 8, "max_ctas": 0},
    {"variant": 13, "schedule": 1, "graph_steps": 16, "max_ctas": 0},
    {"variant": 1, "schedule": 0, "graph_steps": 8, "max_ctas": 0},
    {"variant": 0, "schedule": 0, "graph_steps": 8, "max_ctas": 0},
]

_cache = {}


def signature(h):
    info = h.info()
    return "|".join([",".join(map(str, info["nx"])), ",".join(map(str, info["ny"])),
                     ",".join(map(str, info["active_cells"])), "om-1" if info["beta"] == 1.0 else "om"])


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
