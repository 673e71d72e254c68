"""Serving benchmark plus the oracle's check of a sample of its results.

  python tests/serving_oracle_sample.py [serve options] [--sample 32]

Runs ``paper_2609_35529_b300.serve`` (the continuous-batching request loop,
its p50/p99 and capacity figures) keeping the batched results of the
`--sample` smallest requests, then runs each of those requests through the
oracle (test infrastructure, CPU) and reports the worst field-wise relative
difference over every level's active cells (0.0 = identical bits).  The
serving package itself never runs the oracle; this script is the checker.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2609_35529_b300 import serve as S  # noqa: E402


def run_oracle(req):
    """The oracle's answer for one request: the same recipe, layout policy
    (static boxes or tag-driven regrids every 4 coarse steps) and step count."""
    cs = S.make_case(req)
    o = O.Hierarchy(cs.nx0, cs.ny0, cs.nlev, 2, cs.bc, cs.gamma, cs.c, cs.beta, cs.inflow)
    o.set_layout(None)
    o.set_state(0, cs.W[0])
    if req.adaptive:
        for _ in range(cs.nlev - 1):
            o.regrid_tagged(cs.amr["tol"], cs.amr["buffer"], 8)
    elif cs.nlev > 1:
        o.regrid(cs.refs)
    left = cs.steps
    every = 4 if req.adaptive else 0
    while left > 0:
        n = min(left, every) if every else left
        o.advance(n)
        left -= n
        if every and left > 0:
            o.regrid_tagged(cs.amr["tol"], cs.amr["buffer"], 8)
    return o


def agreement(result, oracle_h):
    """Worst field-wise relative difference between a served result
    (per-level populations) and the oracle over every level's active cells;
    a nonzero bit difference within tolerance reports at least 1e-300."""
    worst = 0.0
    for l, fg in enumerate(result):
        a, b = oracle_h.layout(l)
        act = (a == 1) & (b == 0)
        if not act.any():
            continue
        fo = oracle_h.get_f(l)
        Wg = fg.reshape(4, 4, *fg.shape[1:]).sum(axis=0)
        Wo = fo.reshape(4, 4, *fo.shape[1:]).sum(axis=0)
        for k in range(4):
            scale = max(float(np.max(np.abs(Wo[k][act]))), 1e-300)
            worst = max(worst, float(np.max(np.abs(Wg[k][act] - Wo[k][act]))) / scale)
        if not np.array_equal(fg[:, act], fo[:, act]):
            worst = max(worst, 1e-300)
    return worst


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    n = 32
    if "--sample" in argv:
        i = argv.index("--sample")
        n = int(argv[i + 1])
        del argv[i:i + 2]
    out, reqs = S.run(argv + ["--keep-sample", str(n)])
    worst, checked = 0.0, 0
    for r in reqs:
        if r.result is not None:
            worst = max(worst, agreement(r.result, run_oracle(r)))
            checked += 1
    out["oracle_sample"] = checked
    out["oracle_worst_rel_err"] = worst
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
