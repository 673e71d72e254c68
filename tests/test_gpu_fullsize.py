"""Parity with the oracle at the paper workloads' full sizes, in the launch
configurations the benchmark uses: every population of every active cell
bit for bit (after the stated 1e-11 relative bar), layouts equal after each
regrid, totals exact.  The oracle is plain single-threaded C with dense
levels, so each case holds up to ~13 GB of host memory and runs tens of
seconds."""
import numpy as np
import pytest

from paper_2609_35529_b300 import inputs as I

from test_gpu_parity import compare, drift, oracle_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, vlbm
    build.build()
    return vlbm


def test_vortex_512_two_persistent_launches_with_exact_audit(V):
    """The advected vortex at N = 512 with its central ratio-2 patch, 128
    coarse steps as two persistent launches of 64 steps with the exact
    per-step audit on: every step's totals equal math.fsum of the oracle's
    weighted W at the same step; the final state is bit for bit the
    oracle's."""
    cs = I.vortex(N=512, steps=128)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=1, graph_steps=64, schedule=1)
    g.set_step_totals(True)
    o = oracle_of(cs)
    g.advance(cs.steps)
    rows = g.step_totals()
    assert rows.shape == (cs.steps, 8)
    done = 0
    for st in (0, 1, 63, 64, 127):  # rows[st]: the totals at the start of step st
        o.advance(st - done)
        done = st
        ot, oa = o.totals()
        assert np.array_equal(rows[st, :4], ot), st
        assert np.array_equal(rows[st, 4:], oa), st
    o.advance(cs.steps - done)
    compare(o, g, 2)
    g.close()


def test_laxliu3_1024_three_levels(V):
    """Lax-Liu configuration 3 on the 1024^2 coarse grid with the two static
    levels over the diagonal band, 8 coarse steps on the persistent schedule
    and 8 more per phase."""
    cs = I.riemann3(N=1024, nlev=3, steps=8)
    o = oracle_of(cs)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=1, graph_steps=8, schedule=1)
    g.advance(8)
    o.advance(8)
    compare(o, g, 3)
    g.set_tuning(variant=1, graph_steps=4, schedule=0)
    g.advance(8)
    o.advance(8)
    compare(o, g, 3)
    g.close()


@pytest.mark.parametrize("schedule", [0, 1])
def test_shockbubble_2048_two_regrids(V, schedule):
    """The benchmarked adaptive shock-bubble itself (2048 x 1024 coarse, three
    levels, regrid every 4 coarse steps on the device), its initial layout
    and 8 coarse steps spanning two regrids in the benchmark's launch shape
    (4 steps per graph launch; per-phase or persistent): layouts and
    populations equal the oracle's after every regrid, totals unchanged
    across each regrid."""
    cs = I.shockbubble()
    tol, buf, every = cs.amr["tol"], cs.amr["buffer"], cs.amr["every"]
    o = oracle_of(cs)
    for _ in range(cs.nlev - 1):
        o.regrid_tagged(tol, buf, 8)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=1, graph_steps=every, schedule=schedule, persist_after=0)
    for _ in range(cs.nlev - 1):
        g.regrid()
    compare(o, g, 3)
    for cycle in range(2):
        g.advance(every)
        o.advance(every)
        t0, a0 = g.audit()
        g.regrid()
        o.regrid_tagged(tol, buf, 8)
        t1, _ = g.audit()
        assert drift(t0, t1, a0) < 1e-14
        compare(o, g, 3)
    g.close()
