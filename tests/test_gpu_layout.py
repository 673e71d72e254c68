"""Device-resident layouts: the adaptive regrid and the persistent schedule's
task lists computed on the GPU (no host round trip), checked against the
host's builders and, through whole adaptive runs, against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
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


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_device_layouts_and_task_lists_equal_the_host_builders(V, seed):
    """Random block flags on ragged, periodic and non-periodic hierarchies of
    2-4 levels: block maps, tile lists, reconstruction map, active cells and
    the task lists of 1-3 coarse steps built on the device equal the host's,
    element for element."""
    bad, big, first = V.selftest_layout(seed, 40)
    assert bad == 0, first
    assert big > 0  # some dense random layouts fill the overflow area


@pytest.mark.parametrize("schedule", [1, 0, 2])
def test_adaptive_run_without_host_round_trips(V, schedule):
    """The shock-bubble, 128 x 64, three adaptive levels, regrid every 4
    coarse steps: 8 cycles queued back to back with no synchronisation in
    between (regrids on the device, task lists rebuilt on the device for the
    persistent schedule), then compared with the oracle bit for bit; the
    device's cell-update counter equals the sum over the cycles."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    tol, buf, every = cs.amr["tol"], cs.amr["buffer"], cs.amr["every"]
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(schedule=schedule, graph_steps=every)
    o = oracle_of(cs)
    for _ in range(2):
        g.regrid()
        o.regrid_tagged(tol, buf, 8)
    lups = 0
    start = g.lups_done()
    for cycle in range(8):
        g.advance(every)
        o.advance(every)
        g.regrid()
        o.regrid_tagged(tol, buf, 8)
    compare(o, g, 3)
    done = g.lups_done() - start
    assert done > 0
    # one more cycle, counted against the reported layout
    per = g.info()["lups_per_step"]
    g.advance(every)
    o.advance(every)
    assert g.lups_done() - start - done == per * every
    compare(o, g, 3)


def test_regrid_conserves_without_synchronising(V):
    """Totals before and after each device regrid (exact audits) agree to the
    last bit of the exact sums' rounding, cycle after cycle."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(schedule=1, graph_steps=cs.amr["every"])
    for _ in range(2):
        g.regrid()
    for cycle in range(6):
        g.advance(cs.amr["every"])
        t0, a0 = g.audit()
        g.regrid()
        t1, _ = g.audit()
        assert drift(t0, t1, a0) < 1e-14


def test_device_regrid_nesting_and_layout_reads(V):
    """After device regrids the host-side views (layout masks, info, a
    checkpoint round trip) see the device's layout."""
    cs = I.shockbubble(nx0=64, ny0=32, nlev=3)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    for _ in range(2):
        g.regrid()
        o.regrid_tagged(cs.amr["tol"], cs.amr["buffer"], 8)
    g.advance(4)
    o.advance(4)
    g.regrid()
    o.regrid_tagged(cs.amr["tol"], cs.amr["buffer"], 8)
    for l in range(3):
        a, b = o.layout(l)
        ga, gb = g.layout(l)
        assert np.array_equal(a, ga) and np.array_equal(b, gb)
    blob = g.checkpoint()
    g.advance(4)
    o.advance(4)
    compare(o, g, 3)
    g.restore(blob)
    g.advance(4)
    compare(o, g, 3)


def test_task_kernels_share_completion_marks(V):
    """The persistent schedule switching between whole-tile and half-tile
    task kernels on the same device-built task list, and task lists that grow
    between regrids: completion marks left by either kernel never stall the
    other (a stale mark is always below the launch's), results bit for bit
    the oracle's."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    tol, buf, every = cs.amr["tol"], cs.amr["buffer"], cs.amr["every"]
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    for _ in range(2):
        g.regrid()
        o.regrid_tagged(tol, buf, 8)
    for cycle, var in enumerate([1, 3, 4, 0, 3, 2, 4, 1]):
        g.set_tuning(variant=var, schedule=1, graph_steps=every if cycle % 2 else 2, persist_after=0)
        g.advance(every)
        o.advance(every)
        if cycle % 3 != 2:  # some layouts live through a variant switch
            g.regrid()
            o.regrid_tagged(tol, buf, 8)
    g.sync()
    compare(o, g, 3)
