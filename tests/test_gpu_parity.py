"""Parity of the CUDA path (through the C ABI) with the oracle.

Both sides evaluate the same canonical FP64 expressions, so the populations
are expected to agree bit for bit; the bar the tests enforce first is the
stated one -- max relative error <= 1e-11 on every conserved field, relative
to the field's largest magnitude -- and then exact equality.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_35529_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, vlbm
    build.build()
    return vlbm


def oracle_of(case, refs="case"):
    o = O.Hierarchy(case.nx0, case.ny0, case.nlev, 2, case.bc, case.gamma, case.c, case.beta, case.inflow)
    o.set_layout(case.refs if refs == "case" else refs)
    for l in range(case.nlev):
        o.set_state(l, case.W[l])
    return o


def compare(o, g, nlev, exact=True):
    """Asserts layout equality, field-wise relative error <= TOL, then bitwise
    equality of every population on every active cell.  Returns the worst
    relative error."""
    worst = 0.0
    for l in range(nlev):
        oin, oref = o.layout(l)
        gin, gref = g.layout(l)
        assert np.array_equal(oin, gin), f"level {l}: level membership differs"
        assert np.array_equal(oref, gref), f"level {l}: refinement differs"
        act = (oin == 1) & (oref == 0)
        Wo, _ = o.get_W(l)
        Wg, vg = g.get_conserved(l)
        assert np.array_equal(vg, act)
        for k in range(4):
            a, b = Wo[k][act], Wg[k][act]
            if a.size == 0:
                continue
            scale = max(np.max(np.abs(a)), 1e-300)
            err = float(np.max(np.abs(a - b))) / scale
            worst = max(worst, err)
            assert err <= TOL, f"level {l} field {k}: rel err {err:.3e}"
        if exact:
            fo = o.get_f(l)[:, act]
            fg = g.get_populations(l)[:, act]
            nd = int(np.count_nonzero(fo != fg))
            assert nd == 0, f"level {l}: {nd} populations differ (max {np.max(np.abs(fo - fg)):.3e})"
    return worst


def drift(t0, t1, a0):
    """Largest relative change of a total; a field whose |W| total is zero
    (e.g. rho v of a flow without v) must stay exactly zero."""
    d = np.abs(t1 - t0)
    return max(float(np.max(np.where(a0 > 0, d / np.where(a0 > 0, a0, 1.0), d))), 0.0)


def test_library_loads_and_creates(V):
    h = V.Hierarchy(16, 16, 1, (0, 0, 0, 0), 1.4, 5.0, 0.9)
    info = h.info()
    assert info["nx"] == [16] and info["lups_per_step"] == 256
    h.close()


def test_pure_streaming_bitwise(V):
    cs = I.smooth_random(24, 16, 1, [], seed=3, beta=0.0)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs, refs=None)
    rng = np.random.default_rng(8)
    # equilibrium populations of a smooth state, perturbed by 1 %: every
    # streamed mixture stays a physical state
    feq = O.feq(cs.gamma, cs.c, cs.W[0][:, 0, 0])
    f0 = feq[:, None, None] * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, (16, 16, 24)))
    g.set_populations(0, f0)
    o.set_f(0, f0)
    g.advance(48)
    assert np.array_equal(g.get_populations(0), f0)
    g.advance(3)
    o.advance(51)
    compare(o, g, 1)


def test_uniform_grid_smooth(V):
    cs = I.smooth_random(40, 24, 1, [], seed=1, amp=0.2, beta=0.85, steps=30)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs, refs=None)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 1)


def test_two_level_pulse_full_run(V):
    """Two-level static refinement, periodic 64^2, 200 coarse steps."""
    cs = I.pulse2l()
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    t0, a0 = g.audit()
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 2)
    t1, _ = g.audit()
    assert drift(t0, t1, a0) < 1e-13
    ot, oa = o.totals()
    np.testing.assert_allclose(t1, ot, rtol=1e-14, atol=1e-14 * oa.max())


@pytest.mark.parametrize("schedule,graph_steps,variant",
                         [(1, 8, 1), (0, 8, 1), (1, 3, 1), (2, 4, 1), (1, 8, 2), (0, 8, 0), (1, 8, 3), (1, 3, 4)])
def test_three_level_periodic_ragged(V, schedule, graph_steps, variant):
    """Three levels on a domain whose size is not a multiple of the tile
    (ragged last tile column/row), including a patch that wraps across the
    periodic seam; every schedule (per-phase launches, the persistent task
    kernel with an odd number of steps per launch, and auto switching from
    the first to the second after 7 steps, inside one advance call) and the
    launch-shape variants (2 and 4 CTAs/SM; warps on half-tile tasks at 3
    and 2 CTAs/SM)."""
    nx0, ny0 = 52, 44
    refs = I.box_refs(nx0, ny0, 3, [(0, 8, 8, 24, 16), (0, 0, 32, 8, 8), (0, 48, 32, 4, 8)])
    refs[1][24:40, 24:56] = 1
    cs = I.smooth_random(nx0, ny0, 3, refs, seed=21, amp=0.25, beta=0.8, steps=25)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=variant, graph_steps=graph_steps, schedule=schedule, persist_after=7)
    o = oracle_of(cs)
    t0, a0 = g.audit()
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 3)
    t1, _ = g.audit()
    assert drift(t0, t1, a0) < 1e-13


@pytest.mark.parametrize("schedule", [1, 0])
def test_riemann3_three_levels_outflow(V, schedule):
    cs = I.riemann3(N=64, nlev=3, steps=60)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(schedule=schedule)
    o = oracle_of(cs)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 3)


@pytest.mark.parametrize("sensor", [False, True])
def test_riemann3_transpose_symmetric(V, sensor):
    cs = I.riemann3(N=64, nlev=3, steps=40, beta=1.0 if sensor else 0.7)
    g = V.Hierarchy.from_case(cs)
    if sensor:
        g.set_sensor(True, beta_min=0.5, c_sensor=64.0)
    g.advance(cs.steps)
    for l in range(3):
        f = g.get_populations(l).reshape(4, 4, *g.shapes[l])
        gin, gref = g.layout(l)
        act = (gin == 1) & (gref == 0)
        ft = f.transpose(0, 1, 3, 2)[[2, 3, 0, 1]][:, [0, 2, 1, 3]]
        assert np.array_equal(f[:, :, act], ft[:, :, act])


def test_reflective_walls_with_patch(V):
    """Explosion in a box (Sec. 4.2, Eq. 31) on a small grid: reflective walls
    on all sides, a centred ratio-2 patch."""
    cs = I.explosion(N=64, steps=50)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    t0, a0 = g.audit()
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 2)
    t1, _ = g.audit()
    # walls: mass and energy conserved, momentum is not
    assert abs(t1[0] - t0[0]) / a0[0] < 1e-13 and abs(t1[3] - t0[3]) / a0[3] < 1e-13


def test_inflow_outflow_static(V):
    """Inflow (west), outflow (east), periodic (south/north) with a static
    patch that the shock crosses."""
    cs = I.shockbubble(nx0=64, ny0=32, nlev=2, steps=40)
    cs.refs = I.box_refs(64, 32, 2, [(0, 8, 8, 24, 16)])
    # level-1 state: the same initial condition on the fine cell centres
    cs.W = [cs.W[0], I.shockbubble(nx0=128, ny0=64, nlev=1).W[0]]
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 2)


def test_regrid_to_masks(V):
    n = 48
    refs_a = I.box_refs(n, n, 3, [(0, 8, 8, 24, 24)])
    refs_a[1][24:56, 24:40] = 1
    refs_b = I.box_refs(n, n, 3, [(0, 16, 8, 24, 32)])
    refs_b[1][32:48, 40:64] = 1
    cs = I.smooth_random(n, n, 3, refs_a, seed=31, amp=0.3, beta=0.9)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    g.advance(6)
    o.advance(6)
    t0, a0 = g.audit()
    # the audit is exact: it equals math.fsum of the oracle's weighted W
    ot, oa = o.totals()
    assert np.array_equal(t0, ot) and np.array_equal(a0, oa)
    g.regrid_masks(refs_b)
    o.regrid(refs_b)
    t1, a1 = g.audit()
    assert drift(t0, t1, a0) < 1e-14
    ot, oa = o.totals()
    assert np.array_equal(t1, ot) and np.array_equal(a1, oa)
    compare(o, g, 3)
    g.advance(7)
    o.advance(7)
    compare(o, g, 3)
    g.regrid_masks(I.empty_refs(n, n, 3))
    o.regrid(I.empty_refs(n, n, 3))
    g.advance(2)
    o.advance(2)
    compare(o, g, 3)


def test_adaptive_shockbubble_small(V):
    """Adaptive shock-bubble on a 128 x 64 coarse grid, three levels, regrid
    every 4 coarse steps from the density-gradient indicator: layouts and
    populations match the oracle, totals are conserved across each regrid."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    tol, buf, every = cs.amr["tol"], cs.amr["buffer"], cs.amr["every"]
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    for _ in range(2):  # build the initial levels from the initial state
        g.regrid()
        o.regrid_tagged(tol, buf, 8)
    compare(o, g, 3)
    for cycle in range(6):
        g.advance(every)
        o.advance(every)
        t0, a0 = g.audit()
        g.regrid()
        o.regrid_tagged(tol, buf, 8)
        t1, _ = g.audit()
        assert drift(t0, t1, a0) < 1e-14
        compare(o, g, 3)
    info = g.info()
    assert info["active_cells"][1] > 0 and info["active_cells"][2] > 0


@pytest.mark.parametrize("schedule,graph_steps,variant,sensor", [(1, 4, 1, False), (1, 1, 3, False), (0, 4, 1, False),
                                                                 (1, 4, 2, True)])
def test_regrid_audit_rows_equal_separate_audits(V, schedule, graph_steps, variant, sensor):
    """The exact totals recorded before and after each device regrid equal
    separate audits of the same states, however the totals after a regrid
    are taken: from the first sweeps of the next persistent launch (their
    moments reduced by tasks of the same launch; also with the relaxation
    sensor's passes in the list), or by a separate audit (per-phase steps, a
    second regrid with no step between, or reading the rows before the next
    step)."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=variant, schedule=schedule, graph_steps=graph_steps, persist_after=0)
    for _ in range(2):
        g.regrid()
    if sensor:
        g.set_sensor(True, beta_min=0.5, c_sensor=16.0)
    g.set_regrid_audit(True)
    want = []
    for cycle in range(7):
        g.advance(4)
        b = g.audit()
        g.regrid()
        want.append((b, g.audit()))
        if cycle == 3:  # a second regrid straight after the first
            b = g.audit()
            g.regrid()
            want.append((b, g.audit()))
    g.advance(3)
    rows = g.regrid_audits()
    b = g.audit()
    g.regrid()
    want.append((b, g.audit()))
    rows = np.concatenate([rows, g.regrid_audits()])  # the last row's totals after: read before any step
    assert rows.shape == (len(want), 16)
    for r, ((t0, a0), (t1, a1)) in zip(rows, want):
        assert np.array_equal(r[0:4], t0) and np.array_equal(r[4:8], a0)
        assert np.array_equal(r[8:12], t1) and np.array_equal(r[12:16], a1)
        assert drift(t0, t1, a0) < 1e-14


def test_regrid_audit_row_settled_when_an_engine_admits_the_hierarchy(V):
    """A hierarchy admitted to an engine right after a device regrid gets
    that regrid's totals after from a separate audit at admission, equal to
    an audit of the same state."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    g = V.Hierarchy.from_case(cs)
    for _ in range(2):
        g.regrid()
    g.set_regrid_audit(True)
    g.advance(4)
    b = g.audit()
    g.regrid()
    a = g.audit()
    e = V.Engine()
    slot = e.admit(g, 4)
    done = []
    while not done:
        done, _ = e.advance(4)
    e.release(slot)
    e.close()
    rows = g.regrid_audits()
    assert rows.shape == (1, 16)
    assert np.array_equal(rows[0, 0:4], b[0]) and np.array_equal(rows[0, 4:8], b[1])
    assert np.array_equal(rows[0, 8:12], a[0]) and np.array_equal(rows[0, 12:16], a[1])


def test_adaptive_shockbubble_flux_jump_sensor(V):
    """The same adaptive run driven by the paper's flux-jump sensor (Sec. 3.4,
    Eq. amr-sigma, tol 0.01): tags, layouts and populations match the oracle
    through every regrid, totals are conserved across each regrid."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    cs.amr = dict(cs.amr, tol=0.01, sensor=1)
    tol, buf, every = cs.amr["tol"], cs.amr["buffer"], cs.amr["every"]
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    for _ in range(2):
        g.regrid()
        o.regrid_tagged(tol, buf, 8, sensor=1)
    compare(o, g, 3)
    for cycle in range(5):
        g.advance(every)
        o.advance(every)
        t0, a0 = g.audit()
        g.regrid()
        o.regrid_tagged(tol, buf, 8, sensor=1)
        t1, _ = g.audit()
        assert drift(t0, t1, a0) < 1e-14
        compare(o, g, 3)
    info = g.info()
    assert info["active_cells"][1] > 0 and info["active_cells"][2] > 0


@pytest.mark.parametrize("schedule", [1, 0])
def test_engine_results_equal_alone_and_in_mix(V, schedule):
    cases = [I.pulse2l(steps=30), I.riemann3(N=64, nlev=3, steps=25),
             I.smooth_random(40, 32, 1, [], seed=5, amp=0.2, steps=35)]
    alone = []
    for cs in cases:
        g = V.Hierarchy.from_case(cs)
        g.advance(cs.steps)
        alone.append([g.get_populations(l) for l in range(cs.nlev)])
        g.close()
    e = V.Engine(allocator="torch", schedule=schedule)  # the engine's tables from torch's caching allocator
    hs = [V.Hierarchy.from_case(cs) for cs in cases]
    slots = [e.admit(h, cs.steps) for h, cs in zip(hs, cases)]
    done = set()
    while len(done) < len(cases):
        for s in e.step():
            done.add(s)
    for cs, h, a in zip(cases, hs, alone):
        for l in range(cs.nlev):
            gin, gref = h.layout(l)
            act = (gin == 1) & (gref == 0)
            assert np.array_equal(h.get_populations(l)[:, act], a[l][:, act])
    for s in slots:
        e.release(s)
    e.close()


@pytest.mark.parametrize("max_steps,schedule", [(1, 1), (5, 1), (16, 1), (1, 0), (16, 0)])
def test_engine_static_and_adaptive_residents_equal_alone(V, max_steps, schedule):
    """Continuous batching with static residents and adaptive residents
    regridding every 4 of their own steps, admitted at different times, on
    one persistent launch per call (the residents' device-built task lists
    merged phase-major) or on shared per-phase launches: every result is
    bit-identical to the same request advanced alone, whatever the number of
    steps per engine call."""
    def adaptive_case(steps):
        return I.shockbubble(nx0=64, ny0=32, nlev=3, steps=steps)

    specs = [(I.pulse2l(steps=30), 0, 0), (adaptive_case(22), 4, 0), (I.riemann3(N=64, nlev=3, steps=25), 0, 3),
             (adaptive_case(13), 4, 7), (I.smooth_random(40, 32, 1, [], seed=5, amp=0.2, steps=9), 0, 11)]

    def start(cs, every):
        g = V.Hierarchy.from_case(cs)
        if every:
            for _ in range(cs.nlev - 1):
                g.regrid()
        return g

    alone = []
    for cs, every, _ in specs:
        g = start(cs, every)
        left = cs.steps
        while left > 0:
            n = min(left, every) if every else left
            g.advance(n)
            left -= n
            if every and left > 0:
                g.regrid()
        alone.append([g.get_populations(l) for l in range(cs.nlev)])
        g.close()
    e = V.Engine(schedule=schedule)
    hs, slots = [None] * len(specs), [None] * len(specs)
    done, t = set(), 0
    while len(done) < len(specs):
        for i, (cs, every, at) in enumerate(specs):
            if hs[i] is None and at <= t:
                hs[i] = start(cs, every)
                slots[i] = e.admit(hs[i], cs.steps, every)
        fin, k = e.advance(max_steps)
        assert 0 <= k <= max_steps
        t += max(k, 1)  # nothing resident: let the clock reach the next admission
        done.update(fin)
    for (cs, _, _), h, a in zip(specs, hs, alone):
        for l in range(cs.nlev):
            gin, gref = h.layout(l)
            act = (gin == 1) & (gref == 0)
            assert np.array_equal(h.get_populations(l)[:, act], a[l][:, act])
    for s in slots:
        e.release(s)
    e.close()


def test_nonphysical_state_is_reported(V):
    cs = I.smooth_random(16, 16, 1, [], seed=2)
    cs.W[0][0, 3, 4] = -1.0
    g = V.Hierarchy.from_case(cs)
    g.advance(1)
    with pytest.raises(V.VlbmError) as ei:
        g.sync()
    assert ei.value.name == "ERR_NONPHYSICAL"
    with pytest.raises(V.VlbmError) as ei:
        g.advance(1)
    assert ei.value.name == "ERR_STATE"


def test_nesting_violation_rejected(V):
    # a level-2 block touching level-0 territory
    with pytest.raises(V.VlbmError) as ei:
        V.Hierarchy(32, 32, 3, (0, 0, 0, 0), 1.4, 5.0, 0.9, boxes=[(0, 8, 8, 8, 8), (1, 16, 16, 8, 8)])
    assert ei.value.name == "ERR_NESTING"
    with pytest.raises(V.VlbmError) as ei:
        V.Hierarchy(32, 32, 2, (0, 0, 0, 0), 1.4, 5.0, 0.9, boxes=[(0, 4, 8, 8, 8)])
    assert ei.value.name == "ERR_ARG"


def test_torch_allocator_and_stream(V):
    import torch
    s = torch.cuda.Stream()
    cs = I.pulse2l(steps=20)
    g = V.Hierarchy.from_case(cs, stream=s, allocator="torch")
    o = oracle_of(cs)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 2)
    g.close()


def test_vortex_512_bench_configuration(V):
    """The benchmarked configuration itself (512^2 coarse + central ratio-2
    patch), in the bench's launch configuration, for a few coarse steps."""
    cs = I.vortex(N=512, steps=4)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 2)


@pytest.mark.parametrize("graph_steps", [8, 3])
def test_step_totals_are_exact_every_step(V, graph_steps):
    """The fused per-step audit returns, for every coarse step, the exactly
    rounded totals of the state at the start of the step: they equal
    math.fsum of the oracle's W (area-weighted) at the same times."""
    n = 40
    refs = I.box_refs(n, n, 3, [(0, 8, 8, 24, 16)])
    refs[1][24:40, 24:56] = 1
    cs = I.smooth_random(n, n, 3, refs, seed=51, amp=0.25, beta=0.85, steps=13)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=1, graph_steps=graph_steps, schedule=1)
    g.set_step_totals(True)
    o = oracle_of(cs)
    g.advance(cs.steps)
    rows = g.step_totals()
    assert rows.shape == (cs.steps, 8)
    for st in range(cs.steps):
        ot, oa = o.totals()
        assert np.array_equal(rows[st, :4], ot), (st, rows[st, :4] - ot)
        assert np.array_equal(rows[st, 4:], oa), (st, rows[st, 4:] - oa)
        o.advance(1)
    # the recorded totals stay constant to round-off (periodic domain)
    d = np.abs(rows[:, :4] - rows[0, :4]) / rows[0, 4:]
    assert d.max() < 1e-14
    assert len(g.step_totals()) == 0


def test_laxliu12_three_levels(V):
    """Lax-Liu configuration 12 (Sec. 4.3.2) with three levels."""
    cs = I.laxliu12(N=64, nlev=3, steps=50)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 3)


def test_checkpoint_resume_is_bitwise(V):
    """A run checkpointed mid-way and resumed in a fresh hierarchy continues
    exactly as the uninterrupted run (including the faces' previous samples
    and an adaptive regrid)."""
    cs = I.shockbubble(nx0=128, ny0=64, nlev=3)
    a = V.Hierarchy.from_case(cs)
    for _ in range(2):
        a.regrid()
    a.advance(6)
    a.regrid()
    a.advance(3)
    blob = a.checkpoint()
    a.advance(5)
    a.regrid()
    a.advance(4)
    b = V.Hierarchy(cs.nx0, cs.ny0, cs.nlev, cs.bc, cs.gamma, cs.c, cs.beta, dx0=cs.dx0, inflow=cs.inflow,
                    tag_tol=cs.amr["tol"], tag_buffer=cs.amr["buffer"])
    b.restore(blob)
    b.advance(5)
    b.regrid()
    b.advance(4)
    assert a.info()["steps"] == b.info()["steps"]
    for l in range(cs.nlev):
        assert np.array_equal(a.layout(l)[0], b.layout(l)[0])
        assert np.array_equal(a.layout(l)[1], b.layout(l)[1])
        ia, ra = a.layout(l)
        act = (ia == 1) & (ra == 0)
        assert np.array_equal(a.get_populations(l)[:, act], b.get_populations(l)[:, act])


def test_exact_totals_on_wide_value_ranges(V):
    """The exact audits (fused per-step totals and vlbm_audit) on two-level
    states whose momenta take zeros, subnormals and values of both signs
    over many decades, and whose densities and energies span six and four
    decades: both equal math.fsum of the area-weighted moments, which the
    test computes from the populations themselves (the same additions as
    the sweep).  Momenta stay small against the pressure so that the one
    step taken stays physical across the interface."""
    n = 40
    refs = I.box_refs(n, n, 2, [(0, 8, 16, 24, 16)])
    cs = I.smooth_random(n, n, 2, refs, seed=5, steps=1, beta=0.5)
    rng = np.random.default_rng(2024)

    def momentum(shape, rho):
        kind = rng.integers(0, 4, size=shape)
        sign = np.where(rng.random(shape) < 0.5, -1.0, 1.0)
        m = sign * rho * 10.0 ** rng.uniform(-8, -3, size=shape)
        m = np.where(kind == 0, 0.0, m)
        m = np.where(kind == 1, sign * 10.0 ** rng.uniform(-320, -250, size=shape), m)
        return m

    for l in range(cs.nlev):
        shape = cs.W[l].shape[1:]
        rho = 10.0 ** rng.uniform(-3, 3, size=shape)
        mu, mv = momentum(shape, rho), momentum(shape, rho)
        p = 10.0 ** rng.uniform(-2, 2, size=shape)
        cs.W[l] = np.stack([rho, mu, mv, 0.5 * (mu * mu + mv * mv) / rho + p / (cs.gamma - 1.0)])
    cs.c *= 100.0  # one quiet step: every intermediate state stays physical
    g = V.Hierarchy.from_case(cs)
    tot = [[] for _ in range(4)]
    for l in range(cs.nlev):
        f = g.get_populations(l)
        a, b = g.layout(l)
        act = (a == 1) & (b == 0)
        for k in range(4):
            w = (f[k] + f[4 + k]) + (f[8 + k] + f[12 + k])
            tot[k].append(w[act] * 0.25 ** l)
    exp_t = np.array([math.fsum(np.concatenate(t)) for t in tot])
    exp_a = np.array([math.fsum(np.abs(np.concatenate(t))) for t in tot])
    t0, a0 = g.audit()
    assert np.array_equal(t0, exp_t), t0 - exp_t
    assert np.array_equal(a0, exp_a), a0 - exp_a
    g.set_step_totals(True)
    g.advance(1)
    rows = g.step_totals()
    assert np.array_equal(rows[0, :4], exp_t) and np.array_equal(rows[0, 4:], exp_a)


def test_bounded_wait_gives_up_and_context_survives(V):
    """Failure detection of the persistent schedule: a task waiting on a
    completion mark that nothing sets gives up after its poll limit, the
    kernel reports VLBM_ERR_TIMEOUT through its status word, and the CUDA
    context stays usable (a run afterwards still matches the oracle)."""
    st, ms, word = V.selftest_timeout()
    assert st == 6, (st, ms, word)  # VLBM_ERR_TIMEOUT
    assert word & 2
    assert 20.0 < ms < 30000.0, ms  # waited, then returned
    cs = I.pulse2l(steps=6)
    g = V.Hierarchy.from_case(cs)
    o = oracle_of(cs)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, cs.nlev)


@pytest.mark.parametrize("which,schedule,variant", [("smooth3", 1, 1), ("smooth3", 1, 2), ("smooth3", 1, 3),
                                                    ("smooth3", 0, 1), ("laxliu3", 1, 2), ("laxliu3", 0, 1),
                                                    ("laxliu3_128", 1, 2)])
def test_sensor_driven_relaxation_matches_oracle(V, which, schedule, variant):
    """The sensor-driven relaxation (Sec. 2.2, Eq. sensor-B; per-cell beta
    from the flux-jump rate and the Ducros gate, two sensor passes before
    every level sweep: separate launches, or tasks of the persistent launch)
    reproduces the oracle bit for bit: a three-level ragged periodic field
    with the sensor acting, and Lax-Liu 3 on three levels with outflow
    boundaries (where the sensor keeps the run physical)."""
    if which == "smooth3":
        nx0, ny0 = 44, 36
        refs = I.box_refs(nx0, ny0, 3, [(0, 8, 8, 16, 16)])
        refs[1][24:40, 24:40] = 1
        cs = I.smooth_random(nx0, ny0, 3, refs, seed=67, amp=0.35, beta=1.0, steps=9)
        kw = dict(beta_min=0.5, c_sensor=20.0)
    elif which == "laxliu3":
        cs = I.riemann3(N=64, nlev=3, steps=40, beta=1.0)
        kw = dict(beta_min=0.5, c_sensor=16.0)
    else:  # to t = 0.3 on 128^2 with three levels (a gain of 16 lets a fine
        # level lose positivity for a few steps there; 64 does not)
        cs = I.riemann3(N=128, nlev=3, beta=1.0)
        kw = dict(beta_min=0.5, c_sensor=64.0)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=variant, schedule=schedule, graph_steps=4)
    o = oracle_of(cs)
    g.set_sensor(True, **kw)
    o.set_sensor(True, **kw)
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, cs.nlev)
    # and the engine advances such a hierarchy to the same result
    g2 = V.Hierarchy.from_case(cs)
    g2.set_sensor(True, **kw)
    e = V.Engine()
    slot = e.admit(g2, cs.steps)
    done = []
    while not done:
        done, _ = e.advance(7)
    for l in range(cs.nlev):
        gin, gref = g.layout(l)
        act = (gin == 1) & (gref == 0)
        assert np.array_equal(g2.get_populations(l)[:, act], g.get_populations(l)[:, act])
    e.release(slot)
    e.close()


def test_get_conserved_into_caller_buffer(V):
    """Reading W into a caller-owned (pinned) buffer gives the same values as
    the default read."""
    import torch
    cs = I.pulse2l(steps=6)
    g = V.Hierarchy.from_case(cs)
    g.advance(cs.steps)
    for l in range(cs.nlev):
        W, _ = g.get_conserved(l)
        buf = torch.empty(W.shape, dtype=torch.float64).pin_memory().numpy()
        W2, v2 = g.get_conserved(l, out=buf, valid=False)
        assert v2 is None and W2 is buf
        assert np.array_equal(W, W2)
    g.close()


@pytest.mark.parametrize("schedule,graph_steps", [(0, 8), (1, 3)])
def test_four_levels_maximum_depth(V, schedule, graph_steps):
    """The deepest hierarchy the library takes: four levels, each nested in
    the previous one with a one-block margin (eight level-3 sub-steps per
    coarse step), per-phase and persistent schedules: bitwise equal to the
    oracle, totals conserved."""
    n = 40
    refs = I.box_refs(n, n, 4, [(0, 8, 8, 24, 24)])
    refs[1][24:56, 24:56] = 1
    refs[2][56:104, 56:104] = 1
    cs = I.smooth_random(n, n, 4, refs, seed=71, amp=0.2, beta=0.9, steps=6)
    g = V.Hierarchy.from_case(cs)
    g.set_tuning(variant=1, graph_steps=graph_steps, schedule=schedule)
    o = oracle_of(cs)
    t0, a0 = g.audit()
    g.advance(cs.steps)
    o.advance(cs.steps)
    compare(o, g, 4)
    t1, _ = g.audit()
    assert drift(t0, t1, a0) < 1e-13
    g.close()


def test_degenerate_calls(V):
    """advance(0) changes nothing; an engine with nothing resident queues no
    steps and reports nothing; a resident admitted for zero steps is
    reported finished, unchanged."""
    cs = I.pulse2l(steps=3)
    g = V.Hierarchy.from_case(cs)
    before = [g.get_populations(l) for l in range(cs.nlev)]
    g.advance(0)
    for l in range(cs.nlev):
        assert np.array_equal(g.get_populations(l), before[l])
    e = V.Engine()
    fin, k = e.advance(4)
    assert list(fin) == [] and k == 0
    slot = e.admit(g, 0)
    done = []
    for _ in range(3):
        fin, k = e.advance(4)
        done += list(fin)
        if done:
            break
    assert done == [slot]
    e.release(slot)
    for l in range(cs.nlev):
        assert np.array_equal(g.get_populations(l), before[l])
    e.close()
    g.close()
