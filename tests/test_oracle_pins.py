"""Pins of the oracle to things other than itself.

Closed forms (equilibrium moments, the Euler flux from primitive variables),
invariants (per-cell conservation of the collision, exact conservation
across interfaces and regrids, preservation of a uniform state, the ratio-1
limit, transpose and translation symmetry), textbook solutions (Sod exact
Riemann solution) and the numbers the paper prints (mass drift, convergence
order).  Each test is chosen so that a plausible slip in the oracle (a dropped
term, a sign, an index, a transposed operand) fails one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_35529_b300 import inputs as I

import exact_riemann as ER

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    vals = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def rand_state(rng, n=1):
    rho = rng.uniform(0.2, 3.0, n)
    u = rng.uniform(-1.5, 1.5, n)
    v = rng.uniform(-1.5, 1.5, n)
    p = rng.uniform(0.1, 3.0, n)
    return rho, u, v, p


def flux_from_primitives(rho, u, v, p, gamma=1.4):
    """Euler flux written from primitive variables (Sec. 2.1)."""
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    Qx = np.array([rho * u, rho * u * u + p, rho * u * v, (E + p) * u])
    Qy = np.array([rho * v, rho * u * v, rho * v * v + p, (E + p) * v])
    return Qx, Qy


# ----------------------------------------------------------------------
# single-cell operators
# ----------------------------------------------------------------------

def test_equilibrium_moments_match_flux():
    """Eq. 3-4: sum_i f_i^eq = W and sum_i c_i f_i^eq = Q(W)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        rho, u, v, p = (a[0] for a in rand_state(rng))
        c = rng.uniform(4.0, 12.0)
        W = I.conserved(np.array(rho), u, v, p)
        fe = O.feq(1.4, c, W).reshape(4, 4)  # [dir][field]
        Qx, Qy = flux_from_primitives(rho, u, v, p)
        np.testing.assert_allclose(fe.sum(axis=0), W, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(c * (fe[0] - fe[1]), Qx, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(c * (fe[2] - fe[3]), Qy, rtol=1e-13, atol=1e-13)


def test_collision_conserves_every_field_for_any_beta():
    """Eq. 6: the zeroth moment is invariant under relaxation, cell by cell."""
    rng = np.random.default_rng(2)
    for _ in range(300):
        rho, u, v, p = (a[0] for a in rand_state(rng))
        c = rng.uniform(4.0, 12.0)
        W = I.conserved(np.array(rho), u, v, p)
        f = O.feq(1.4, c, W) * (1 + 0.3 * rng.normal(size=16))
        beta = rng.uniform(0.01, 1.0)
        fs = O.collide(1.4, c, beta, f)
        W0 = f.reshape(4, 4).sum(axis=0)
        W1 = fs.reshape(4, 4).sum(axis=0)
        scale = np.abs(f.reshape(4, 4)).sum(axis=0) + np.abs(fs.reshape(4, 4)).sum(axis=0)
        assert np.all(np.abs(W1 - W0) <= 8e-16 * scale)


def test_collision_first_moment_relaxes_towards_flux():
    """Eq. 6 on the first moment: sum_i c_i f*_i = 2 beta Q + (1-2beta) sum_i c_i f_i."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        rho, u, v, p = (a[0] for a in rand_state(rng))
        c = rng.uniform(4.0, 12.0)
        W = I.conserved(np.array(rho), u, v, p)
        f = O.feq(1.4, c, W) + 0.05 * rng.normal(size=16)
        Wf = f.reshape(4, 4).sum(axis=0)
        Qx, Qy = flux_from_primitives(Wf[0], Wf[1] / Wf[0], Wf[2] / Wf[0],
                                      0.4 * (Wf[3] - 0.5 * (Wf[1] ** 2 + Wf[2] ** 2) / Wf[0]))
        beta = rng.uniform(0.1, 1.0)
        fs = O.collide(1.4, c, beta, f).reshape(4, 4)
        fr = f.reshape(4, 4)
        jx = c * (fs[0] - fs[1])
        want = 2 * beta * Qx + (1 - 2 * beta) * c * (fr[0] - fr[1])
        np.testing.assert_allclose(jx, want, rtol=1e-12, atol=1e-12)
        jy = c * (fs[2] - fs[3])
        want = 2 * beta * Qy + (1 - 2 * beta) * c * (fr[2] - fr[3])
        np.testing.assert_allclose(jy, want, rtol=1e-12, atol=1e-12)


def test_beta_half_lands_on_equilibrium():
    rng = np.random.default_rng(4)
    W = I.conserved(np.array(1.3), 0.4, -0.2, 0.9)
    f = O.feq(1.4, 6.0, W) + 0.01 * rng.normal(size=16)
    Wf = f.reshape(4, 4).sum(axis=0)
    np.testing.assert_allclose(O.collide(1.4, 6.0, 0.5, f), O.feq(1.4, 6.0, Wf), rtol=1e-14, atol=1e-15)


def test_beta_zero_is_identity():
    rng = np.random.default_rng(5)
    f = rng.uniform(0.1, 1.0, 16)
    assert np.array_equal(O.collide(1.4, 6.0, 0.0, f), f)


def test_minmod_truth_table():
    assert O.minmod(1.0, 2.0) == 1.0
    assert O.minmod(3.0, 2.0) == 2.0
    assert O.minmod(-1.0, -2.0) == -1.0
    assert O.minmod(-3.0, -2.0) == -2.0
    assert O.minmod(1.0, -2.0) == 0.0
    assert O.minmod(-1.0, 2.0) == 0.0
    assert O.minmod(0.0, 2.0) == 0.0
    assert O.minmod(2.0, 0.0) == 0.0
    assert O.minmod(1e-300, 1e-300) == 1e-300  # no underflow of a*b


def test_recon_weights_r2_closed_form():
    """Eq. 23 at r = 2: weights (2k-3)/4 in time and (2j-1)/4 across the edge."""
    a, ap, s = 0.7, 0.5, 0.08
    d = a - ap
    assert O.recon(a, ap, s, 2, 1, 0) == pytest.approx(a - d / 4 - s / 4, abs=1e-16)
    assert O.recon(a, ap, s, 2, 1, 1) == pytest.approx(a - d / 4 + s / 4, abs=1e-16)
    assert O.recon(a, ap, s, 2, 2, 0) == pytest.approx(a + d / 4 - s / 4, abs=1e-16)
    assert O.recon(a, ap, s, 2, 2, 1) == pytest.approx(a + d / 4 + s / 4, abs=1e-16)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_recon_is_mean_preserving(r):
    """Eqs. 19 and 23: the r*r reconstructed values average to the coarse sample,
    and the time average along each row is the purely temporal value plus the
    tangential offset (the time term telescopes)."""
    rng = np.random.default_rng(6 + r)
    for _ in range(50):
        a, ap, s = rng.normal(size=3)
        vals = np.array([[O.recon(a, ap, s, r, k, j) for j in range(r)] for k in range(1, r + 1)])
        assert vals.mean() == pytest.approx(a, abs=1e-14)
        for j in range(r):
            assert vals[:, j].mean() == pytest.approx(a + s * (2 * j - r + 1) / (2 * r), abs=1e-14)


def test_merge_of_split_returns_parent():
    """Eqs. 25-27: the offsets sum to zero, so merge(split(f)) = f for any slope,
    and a flat split is a bitwise copy."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        fc, sx, sy = rng.normal(size=3)
        ch = [O.split_child(fc, sx, sy, 2, a, b) for b in range(2) for a in range(2)]
        m = O.merge4(ch[0], ch[1], ch[2], ch[3])
        assert abs(m - fc) <= 4 * np.spacing(abs(fc) + abs(sx) + abs(sy))
        assert O.split_child(fc, 0.0, 0.0, 2, 1, 0) == fc


# ----------------------------------------------------------------------
# whole-scheme invariants
# ----------------------------------------------------------------------

def make(cs, r=2, refs="case"):
    h = O.Hierarchy(cs.nx0, cs.ny0, cs.nlev, r, cs.bc, cs.gamma, cs.c, cs.beta, cs.inflow)
    h.set_layout(cs.refs if refs == "case" else refs)
    for l in range(cs.nlev):
        h.set_state(l, cs.W[l])
    return h


def three_level_refs(n=32):
    refs = I.box_refs(n, n, 3, [(0, 8, 8, 16, 16)])
    refs[1][24:40, 24:40] = 1
    return refs


def test_pure_streaming_returns_after_one_period():
    """beta = 0: collision is the identity and shift streaming (Eq. 5) returns
    every population to its start after nx steps on a periodic grid."""
    cs = I.smooth_random(24, 16, 1, [], seed=3, beta=0.0)
    h = make(cs, refs=None)
    rng = np.random.default_rng(8)
    f0 = rng.uniform(0.1, 1.0, (16, 16, 24))
    h.set_f(0, f0)
    h.advance(48)  # lcm(24, 16)
    assert np.array_equal(h.get_f(0), f0)
    h.advance(1)
    f1 = h.get_f(0).reshape(4, 4, 16, 24)
    f0r = f0.reshape(4, 4, 16, 24)
    assert np.array_equal(f1[0], np.roll(f0r[0], 1, axis=2))   # +x moves right
    assert np.array_equal(f1[1], np.roll(f0r[1], -1, axis=2))  # -x moves left
    assert np.array_equal(f1[2], np.roll(f0r[2], 1, axis=1))   # +y moves up
    assert np.array_equal(f1[3], np.roll(f0r[3], -1, axis=1))  # -y moves down


@pytest.mark.parametrize("nlev", [2, 3])
def test_uniform_state_is_preserved_through_interfaces(nlev):
    n = 32
    refs = three_level_refs(n)[: nlev - 1]
    Ws = [I.conserved(np.full((n * 2 ** l, n * 2 ** l), 1.2), 0.3, -0.1, 0.8) for l in range(nlev)]
    c = I.link_speed([Ws[0]])
    cs = I.Case("u", n, n, nlev, (0, 0, 0, 0), 1.4, c, 0.9, Ws, refs, 0)
    h = make(cs)
    h.advance(37)
    # The collision map has no exact floating-point fixed point (over-relaxation
    # settles into a two-cycle one ulp wide), and the fine level takes r steps
    # per coarse step, so "preserved" means to a few ulps, everywhere, without drift.
    f0 = h.get_f(0)[:, 0, 0]
    for l in range(nlev):
        f = h.get_f(l)
        act = h.active_masks()[l]
        vals = f[:, act]
        assert np.max(np.abs(vals - f0[:, None])) <= 2e-15, l
        W, fl = h.get_W(l)
        np.testing.assert_allclose(W[:, act], np.repeat(Ws[0][:, :1, 0], act.sum(), axis=1), rtol=0, atol=4e-15)


def test_ratio_one_hierarchy_equals_uniform_grid():
    """At r = 1 the reconstruction and reflux weights reduce to the identity
    (Eqs. 20, 24), so a ratio-1 'patch' reproduces the uniform grid bitwise."""
    n = 32
    refs = [np.zeros((n, n), np.uint8)]
    refs[0][8:20, 12:28] = 1
    cs = I.smooth_random(n, n, 1, [], seed=11, amp=0.1, beta=0.8)
    u = make(cs, refs=None)
    h = O.Hierarchy(n, n, 2, 1, cs.bc, cs.gamma, cs.c, cs.beta)
    h.set_layout(refs)
    h.set_state(0, cs.W[0])
    h.set_state(1, cs.W[0])
    u.advance(25)
    h.advance(25)
    fu = u.get_f(0)
    f0, f1 = h.get_f(0), h.get_f(1)
    act0 = h.active_masks()[0]
    act1 = h.active_masks()[1]
    assert np.array_equal(f0[:, act0], fu[:, act0])
    assert np.array_equal(f1[:, act1], fu[:, act1])


@pytest.mark.parametrize("which", ["pulse", "smooth3", "smooth2_offcentre"])
def test_exact_conservation_periodic(which):
    """Sec. 3.2-3.3: reconstruction and reflux together conserve mass,
    momentum and energy exactly (round-off) on a periodic domain."""
    if which == "pulse":
        cs = I.pulse2l(steps=100)
    elif which == "smooth3":
        cs = I.smooth_random(32, 32, 3, three_level_refs(32), seed=4, amp=0.2, beta=0.9, steps=30)
    else:
        refs = I.box_refs(40, 24, 2, [(0, 0, 8, 16, 8), (0, 32, 16, 8, 8)])  # wraps across the seam
        cs = I.smooth_random(40, 24, 2, refs, seed=5, amp=0.2, beta=0.7, steps=60)
    h = make(cs)
    t0, a0 = h.totals()
    h.advance(cs.steps)
    t1, _ = h.totals()
    drift = np.abs(t1 - t0) / a0
    assert np.all(drift < 1e-14), drift


@pytest.mark.parametrize("sensor", [False, True])
def test_transpose_symmetry_is_bitwise(sensor):
    """Lax-Liu configuration 3 is symmetric under x <-> y (with u <-> v); the
    canonical arithmetic is written symmetrically, so the three-level run
    stays exactly symmetric -- also with the sensor-driven relaxation, whose
    sums over fields and over the 3 x 3 neighbourhood are grouped in pairs
    that swap into each other."""
    cs = I.riemann3(N=64, nlev=3, steps=40, beta=1.0 if sensor else 0.7)
    h = make(cs)
    if sensor:
        h.set_sensor(True, beta_min=0.5, c_sensor=64.0)
        b = h.sensor_beta(0)
        assert b[b > 0].min() < 1.0  # the sensor acts
    h.advance(cs.steps)
    for l in range(cs.nlev):
        f = h.get_f(l).reshape(4, 4, *h.shapes[l])
        act = h.active_masks()[l]
        assert np.array_equal(act, act.T)
        ft = f.transpose(0, 1, 3, 2)[[2, 3, 0, 1]][:, [0, 2, 1, 3]]
        assert np.array_equal(f[:, :, act], ft[:, :, act]), f"level {l}"


def test_translation_invariance_periodic():
    """Shifting the initial state and the layout by one block shifts the
    result by the same amount, bitwise."""
    n = 32
    refs = three_level_refs(n)
    cs = I.smooth_random(n, n, 3, refs, seed=9, amp=0.2, beta=0.85, steps=12)
    a = make(cs)
    a.advance(cs.steps)
    sh = 8
    refs2 = [np.roll(refs[0], sh, axis=1), np.roll(refs[1], 2 * sh, axis=1)]
    W2 = [np.roll(cs.W[l], sh * 2 ** l, axis=2) for l in range(3)]
    b = O.Hierarchy(n, n, 3, 2, cs.bc, cs.gamma, cs.c, cs.beta)
    b.set_layout(refs2)
    for l in range(3):
        b.set_state(l, W2[l])
    b.advance(cs.steps)
    for l in range(3):
        act = a.active_masks()[l]
        fa = a.get_f(l)
        fb = np.roll(b.get_f(l), -sh * 2 ** l, axis=2)
        assert np.array_equal(fa[:, act], fb[:, act])


# ----------------------------------------------------------------------
# adaptive refinement (Sec. 3.4)
# ----------------------------------------------------------------------

def test_layout_rule_single_tag_two_levels():
    """One tagged cell, buffer 1, blocks of 4: the refined set is exactly the
    blocks touched by the 3x3 neighbourhood of the tag."""
    n = 32
    h = O.Hierarchy(n, n, 2, 2, (0, 0, 0, 0), 1.4, 5.0, 0.9)
    h.set_layout(None)
    tags = [np.zeros((n, n), np.uint8)]
    tags[0][7, 12] = 1  # (y=7, x=12): neighbourhood x 11..13, y 6..8
    ref = h.layout_from_tags(tags, 1, 4)[0]
    want = np.zeros((n, n), np.uint8)
    want[4:12, 8:16] = 1
    assert np.array_equal(ref, want)


def test_layout_rule_three_levels_nests():
    """A level-1 tag forces the coarse level to refine the parents of its
    refined block and their neighbours (proper nesting)."""
    n = 32
    h = O.Hierarchy(n, n, 3, 2, (1, 1, 1, 1), 1.4, 5.0, 0.9)
    refs = I.box_refs(n, n, 3, [(0, 8, 8, 16, 16)])
    h.set_layout(refs)
    tags = [np.zeros((n, n), np.uint8), np.zeros((2 * n, 2 * n), np.uint8)]
    tags[1][20, 20] = 1
    r0, r1 = h.layout_from_tags(tags, 0, 4)
    want1 = np.zeros((2 * n, 2 * n), np.uint8)
    want1[20:24, 20:24] = 1
    assert np.array_equal(r1, want1)
    # parents of the 8-neighbourhood of [20,24)^2 are coarse cells 9..12 -> blocks [8,16)
    want0 = np.zeros((n, n), np.uint8)
    want0[8:16, 8:16] = 1
    assert np.array_equal(r0, want0)


def test_regrid_conserves_and_round_trips():
    """Merge (Eq. 25) and split (Eqs. 26-27) leave the totals unchanged, and
    refining then un-refining a region restores the coarse populations to
    round-off."""
    n = 32
    cs = I.smooth_random(n, n, 3, I.empty_refs(n, n, 3), seed=12, amp=0.3, beta=0.9, steps=5)
    h = make(cs)
    f0 = h.get_f(0)
    t0, a0 = h.totals()
    h.regrid(three_level_refs(n))
    t1, _ = h.totals()
    assert np.all(np.abs(t1 - t0) / a0 < 1e-15)
    h.regrid(I.empty_refs(n, n, 3))
    t2, _ = h.totals()
    assert np.all(np.abs(t2 - t0) / a0 < 1e-15)
    f2 = h.get_f(0)
    assert np.max(np.abs(f2 - f0)) <= 8 * np.spacing(np.max(np.abs(f0)))


def test_regrid_of_flat_field_is_exact():
    n = 32
    Ws = [I.conserved(np.full((n * 2 ** l, n * 2 ** l), 0.9), 0.2, 0.1, 1.1) for l in range(3)]
    cs = I.Case("u", n, n, 3, (0, 0, 0, 0), 1.4, 5.0, 0.9, Ws, I.empty_refs(n, n, 3), 0)
    h = make(cs)
    v = h.get_f(0)[:, 0, 0]
    h.regrid(three_level_refs(n))
    for l in range(3):
        act = h.active_masks()[l]
        assert np.all(h.get_f(l)[:, act] == v[:, None])


def test_adaptive_run_conserves_across_regrids():
    """A periodic adaptive run: tag, dilate, tile, merge/split every 3 steps;
    totals stay at round-off across every regrid and every step."""
    n = 48
    cs = I.smooth_random(n, n, 3, I.empty_refs(n, n, 3), seed=13, amp=0.3, beta=0.9, modes=4)
    h = make(cs)
    t0, a0 = h.totals()
    nref = []
    for it in range(6):
        refs = h.regrid_tagged(0.01, 1, 8)
        nref.append(sum(int(r.sum()) for r in refs))
        t, _ = h.totals()
        assert np.all(np.abs(t - t0) / a0 < 1e-14)
        h.advance(3)
    t, _ = h.totals()
    assert np.all(np.abs(t - t0) / a0 < 1e-14)
    assert max(nref) > 0


def flux_sensor_hierarchy(rho, u, v, p, periodic=True):
    """Two-level oracle hierarchy (no refinement yet) holding the given
    level-0 primitive fields."""
    ny, nx = rho.shape
    bc = (0, 0, 0, 0) if periodic else (1, 1, 1, 1)
    h = O.Hierarchy(nx, ny, 2, 2, bc, 1.4, 10.0, 0.9, None)
    h.set_layout(I.empty_refs(nx, ny, 2))
    h.set_state(0, I.conserved(rho, u, v, p))
    h.set_state(1, np.zeros((4, 2 * ny, 2 * nx)))
    return h


def test_flux_jump_sensor_tags_a_pressure_step_by_its_closed_form():
    """Flux-jump sensor (Sec. 3.4): at rest, a pressure step from 1 to 2 makes
    Q_x of the momentum field jump by 1 with max |Q| = 2, so the two columns
    beside the step (and beside the periodic wrap) have s = 1 / (2 * 2) =
    0.25: tagged for tol 0.24, untagged for tol 0.26; nothing else is."""
    ny, nx = 16, 24
    z = np.zeros((ny, nx))
    p = np.ones((ny, nx))
    p[:, 10:] = 2.0
    h = flux_sensor_hierarchy(z + 1.0, z, z, p)
    qmax = h.flux_max()
    # at rest only the pressure terms survive: Q_x of rho u and Q_y of rho v
    assert qmax[0] == 0.0 and qmax[3] == 0.0
    assert abs(qmax[1] - 2.0) < 1e-14 and abs(qmax[2] - 2.0) < 1e-14
    t = h.tags(0.24, sensor=1)[0]
    want = np.zeros((ny, nx), dtype=np.uint8)
    want[:, [9, 10, nx - 1, 0]] = 1
    assert np.array_equal(t, want)
    assert not h.tags(0.26, sensor=1)[0].any()


def test_flux_jump_sensor_ignores_contacts_and_shear():
    """A density jump at rest and uniform pressure (a contact) and a shear
    layer u(y) carry no jump of div Q, so the flux-jump sensor tags neither,
    while the density-gradient indicator does tag the contact."""
    ny, nx = 16, 16
    z = np.zeros((ny, nx))
    rho = np.ones((ny, nx))
    rho[:, 8:] = 3.0
    h = flux_sensor_hierarchy(rho, z, z, z + 1.0)
    assert not h.tags(1e-6, sensor=1)[0].any()
    assert h.tags(0.02, sensor=0)[0].any()
    u = np.where(np.arange(ny)[:, None] < 8, 0.5, -0.5) * np.ones((ny, nx))
    h = flux_sensor_hierarchy(z + 1.0, u, z, z + 1.0)
    assert not h.tags(1e-6, sensor=1)[0].any()


def test_flux_jump_sensor_uses_the_max_norm_over_fields():
    """A jump in one conserved field's flux is not diluted by the others: with
    v jumping from 0 to 0.1 across a horizontal line, the mass flux rho v
    jumps by its own maximum, so the rows beside the line have s_0 = 0.5
    and tag at just below that tolerance, whatever the other fields do."""
    ny, nx = 16, 16
    z = np.zeros((ny, nx))
    v = np.where(np.arange(ny)[:, None] < 8, 0.0, 0.1) * np.ones((ny, nx))
    h = flux_sensor_hierarchy(z + 1.0, z, v, z + 1.0, periodic=False)
    qmax = h.flux_max()
    # rho field: Q_y = rho v jumps 0 -> 0.1 between rows 7 and 8; qmax_0 = 0.1,
    # so s_0 = 0.1 / (2 * 0.1) = 0.5 there, whatever the other fields do
    assert abs(qmax[0] - 0.1) < 1e-15
    t = h.tags(0.49, sensor=1)[0]
    assert t[7].all() and t[8].all()
    assert not h.tags(0.51, sensor=1)[0][[7, 8]].any()


# ----------------------------------------------------------------------
# sensor-driven relaxation (Sec. 2.2, Eq. sensor-B)
# ----------------------------------------------------------------------

def sensor_level0(rho, u, v, p, beta=1.0, periodic=True, **kw):
    ny, nx = rho.shape
    bc = (0, 0, 0, 0) if periodic else (1, 1, 1, 1)
    h = O.Hierarchy(nx, ny, 1, 2, bc, 1.4, 10.0, beta, None)
    h.set_layout([])
    h.set_state(0, I.conserved(rho, u, v, p))
    h.set_sensor(True, **kw)
    return h


def test_sensor_with_zero_gain_is_the_constant_beta_scheme_bitwise():
    """C_sensor = 0 clips to 0, so beta = beta_max on every cell and the run
    is the constant-beta run bit for bit (three levels, ragged, periodic)."""
    nx0, ny0 = 44, 36
    refs = I.box_refs(nx0, ny0, 3, [(0, 8, 8, 16, 16)])
    refs[1][24:40, 24:40] = 1
    cs = I.smooth_random(nx0, ny0, 3, refs, seed=61, amp=0.25, beta=0.85, steps=7)
    a, b = make(cs), make(cs)
    b.set_sensor(True, beta_min=0.5, c_sensor=0.0)
    a.advance(cs.steps)
    b.advance(cs.steps)
    for l in range(3):
        assert np.array_equal(a.get_f(l), b.get_f(l))


def test_sensor_keeps_beta_max_in_uniform_flow_shear_and_expansion():
    """No compression, no sensor response: a uniform moving state, a shear
    layer u(y) (div u = 0, the Ducros gate closes) and a pure expansion
    (div u > 0) keep beta = beta_max on every cell, however large C."""
    ny, nx = 16, 24
    one = np.ones((ny, nx))
    h = sensor_level0(one, 0.3 * one, -0.2 * one, one, c_sensor=1e6)
    assert np.all(h.sensor_beta(0) == 1.0)
    yy = np.arange(ny)[:, None] * one
    h = sensor_level0(one, np.where(yy < 8, 0.5, -0.5), 0 * one, one, c_sensor=1e6)
    assert np.all(h.sensor_beta(0) == 1.0)
    xx = np.arange(nx)[None, :] * one
    h = sensor_level0(one, 0.01 * xx, 0 * one, one, periodic=False, c_sensor=1e6)
    assert np.all(h.sensor_beta(0) == 1.0)


def test_sensor_lowers_beta_only_at_a_compression():
    """A compression band (u falling from +0.5 to -0.5 over two cells, with
    the pressure jump of a shock) drives beta to beta_min there for a large
    gain, while cells more than two cells away (beyond the 3 x 3 filter of
    the 3-point differences) keep beta_max; beta stays in [beta_min, beta_max]."""
    ny, nx = 8, 32
    one = np.ones((ny, nx))
    xx = np.arange(nx)[None, :] * one
    u = np.clip((15.5 - xx) * 0.5, -0.5, 0.5)
    p = np.where(xx < 16, 2.0, 1.0)
    h = sensor_level0(one, u, 0 * one, p, periodic=False, beta_min=0.5, c_sensor=1e6)
    b = h.sensor_beta(0)
    assert np.all((b >= 0.5) & (b <= 1.0))
    assert np.all(b[:, 15:17] == 0.5)
    assert np.all(b[:, :11] == 1.0) and np.all(b[:, 21:] == 1.0)


def test_sensor_run_conserves_exactly():
    """beta varies per cell, W stays a collision invariant cell by cell
    (Eq. 6), so the totals of a three-level periodic run with the sensor
    acting stay at round-off."""
    n = 40
    refs = I.box_refs(n, n, 3, [(0, 8, 8, 16, 16)])
    refs[1][24:40, 24:40] = 1
    cs = I.smooth_random(n, n, 3, refs, seed=67, amp=0.35, beta=1.0, steps=8)
    h = make(cs)
    h.set_sensor(True, beta_min=0.5, c_sensor=20.0)
    b = h.sensor_beta(0)
    assert b[b > 0].min() < 1.0  # the sensor acts somewhere
    t0, a0 = h.totals()
    h.advance(cs.steps)
    t1, _ = h.totals()
    assert np.all(np.abs(t1 - t0) / a0 < 1e-14)


def test_sensor_keeps_lax_liu_3_physical_where_constant_beta_fails():
    """Lax-Liu configuration 3 on 128^2 to t = 0.3: with a constant beta of
    0.9 the scheme loses positivity, with the sensor (beta between 0.5 and 1,
    C = 16) density and pressure stay positive after every coarse step."""
    cs = I.riemann3(N=128, nlev=1, beta=1.0)

    def physical_to_end(beta, sensor):
        o = O.Hierarchy(cs.nx0, cs.ny0, 1, 2, cs.bc, cs.gamma, cs.c, beta, cs.inflow)
        o.set_layout([])
        o.set_state(0, cs.W[0])
        if sensor:
            o.set_sensor(True, beta_min=0.5, c_sensor=16.0)
        for _ in range(cs.steps):  # checked after every coarse step
            o.advance(1)
            W, _ = o.get_W(0)
            p = 0.4 * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])
            if not (np.all(np.isfinite(p)) and W[0].min() > 0 and p.min() > 0):
                return False
        return True

    assert not physical_to_end(0.9, False)
    assert physical_to_end(1.0, True)


# ----------------------------------------------------------------------
# the paper's validation numbers
# ----------------------------------------------------------------------

def test_exact_riemann_solver_matches_textbook_star_state():
    g = golden("sod_star_state.txt")
    p, u = ER.star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert p == pytest.approx(g["p_star"], abs=1e-5)
    assert u == pytest.approx(g["u_star"], abs=1e-5)
    s = ER.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.array([u - 1e-9, u + 1e-9]))
    assert s[0, 0] == pytest.approx(g["rho_star_L"], abs=1e-5)
    assert s[0, 1] == pytest.approx(g["rho_star_R"], abs=1e-5)


@pytest.mark.slow
def test_sod_across_interface():
    """Sec. 4.1.2: Sod tube with the interface at the diaphragm, beta = 0.9,
    t = 0.2: agreement with the exact solution, better than the uniform coarse
    grid, and total mass conserved to round-off."""
    g = golden("paper_numbers.txt")
    errs = {}
    for refine in (True, False):
        cs = I.sod_strip(n=1000, refine_right=refine)
        h = make(cs, refs=cs.refs if refine else None)
        t0, a0 = h.totals()
        h.advance(cs.steps)
        t1, _ = h.totals()
        tt = cs.steps * cs.dx0 / cs.c
        if refine:
            assert abs(t1[0] - t0[0]) / a0[0] < 10 * g["sod_mass_drift"]
        err = 0.0
        for l in range(cs.nlev):
            W, fl = h.get_W(l)
            act = fl[0] == 1
            dx = cs.dx0 / 2 ** l
            xs = -0.5 + (np.arange(W.shape[2]) + 0.5) * dx
            ex = ER.sample((1, 0, 1), (0.125, 0, 0.1), xs / tt)
            err += np.sum(np.abs(W[0][0][act] - ex[0][act])) * dx
        errs[refine] = err
    assert errs[True] < 0.0025
    assert errs[True] < errs[False]


@pytest.mark.slow
def test_stationary_vortex_second_order_with_and_without_patch():
    """Sec. 4.1.3, Eq. 30: beta_v = 2, R_c = 0.05, periodic [0,1]^2, t = 0.5;
    L2 error of |u| converges close to second order for both series, and the
    periodic totals stay at round-off."""
    g = golden("paper_numbers.txt")
    for patch in (False, True):
        errs = []
        for N in (32, 64, 128):
            nlev = 2 if patch else 1
            refs = I.box_refs(N, N, 2, [(0, N // 4, N // 4, N // 2, N // 2)]) if patch else None
            fn = lambda X, Y: I.vortex_state(X, Y, L=1.0, strength=2.0, rc=0.05, xc=0.5, yc=0.5,
                                             uinf=0.0, vinf=0.0)
            Ws = I.fill_levels(N, N, nlev, 1.0 / N, fn)
            c = I.link_speed([Ws[0]])
            h = O.Hierarchy(N, N, nlev, 2, (0, 0, 0, 0), 1.4, c, 1.0)
            h.set_layout(refs)
            for l in range(nlev):
                h.set_state(l, Ws[l])
            t0, a0 = h.totals()
            h.advance(int(round(0.5 * c * N)))
            t1, _ = h.totals()
            assert np.all(np.abs(t1 - t0) / a0 < g["vortex_conservation"])
            e2 = 0.0
            for l in range(nlev):
                W, fl = h.get_W(l)
                act = fl == 1
                dx = 1.0 / N / 2 ** l
                with np.errstate(invalid="ignore", divide="ignore"):
                    sp = np.hypot(W[1] / W[0], W[2] / W[0])
                ex = np.hypot(Ws[l][1] / Ws[l][0], Ws[l][2] / Ws[l][0])
                e2 += np.sum((sp - ex)[act] ** 2) * dx * dx
            errs.append(math.sqrt(e2))
        orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert orders[-1] > 0.9 * g["vortex_order"], (patch, errs, orders)
        assert orders[0] > 1.6


@pytest.mark.slow
def test_explosion_in_a_box_drift_within_the_papers_values():
    """Sec. 4.2: explosion in a box with reflective walls, N0 = 256 plus the
    centred ratio-2 patch over [0.25, 0.75]^2, sampled every 0.05 up to
    t = 0.5.  The paper's refined run drifts at most 3.2e-14 in mass and
    5.3e-14 in energy; walls exchange no mass or energy, so the oracle's
    drift (exact sums of its state) must stay within those values."""
    g = golden("paper_numbers.txt")
    cs = I.explosion(N=256, beta=0.9)
    h = O.Hierarchy(cs.nx0, cs.ny0, cs.nlev, 2, cs.bc, cs.gamma, cs.c, cs.beta)
    h.set_layout(cs.refs)
    for l in range(cs.nlev):
        h.set_state(l, cs.W[l])
    t0, _ = h.totals()
    dt = cs.dx0 / cs.c
    done, worst_m, worst_e = 0, 0.0, 0.0
    for i in range(10):
        s = int(round(0.05 * (i + 1) / dt))
        h.advance(s - done)
        done = s
        t1, _ = h.totals()
        worst_m = max(worst_m, abs(t1[0] - t0[0]) / t0[0])
        worst_e = max(worst_e, abs(t1[3] - t0[3]) / t0[3])
    assert worst_m <= g["explosion_mass_drift"], worst_m
    assert worst_e <= g["explosion_energy_drift"], worst_e
