"""Pins of the oracle's coupling and regrid call sites.

The single-cell operators (reconstruction weights, minmod, merge, split) are
pinned elsewhere; these tests pin how the time step and the regrid CALL them:
which coarse sample is "current" and which "previous", the direction of the
temporal slope, the orientation of the tangential index j, the presence of
the tangential slope, the reflux average and the sign and axis of the split
slopes.  Conservation, uniform states, the ratio-1 limit and the symmetry
pins hold for any of those choices, so they cannot tell them apart.

What can: with beta = 0 the collision is the identity and the scheme is pure
shift transport (Sec. 2.2, Eq. 5).  A population field that is LINEAR in
space is then also linear in time at every coarse ring cell, and

  * the temporal reconstruction (Eq. 1d-recon / 2d-recon, k term) of the
    value entering the fine cell after fine sub-step k is exact for data
    linear in time,
  * the tangential minmod term (Eqs. 2d-recon-tanslope, 2d-recon) is exact
    for data linear along the edge (both one-sided differences agree),
  * the reflux average (Eq. 2d-reflux) of a linear field is exact,

so every active cell of every level must hold the exactly transported
linear profile.  With dyadic data every operation is exact in binary64 and
the comparison is bit for bit.  Likewise the minmod slopes of a split
(Eqs. amr-slope, amr-split) reproduce a linear field at the child centres
exactly, and the merge average (Eq. amr-merge) returns the parent centre.

The acoustic pulse of Sec. 4.1.1 pins the whole scheme against the crossing
time the paper prints.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2609_35529_b300 import inputs as I

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


# direction of population q = 4 i + k: i in +x, -x, +y, -y
CX = np.array([1, -1, 0, 0])
CY = np.array([0, 0, 1, -1])


def level_centres(nx0, ny0, l):
    """Cell centres of level l in coarse-cell units (dyadic)."""
    s = 2.0 ** -l
    X = (np.arange(nx0 * 2 ** l) + 0.5) * s
    Y = (np.arange(ny0 * 2 ** l) + 0.5) * s
    return np.meshgrid(X, Y)


def linear_pops(nx0, ny0, l, ax, ay, shift=0):
    """f_q = 1 + ax_q (X - cx_q n) + ay_q (Y - cy_q n): the field at t = 0
    carried `shift` coarse steps by exact shift transport (c dt_0 = one
    coarse cell)."""
    X, Y = level_centres(nx0, ny0, l)
    f = np.empty((16,) + X.shape)
    for q in range(16):
        i = q // 4
        f[q] = 1.0 + ax[q] * (X - CX[i] * shift) + ay[q] * (Y - CY[i] * shift)
    return f


def slopes(axis):
    """Distinct dyadic slopes per population, all along one axis."""
    s = np.array([(q + 1) / 128.0 for q in range(16)])
    z = np.zeros(16)
    return (s, z) if axis == "x" else (z, s)


def patch_refs(nx0, ny0, nlev):
    """A coarse patch in the interior and, for three levels, a nested one."""
    refs = I.box_refs(nx0, ny0, nlev, [(0, 16, 8, 16, 16)])
    if nlev == 3:
        refs[1][24:40, 40:56] = 1  # level-1 cells; its face neighbours are on level 1
    return refs


@pytest.mark.parametrize("nlev", [2, 3])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_linear_profile_is_transported_exactly_across_interfaces(axis, nlev):
    """beta = 0, every population linear along `axis`.  The populations moving
    along `axis` cross the patch edges normal to it (temporal term of Eq.
    2d-recon, reflux of Eq. 2d-reflux); the others are constant in time and
    linear along the edges they cross (tangential term).  After the first
    coarse step -- whose faces have no previous sample yet, so B = 0 -- the
    state is reset to the exact one and the run continues; from then on every
    active cell away from the non-periodic sides must be bit-exact."""
    nx0 = ny0 = 48
    refs = patch_refs(nx0, ny0, nlev)
    if axis == "y":  # the same layout transposed
        refs = [np.ascontiguousarray(r.T) for r in refs]
    ax, ay = slopes(axis)
    # outflow across `axis`, periodic along the other one (the profile is
    # constant there)
    bc = (1, 1, 0, 0) if axis == "x" else (0, 0, 1, 1)
    h = O.Hierarchy(nx0, ny0, nlev, 2, bc, 1.4, 1.0, 0.0)
    h.set_layout(refs)
    for l in range(nlev):
        h.set_f(l, linear_pops(nx0, ny0, l, ax, ay, 0))
    h.advance(1)
    for l in range(nlev):
        h.set_f(l, linear_pops(nx0, ny0, l, ax, ay, 1))
    m = 7
    h.advance(m)
    n = 1 + m
    for l in range(nlev):
        want = linear_pops(nx0, ny0, l, ax, ay, n)
        got = h.get_f(l)
        act = h.active_masks()[l]
        X, Y = level_centres(nx0, ny0, l)
        C = X if axis == "x" else Y
        # boundary values (zero-gradient outflow) travel inwards one coarse
        # cell per coarse step
        keep = act & (C > n + 1) & (C < nx0 - n - 1)
        assert keep.sum() > 0
        assert np.array_equal(got[:, keep], want[:, keep]), f"level {l}"


def test_linear_profile_after_first_cycle_with_a_fresh_face():
    """The first cycle of a new face has no previous sample: the paper's
    affine model then has B = 0 (prev := cur), which hands the current sample
    to both fine sub-steps.  Against the exact transport the two fine cells
    behind the edge are then off by a quarter coarse cell of the linear
    profile, one on each side -- a closed form that pins which sample the
    oracle hands on: the current one, to both sub-steps."""
    nx0 = ny0 = 48
    refs = patch_refs(nx0, ny0, 2)
    ax, ay = slopes("x")
    h = O.Hierarchy(nx0, ny0, 2, 2, (1, 1, 0, 0), 1.4, 1.0, 0.0)
    h.set_layout(refs)
    for l in range(2):
        h.set_f(l, linear_pops(nx0, ny0, l, ax, ay, 0))
    h.advance(1)
    got = h.get_f(1)
    want = linear_pops(nx0, ny0, 1, ax, ay, 1)
    # +x populations: the patch's west edge is at coarse x = 16, fine x = 32.
    # After one coarse step the fine cells 32 and 33 hold what entered during
    # sub-steps 2 and 1: both equal the coarse sample a = f(15.5), whereas the
    # exact values are f(15.75 - 1 + 1) shifted: f(x - 1) at x = 16.25 / 16.75.
    rows = slice(2 * 8, 2 * 24)
    for k in range(4):
        q = 0 * 4 + k
        a = 1.0 + ax[q] * 15.5  # coarse sample of L0 at t = 0
        assert np.all(got[q, rows, 32] == a)
        assert np.all(got[q, rows, 33] == a)
        assert np.all(want[q, rows, 32] == a - ax[q] * 0.25)
        assert np.all(want[q, rows, 33] == a + ax[q] * 0.25)


def linear_field_pops(nx0, ny0, l):
    """Populations linear in both X and Y with different slopes per axis."""
    ax = np.array([(q + 1) / 64.0 for q in range(16)])
    ay = np.array([(17 - q) / 256.0 for q in range(16)])
    X, Y = level_centres(nx0, ny0, l)
    return np.stack([1.0 + ax[q] * X + ay[q] * Y for q in range(16)])


def garbage_under(refs_l, f, value=7.0):
    """Overwrites the populations of covered cells (never read as state)."""
    f = f.copy()
    f[:, refs_l.astype(bool)] = value
    return f


@pytest.mark.parametrize("nlev", [2, 3])
def test_split_of_a_linear_field_is_exact_at_child_centres(nlev):
    """Eqs. amr-slope, amr-split: both one-sided differences of a linear field
    equal its slope, so the minmod slopes are the slopes and the children land
    on the field at their own centres -- bit for bit with dyadic data.  A
    negated slope, a swapped axis or a swapped child offset fails here.  With
    three levels the level-2 cells are split from freshly split level-1 cells
    (coarsest level first)."""
    nx0 = ny0 = 32
    h = O.Hierarchy(nx0, ny0, nlev, 2, (1, 1, 1, 1), 1.4, 5.0, 0.9)
    h.set_layout(None)
    h.set_f(0, linear_field_pops(nx0, ny0, 0))
    refs = I.box_refs(nx0, ny0, nlev, [(0, 8, 8, 16, 16)])
    if nlev == 3:
        refs[1][24:40, 24:40] = 1
    h.regrid(refs)
    for l in range(1, nlev):
        act = h.active_masks()[l]
        assert act.sum() > 0
        got = h.get_f(l)
        want = linear_field_pops(nx0, ny0, l)
        assert np.array_equal(got[:, act], want[:, act]), f"level {l}"


def test_split_next_to_a_covered_neighbour_uses_its_children():
    """Growing a patch: a cell that enters refinement next to one that stays
    covered takes that neighbour's value from the average of its children
    (the covered coarse value itself is not state).  The covered coarse cells
    are filled with garbage first, so only the composite reading is exact."""
    nx0 = ny0 = 32
    h = O.Hierarchy(nx0, ny0, 2, 2, (1, 1, 1, 1), 1.4, 5.0, 0.9)
    small = I.box_refs(nx0, ny0, 2, [(0, 12, 12, 8, 8)])
    h.set_layout(small)
    h.set_f(0, garbage_under(small[0], linear_field_pops(nx0, ny0, 0)))
    h.set_f(1, linear_field_pops(nx0, ny0, 1))
    big = I.box_refs(nx0, ny0, 2, [(0, 8, 8, 16, 16)])
    h.regrid(big)
    act = h.active_masks()[1]
    assert np.array_equal(h.get_f(1)[:, act], linear_field_pops(nx0, ny0, 1)[:, act])


def test_merge_of_a_linear_field_is_the_parent_centre_value():
    """Eq. amr-merge: the plain average of the four children of a linear field
    is the field at the parent centre, exactly."""
    nx0 = ny0 = 32
    h = O.Hierarchy(nx0, ny0, 3, 2, (1, 1, 1, 1), 1.4, 5.0, 0.9)
    refs = I.box_refs(nx0, ny0, 3, [(0, 8, 8, 16, 16)])
    refs[1][24:40, 24:40] = 1
    h.set_layout(refs)
    h.set_f(0, garbage_under(refs[0], linear_field_pops(nx0, ny0, 0)))
    h.set_f(1, garbage_under(refs[1], linear_field_pops(nx0, ny0, 1)))
    h.set_f(2, linear_field_pops(nx0, ny0, 2))
    h.regrid(I.empty_refs(nx0, ny0, 3))
    assert np.array_equal(h.get_f(0), linear_field_pops(nx0, ny0, 0))


# ----------------------------------------------------------------------
# Sec. 4.1.1: acoustic pulse across the interface
# ----------------------------------------------------------------------

def acoustic_pulse_track(refine=True, beta=0.99, t_end=1.0):
    """The paper's set-up in a quasi-1-D strip: coarse x in [-1, 0] (dx 0.01),
    fine x in [0, 1.5] (dx 0.005, r = 2), rho0 = 1, u0 = 0, c_s0 = 1, a
    right-moving linear pulse of amplitude 0.01, sigma 0.05, centred at
    x0 = -0.6 (Eq. val-acoustic-ic); refine=False runs the same strip on the
    coarse grid alone.  Returns per coarse step (t, x_peak, r) with the peak
    located by a three-point parabola on the combined grid and r the largest
    |rho - rho0| left behind in x < -0.1."""
    dx0 = 0.01
    nx0, ny0 = 250, 1
    gamma = 1.4
    rho0, cs0, A, sig, x0 = 1.0, 1.0, 0.01, 0.05, -0.6
    p0 = rho0 * cs0 ** 2 / gamma

    def fn(X, Y):
        rho = rho0 + A * np.exp(-((X - x0) ** 2) / (2 * sig ** 2))
        u = cs0 / rho0 * (rho - rho0)
        p = p0 + cs0 ** 2 * (rho - rho0)
        return I.conserved(rho, u, np.zeros_like(X), p, gamma)

    nlev = 2 if refine else 1
    refs = I.box_refs(nx0, ny0, 2, [(0, 100, 0, 150, 1)])[: nlev - 1]
    Ws = I.fill_levels(nx0, ny0, nlev, dx0, fn, x0=-1.0)
    c = I.link_speed([Ws[0]], gamma)
    h = O.Hierarchy(nx0, ny0, nlev, 2, (1, 1, 0, 0), gamma, c, beta)
    h.set_layout(refs if refine else None)
    for l in range(nlev):
        h.set_state(l, Ws[l])
    if refine:
        xs = np.concatenate([-1.0 + (np.arange(100) + 0.5) * dx0, (np.arange(300) + 0.5) * dx0 / 2])
    else:
        xs = -1.0 + (np.arange(nx0) + 0.5) * dx0
    dt = dx0 / c
    track = []
    for n in range(1, int(t_end / dt) + 1):
        h.advance(1)
        W0, _ = h.get_W(0)
        if refine:
            W1, _ = h.get_W(1)
            d = np.concatenate([W0[0, 0, :100], W1[0, :, 200:].mean(axis=0)]) - rho0
        else:
            d = W0[0, 0] - rho0
        i = int(np.argmax(d))
        x_a, x_b, x_c = xs[i - 1], xs[i], xs[i + 1]
        y_a, y_b, y_c = d[i - 1], d[i], d[i + 1]
        # vertex of the parabola through three (non-uniformly spaced) points
        num = (x_b - x_a) ** 2 * (y_b - y_c) - (x_b - x_c) ** 2 * (y_b - y_a)
        den = (x_b - x_a) * (y_b - y_c) - (x_b - x_c) * (y_b - y_a)
        track.append((n * dt, x_b - 0.5 * num / den, np.abs(d[xs < -0.1]).max()))
    return np.array(track)


def crossing_time(tr):
    t, x = tr[:, 0], tr[:, 1]
    j = int(np.argmax(x > 0.0))
    assert j > 0
    return t[j - 1] + (0.0 - x[j - 1]) * (t[j] - t[j - 1]) / (x[j] - x[j - 1])


@pytest.mark.slow
def test_acoustic_pulse_crosses_the_interface_on_time_and_transparently():
    """Sec. 4.1.1: the paper measures t_cross = 0.6034 against the geometric
    |x0| / c_s0 = 0.600 and a speed error below 1.2 % throughout.  The crest
    of a pulse of amplitude 0.01 moves at its characteristic speed
    u + c_s = 1 + (gamma + 1)/2 * 0.01 = 1.012 rather than at c_s0, so the
    scheme's crossing time may sit on either side of 0.600 by about that
    much: pinned here to the paper's 1.2 % band, and so is the speed on each
    side away from the crossing.  The interface itself must be transparent:
    the crossing time equals that of the same pulse on the coarse grid alone
    to 0.2 %, and what the pulse leaves behind on the coarse side is no more
    than on the coarse grid alone (+10 %)."""
    g = golden("paper_numbers.txt")
    ref = acoustic_pulse_track(refine=True)
    uni = acoustic_pulse_track(refine=False)
    tc, tu = crossing_time(ref), crossing_time(uni)
    assert abs(tc - g["acoustic_t_exact"]) <= 0.012 * g["acoustic_t_exact"], tc
    assert abs(tc - g["acoustic_t_cross"]) <= 0.02 * g["acoustic_t_cross"], tc
    assert abs(tc - tu) <= 0.002 * tu, (tc, tu)
    t, x = ref[:, 0], ref[:, 1]
    for lo, hi in ((-0.5, -0.15), (0.15, 0.35)):
        sel = (x > lo) & (x < hi)
        assert sel.sum() > 5
        speed = np.polyfit(t[sel], x[sel], 1)[0]
        assert abs(speed - 1.0) <= 0.012, (lo, hi, speed)
    late_ref = ref[ref[:, 0] > 0.85, 2].max()
    late_uni = uni[uni[:, 0] > 0.85, 2].max()
    assert late_ref <= 1.1 * late_uni, (late_ref, late_uni)


@pytest.mark.slow
def test_advected_vortex_converges_at_second_order_with_and_without_the_patch():
    """Sec. 4.1.3 reports close to second order with no reduction from the
    refinement interface.  The advected vortex (strength 5, free stream
    (1, 1), one period on [0, 10]^2) at N = 64 and 128, with and without the
    central ratio-2 patch; the error is measured against the exact solution
    at the run's actual end time steps * dt (the vortex carried by the free
    stream over that time), not at t = 10: the step count rounds 10 / dt, and
    the mismatch of up to dt / 2 would add an error of first order in dt."""
    orders = {}
    for patch in (True, False):
        errs = []
        for N in (64, 128):
            cs = I.vortex(N=N, patch=patch)
            h = O.Hierarchy(cs.nx0, cs.ny0, cs.nlev, 2, cs.bc, cs.gamma, cs.c, cs.beta)
            h.set_layout(cs.refs if patch else None)
            for l in range(cs.nlev):
                h.set_state(l, cs.W[l])
            h.advance(cs.steps)
            t_end = cs.steps * cs.dx0 / cs.c
            xc = (5.0 + t_end) % 10.0
            ex = I.fill_levels(N, N, cs.nlev, cs.dx0, lambda X, Y: I.vortex_state(X, Y, xc=xc, yc=xc))
            e = 0.0
            for l in range(cs.nlev):
                W, fl = h.get_W(l)
                act = fl == 1
                a = cs.dx0 / 2 ** l
                e += float(np.sum((W[0][act] - ex[l][0][act]) ** 2)) * a * a
            errs.append(math.sqrt(e))
        orders[patch] = math.log2(errs[0] / errs[1])
    assert orders[True] >= 1.85, orders
    assert orders[False] >= 1.85, orders
    assert abs(orders[True] - orders[False]) <= 0.15, orders
