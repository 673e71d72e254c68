"""Seeded synthetic inputs: initial states, refinement layouts and run settings.

This module holds no arithmetic of the method itself (no equilibrium, no
collision, no coupling); it only builds the closed-form initial conditions of
the paper's two-dimensional test problems and the refinement layouts that go
with them.  Both the CUDA path and the test oracle consume the same recipes.

Conventions: level l has ``nx0 * 2**l`` by ``ny0 * 2**l`` cells; the
conserved state is ``W[4, ny, nx]`` with fields (rho, rho*u, rho*v, rho*E);
a refinement mask ``ref[l]`` is ``uint8[ny_l, nx_l]`` on the level it refines
(1 = covered by level l+1).  Cell centres sit at ``(i + 0.5) * dx_l``.

Recipes (the paper's workloads):
  * ``pulse2l``      two-level Gaussian density pulse straddling a patch edge
  * ``vortex``       advected isentropic vortex (Sec. 4.1.3, Eq. 30) with a
                     central ratio-2 patch
  * ``riemann3``     Lax-Liu configuration 3 quadrant problem (Sec. 4.3.1),
                     three levels over the diagonal band
  * ``shockbubble``  Mach 1.22 shock into a light bubble, adaptive levels
  * ``sod_strip``    Sod tube across an interface (Sec. 4.1.2), quasi-1-D
  * ``laxliu12``     Lax-Liu configuration 12 (Sec. 4.3.2)
  * ``explosion``    explosion in a box with reflective walls (Sec. 4.2)
  * ``smooth_random`` seeded smooth periodic field for invariance tests
"""
from dataclasses import dataclass, field
import math

import numpy as np

GAMMA = 1.4
BC_PERIODIC, BC_OUTFLOW, BC_INFLOW, BC_REFLECT = 0, 1, 2, 3


@dataclass
class Case:
    name: str
    nx0: int
    ny0: int
    nlev: int
    bc: tuple                      # sides W, E, S, N
    gamma: float
    c: float
    beta: float
    W: list                        # per level W[4, ny_l, nx_l]
    refs: list                     # per level l < nlev-1: uint8[ny_l, nx_l]
    steps: int
    dx0: float = 1.0
    block: int = 8
    inflow: np.ndarray = field(default_factory=lambda: np.zeros((4, 4)))
    amr: dict = None               # {"tol":..., "buffer":..., "every":...} when adaptive

    def lups_per_step(self):
        """Cell updates per coarse step (active cells x sub-steps)."""
        tot = 0
        for l in range(self.nlev):
            on = level_in(self.refs, l, self.nlev, (self.ny0, self.nx0))
            cov = self.refs[l].astype(bool) if l < self.nlev - 1 else np.zeros_like(on)
            tot += int(np.count_nonzero(on & ~cov)) * (2 ** l)
        return tot


# --------------------------------------------------------------------------
# primitive <-> conserved (input construction only)
# --------------------------------------------------------------------------

def conserved(rho, u, v, p, gamma=GAMMA):
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E * np.ones_like(rho)])


def link_speed(Ws, gamma=GAMMA, safety=1.1, D=2):
    """c = safety * D * max(|u_alpha| + c_s) over the initial data.

    The D2Q4 vector equilibrium has a non-negative Jacobian,
    1/(2D) - |lambda|/(2c) >= 0, when c >= D max|lambda|.
    """
    m = 0.0
    for W in Ws:
        rho = W[0]
        u = W[1] / rho
        v = W[2] / rho
        p = (gamma - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v))
        cs = np.sqrt(gamma * np.maximum(p, 0.0) / rho)
        m = max(m, float(np.max(np.maximum(np.abs(u), np.abs(v)) + cs)))
    return safety * D * m


def centres(n, dx, x0=0.0):
    return x0 + (np.arange(n) + 0.5) * dx


# --------------------------------------------------------------------------
# layouts
# --------------------------------------------------------------------------

def level_in(refs, l, nlev, shape0=None):
    """Mask of cells of level l (children of cells refined on l-1)."""
    if l == 0:
        shape = refs[0].shape if refs else shape0
        return np.ones(shape, dtype=bool)
    parent = level_in(refs, l - 1, nlev, shape0) & refs[l - 1].astype(bool)
    return np.repeat(np.repeat(parent, 2, axis=0), 2, axis=1)


def empty_refs(nx0, ny0, nlev):
    return [np.zeros((ny0 * 2 ** l, nx0 * 2 ** l), dtype=np.uint8) for l in range(nlev - 1)]


def box_refs(nx0, ny0, nlev, boxes):
    """boxes: list of (level, i0, j0, ni, nj) in level cells -> ref masks."""
    refs = empty_refs(nx0, ny0, nlev)
    for (l, i0, j0, ni, nj) in boxes:
        refs[l][j0:j0 + nj, i0:i0 + ni] = 1
    return refs


def _dilate(mask, periodic_x, periodic_y, rad=1):
    out = mask.copy()
    ny, nx = mask.shape
    for dy in range(-rad, rad + 1):
        for dx in range(-rad, rad + 1):
            if dx == 0 and dy == 0:
                continue
            sh = np.zeros_like(mask)
            ys = slice(max(dy, 0), ny + min(dy, 0))
            yd = slice(max(-dy, 0), ny + min(-dy, 0))
            xs = slice(max(dx, 0), nx + min(dx, 0))
            xd = slice(max(-dx, 0), nx + min(-dx, 0))
            if periodic_x and periodic_y:
                sh = np.roll(np.roll(mask, dy, axis=0), dx, axis=1)
            else:
                sh[ys, xs] = mask[yd, xd]
            out |= sh
    return out


def blocks_from_cells(mask, block):
    """Rounds a cell mask up to aligned block x block blocks."""
    ny, nx = mask.shape
    by, bx = -(-ny // block), -(-nx // block)
    pad = np.zeros((by * block, bx * block), dtype=bool)
    pad[:ny, :nx] = mask
    b = pad.reshape(by, block, bx, block).any(axis=(1, 3))
    full = np.repeat(np.repeat(b, block, axis=0), block, axis=1)[:ny, :nx]
    return full


def nested_band_refs(nx0, ny0, nlev, widths, block=8, bc=(1, 1, 1, 1)):
    """Diagonal band |x - y| <= w_l (unit square), one width per refined level,
    rounded to blocks and trimmed so every level nests properly."""
    refs = empty_refs(nx0, ny0, nlev)
    periodic = bc[0] == BC_PERIODIC
    for l in range(nlev - 1):
        ny, nx = ny0 * 2 ** l, nx0 * 2 ** l
        # block centres
        by, bx = ny // block, nx // block
        xc = (np.arange(bx) + 0.5) * block / nx
        yc = (np.arange(by) + 0.5) * block / ny
        band = np.abs(xc[None, :] - yc[:, None]) <= widths[l]
        cells = np.repeat(np.repeat(band, block, axis=0), block, axis=1)
        m = np.zeros((ny, nx), dtype=bool)
        m[:cells.shape[0], :cells.shape[1]] = cells
        if l >= 1:
            on = level_in(refs, l, nlev)
            # a refined block must keep its 8-neighbourhood on level l
            inner = ~_dilate(~on, periodic, periodic, 1)
            keep = m & inner
            # drop blocks that are not entirely inside
            bl = keep.reshape(ny // block, block, nx // block, block).all(axis=(1, 3)) & \
                m.reshape(ny // block, block, nx // block, block).all(axis=(1, 3))
            m = np.repeat(np.repeat(bl, block, axis=0), block, axis=1)
        refs[l] = m.astype(np.uint8)
    return refs


def fill_levels(nx0, ny0, nlev, dx0, fn, x0=0.0, y0=0.0):
    """Evaluates fn(X, Y) -> W on the cell centres of every level."""
    Ws = []
    for l in range(nlev):
        dx = dx0 / 2 ** l
        xs = centres(nx0 * 2 ** l, dx, x0)
        ys = centres(ny0 * 2 ** l, dx, y0)
        X, Y = np.meshgrid(xs, ys)
        Ws.append(np.ascontiguousarray(fn(X, Y)))
    return Ws


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def pulse2l(n=64, patch=(24, 40), steps=200, amp=0.2, sigma=4.0, beta=0.9, gamma=GAMMA):
    """Two-level static refinement: periodic n x n coarse grid (dx0 = 1), a
    centred ratio-2 patch over coarse cells [patch[0], patch[1])^2, uniform
    rho=1, p=1, u=(0.5, 0.25) plus an isobaric Gaussian density pulse centred
    on the patch's left edge."""
    a, b = patch
    refs = box_refs(n, n, 2, [(0, a, a, b - a, b - a)])
    xc, yc = float(a), 0.5 * (a + b)

    def fn(X, Y):
        r2 = (X - xc) ** 2 + (Y - yc) ** 2
        rho = 1.0 + amp * np.exp(-r2 / (2.0 * sigma ** 2))
        return conserved(rho, 0.5 * np.ones_like(X), 0.25 * np.ones_like(X), np.ones_like(X), gamma)

    Ws = fill_levels(n, n, 2, 1.0, fn)
    c = link_speed([Ws[0]], gamma)
    return Case("pulse2l", n, n, 2, (0, 0, 0, 0), gamma, c, beta, Ws, refs, steps, dx0=1.0)


def vortex_state(X, Y, L=10.0, strength=5.0, rc=1.0, xc=5.0, yc=5.0, uinf=1.0, vinf=1.0, gamma=GAMMA):
    """Isentropic vortex of Eq. 30 (circulation `strength`, core radius rc)
    carried by a free stream (uinf, vinf); rho_inf = p_inf = T_inf = 1.
    Periodic images within one period are superposed in distance only
    through the nearest image."""
    dx = (X - xc + 0.5 * L) % L - 0.5 * L
    dy = (Y - yc + 0.5 * L) % L - 0.5 * L
    r2 = (dx * dx + dy * dy) / (rc * rc)
    g = np.exp(0.5 * (1.0 - r2))
    du = -strength / (2.0 * math.pi) * dy / rc * g
    dv = strength / (2.0 * math.pi) * dx / rc * g
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return conserved(rho, uinf + du, vinf + dv, p, gamma)


def vortex(N=128, steps=None, beta=1.0, periods=1.0, gamma=GAMMA, patch=True, fine_state=True):
    """Advected isentropic vortex on the periodic square [0,10]^2, strength 5,
    free stream (1, 1), N x N coarse cells, a ratio-2 patch over the central
    N/2 x N/2 coarse cells (25 % of the area).  `steps` defaults to one full
    period (t = 10)."""
    L = 10.0
    dx0 = L / N
    nlev = 2 if patch else 1
    refs = box_refs(N, N, 2, [(0, N // 4, N // 4, N // 2, N // 2)]) if patch else []
    Ws = fill_levels(N, N, nlev if fine_state else 1, dx0, lambda X, Y: vortex_state(X, Y, L=L, gamma=gamma))
    c_phys = link_speed([Ws[0]], gamma)          # physical link speed
    dt = dx0 / c_phys
    if steps is None:
        steps = int(round(periods * L / dt))
    # the scheme works in lattice units: c_lattice = dx0 / dt_phys = c_phys * (1/dx0)*dx0
    case = Case("vortex", N, N, nlev, (0, 0, 0, 0), gamma, c_phys, beta, Ws, refs, steps, dx0=dx0)
    return case


LAXLIU3 = {  # (rho, u, v, p) per quadrant, Lax-Liu configuration 3
    "NE": (1.5, 0.0, 0.0, 1.5),
    "NW": (0.5323, 1.206, 0.0, 0.3),
    "SW": (0.138, 1.206, 1.206, 0.029),
    "SE": (0.5323, 0.0, 1.206, 0.3),
}


def quadrant_state(X, Y, states, gamma=GAMMA, xm=0.5, ym=0.5):
    out = np.zeros((4,) + X.shape)
    for key, sel in (("NE", (X >= xm) & (Y >= ym)), ("NW", (X < xm) & (Y >= ym)),
                     ("SW", (X < xm) & (Y < ym)), ("SE", (X >= xm) & (Y < ym))):
        rho, u, v, p = states[key]
        w = conserved(np.full(X.shape, rho), u, v, p, gamma)
        out[:, sel] = w[:, sel]
    return out


def riemann3(N=1024, nlev=3, t_end=0.3, steps=None, beta=0.7, widths=None, gamma=GAMMA, states=None, safety=1.1,
             fine_state=True):
    """Four-quadrant Riemann problem on [0,1]^2 (zero-gradient outflow on all
    sides), N x N coarse cells, static levels over the diagonal band
    |x - y| <= w (about 15 % of the area on level 1, nested narrower bands
    above).  `steps` defaults to t_end / dt0."""
    states = states or LAXLIU3
    dx0 = 1.0 / N
    if widths is None:
        widths = [0.08, 0.04, 0.02][: nlev - 1]
    bc = (BC_OUTFLOW,) * 4
    refs = nested_band_refs(N, N, nlev, widths, block=8, bc=bc) if nlev > 1 else []
    Ws = fill_levels(N, N, nlev if fine_state else 1, dx0, lambda X, Y: quadrant_state(X, Y, states, gamma))
    c = link_speed([Ws[0]], gamma, safety=safety)
    if steps is None:
        steps = int(math.ceil(t_end * c / dx0))
    return Case("riemann3", N, N, nlev, bc, gamma, c, beta, Ws, refs, steps, dx0=dx0)


LAXLIU12 = {  # (rho, u, v, p) per quadrant, Lax-Liu configuration 12 (Sec. 4.3.2, Eq. 32)
    "NE": (0.5313, 0.0, 0.0, 0.4),
    "NW": (1.0, 0.7276, 0.0, 1.0),
    "SW": (0.8, 0.0, 0.0, 1.0),
    "SE": (1.0, 0.0, 0.7276, 1.0),
}


def laxliu12(N=256, nlev=3, t_end=0.25, steps=None, beta=0.7, gamma=GAMMA):
    """Lax-Liu configuration 12 on [0,1]^2 with levels over the diagonal band
    that the NE-NW and NE-SE contacts roll up along (outflow on all sides)."""
    cs = riemann3(N=N, nlev=nlev, t_end=t_end, steps=steps, beta=beta, widths=[0.06, 0.03, 0.015][: nlev - 1],
                  gamma=gamma, states=LAXLIU12)
    cs.name = "laxliu12"
    return cs


def explosion(N=256, patch=True, beta=0.9, t_end=0.5, steps=None, gamma=GAMMA, safety=2.0):
    """Explosion in a box (Sec. 4.2, Eq. 31): rho = p = 5 inside the circle of
    radius 0.3 around (0.4, 0.4), 1 outside, at rest; reflective walls on all
    sides; optional centred ratio-2 patch over [0.25, 0.75]^2."""
    dx0 = 1.0 / N
    nlev = 2 if patch else 1
    refs = box_refs(N, N, 2, [(0, N // 4, N // 4, N // 2, N // 2)]) if patch else []

    def fn(X, Y):
        inside = (X - 0.4) ** 2 + (Y - 0.4) ** 2 < 0.3 ** 2
        rho = np.where(inside, 5.0, 1.0)
        return conserved(rho, np.zeros_like(X), np.zeros_like(X), rho, gamma)

    Ws = fill_levels(N, N, nlev, dx0, fn)
    c = link_speed([Ws[0]], gamma, safety=safety)
    if steps is None:
        steps = int(math.ceil(t_end * c / dx0))
    bc = (BC_REFLECT,) * 4
    return Case("explosion", N, N, nlev, bc, gamma, c, beta, Ws, refs, steps, dx0=dx0)


def normal_shock(mach, rho1=1.0, p1=1.0, gamma=GAMMA):
    """Post-shock state (rho2, u2, p2) behind a shock moving at mach*c1 into
    gas at rest (textbook Rankine-Hugoniot relations) and the shock speed."""
    c1 = math.sqrt(gamma * p1 / rho1)
    M2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p2 = p1 * (2.0 * gamma * M2 - (gamma - 1.0)) / (gamma + 1.0)
    s = mach * c1
    u2 = s * (1.0 - rho1 / rho2)
    return rho2, u2, p2, s


def shockbubble(nx0=2048, ny0=1024, nlev=3, steps=4000, beta=0.7, tol=0.02, buffer=2, every=4,
                mach=1.22, bubble_rho=0.14, gamma=GAMMA):
    """Mach 1.22 planar shock (at x = 0.25, moving +x) into a circular bubble
    of density ratio 0.14, radius H/8, centred at (0.5, 0.5) on [0,2]x[0,1].
    Inflow (post-shock equilibrium) on the west side, outflow east, periodic
    south/north.  Adaptive levels from the density-gradient indicator."""
    dx0 = 2.0 / nx0
    rho2, u2, p2, _ = normal_shock(mach, gamma=gamma)

    def fn(X, Y):
        rho = np.ones_like(X)
        u = np.zeros_like(X)
        p = np.ones_like(X)
        bub = (X - 0.5) ** 2 + (Y - 0.5) ** 2 < 0.125 ** 2
        rho[bub] = bubble_rho
        post = X < 0.25
        rho[post] = rho2
        u[post] = u2
        p[post] = p2
        return conserved(rho, u, np.zeros_like(X), p, gamma)

    Ws = fill_levels(nx0, ny0, 1, dx0, fn)
    c = link_speed(Ws, gamma)
    inflow = np.zeros((4, 4))
    inflow[0] = conserved(np.array(rho2), u2, 0.0, p2, gamma)
    bc = (BC_INFLOW, BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC)
    refs = empty_refs(nx0, ny0, nlev)
    Wl = Ws + [np.zeros((4, ny0 * 2 ** l, nx0 * 2 ** l)) for l in range(1, nlev)]
    return Case("shockbubble", nx0, ny0, nlev, bc, gamma, c, beta, Wl, refs, steps, dx0=dx0,
                inflow=inflow, amr={"tol": tol, "buffer": buffer, "every": every})


def sod_strip(n=1000, strip=4, beta=0.9, t_end=0.2, refine_right=True, block=4, gamma=GAMMA, safety=2.0):
    """Sod tube on [-0.5, 0.5] (interface and diaphragm at x = 0): coarse
    dx = 1/n on the left, ratio-2 level on the right half; a strip of
    `strip` cells, periodic in y; zero-gradient outflow in x."""
    dx0 = 1.0 / n
    nlev = 2 if refine_right else 1
    refs = box_refs(n, strip, 2, [(0, n // 2, 0, n // 2, strip)]) if refine_right else []

    def fn(X, Y):
        left = X < 0.0
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        return conserved(rho, np.zeros_like(X), np.zeros_like(X), p, gamma)

    Ws = fill_levels(n, strip, nlev, dx0, fn, x0=-0.5)
    # the star state moves faster than anything in the initial data
    # (|u| + c_s = 1.93 against 1.18), so the margin is wider here
    c = link_speed([Ws[0]], gamma, safety=safety)
    steps = int(round(t_end * c / dx0))
    bc = (BC_OUTFLOW, BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC)
    return Case("sod", n, strip, nlev, bc, gamma, c, beta, Ws, refs, steps, dx0=dx0, block=block)


def smooth_random(nx0, ny0, nlev, refs, seed=0, amp=0.05, modes=3, beta=0.9, steps=10, gamma=GAMMA,
                  bc=(0, 0, 0, 0)):
    """Seeded smooth periodic field: a few random Fourier modes on top of
    rho = 1, u = (0.3, -0.2), p = 1."""
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=(4, modes, modes, 2))

    def fld(X, Y, k):
        s = np.zeros_like(X)
        for a in range(modes):
            for b in range(modes):
                ph = 2 * math.pi * (a * X / nx0 + b * Y / ny0)
                s += coef[k, a, b, 0] * np.cos(ph) + coef[k, a, b, 1] * np.sin(ph)
        return s / modes

    def fn(X, Y):
        rho = 1.0 + amp * fld(X, Y, 0)
        u = 0.3 + amp * fld(X, Y, 1)
        v = -0.2 + amp * fld(X, Y, 2)
        p = 1.0 + amp * fld(X, Y, 3)
        return conserved(rho, u, v, p, gamma)

    Ws = fill_levels(nx0, ny0, nlev, 1.0, fn)
    c = link_speed([Ws[0]], gamma)
    return Case("smooth", nx0, ny0, nlev, tuple(bc), gamma, c, beta, Ws, refs, steps, dx0=1.0)
