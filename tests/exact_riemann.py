"""Exact solution of the 1-D Riemann problem for an ideal gas.

Textbook construction (Godunov's exact solver): the star pressure is the root
of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-
Hugoniot) branch for p > p_K and the rarefaction (isentropic) branch for
p <= p_K; the solution is then sampled along x/t.  Used only as a test
reference for the oracle (Sod tube, Sec. 4.1.2).
"""
import math

import numpy as np


def _fk(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    r = (p / pk) ** e
    return 2.0 * a / (gamma - 1.0) * (r - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * a)


def star(left, right, gamma=1.4, tol=1e-14):
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, gamma)
        fr, dr = _fk(p, rr, pr, gamma)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, gamma)
    fr, _ = _fk(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, gamma=1.4):
    """(rho, u, p) at similarity coordinates xi = x/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            al = math.sqrt(gamma * pl / rl)
            if ps > pl:  # left shock
                sl = ul - al * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                if s <= sl:
                    out[:, n] = (rl, ul, pl)
                else:
                    out[:, n] = (rl * (ps / pl + g1) / (g1 * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                ast = al * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s <= ul - al:
                    out[:, n] = (rl, ul, pl)
                elif s >= us - ast:
                    out[:, n] = (rl * (ps / pl) ** (1 / gamma), us, ps)
                else:
                    u = 2 / (gamma + 1) * (al + (gamma - 1) / 2 * ul + s)
                    c = 2 / (gamma + 1) * (al + (gamma - 1) / 2 * (ul - s))
                    rho = rl * (c / al) ** (2 / (gamma - 1))
                    out[:, n] = (rho, u, pl * (c / al) ** (2 * gamma / (gamma - 1)))
        else:
            ar = math.sqrt(gamma * pr / rr)
            if ps > pr:  # right shock
                sr = ur + ar * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                if s >= sr:
                    out[:, n] = (rr, ur, pr)
                else:
                    out[:, n] = (rr * (ps / pr + g1) / (g1 * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                ast = ar * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s >= ur + ar:
                    out[:, n] = (rr, ur, pr)
                elif s <= us + ast:
                    out[:, n] = (rr * (ps / pr) ** (1 / gamma), us, ps)
                else:
                    u = 2 / (gamma + 1) * (-ar + (gamma - 1) / 2 * ur + s)
                    c = 2 / (gamma + 1) * (ar - (gamma - 1) / 2 * (ur - s))
                    rho = rr * (c / ar) ** (2 / (gamma - 1))
                    out[:, n] = (rho, u, pr * (c / ar) ** (2 * gamma / (gamma - 1)))
    return out
