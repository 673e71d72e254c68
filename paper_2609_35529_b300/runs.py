"""End-to-end runs of the paper's 2-D workloads on the GPU, with the checks
each one is about.  One JSON line per run on stdout.

  python -m paper_2609_35529_b300.runs [pulse] [vortex] [riemann] [riemann_sensor]
                                      [shockbubble[=steps,every,schedule,nx0]]

pulse        two-level Gaussian pulse, periodic 64^2, 200 coarse steps:
             per-step conservation (fused audit) and the uniform-state run
vortex       advected isentropic vortex, N = 128, 256, 512 with a central
             ratio-2 patch, one period (t = 10): L2 error of rho and |u|
             against the exact solution at the final time, the observed
             order, and the same for uniform grids of N and 2N
riemann      Lax-Liu configuration 3, 1024^2, three levels, t = 0.3:
             throughput, x<->y symmetry of the result (bitwise)
riemann_sensor[=N,levels,beta_max_permille,C]  the same with the sensor-driven
             relaxation (beta between 0.5 and beta_max)
shockbubble  adaptive shock-bubble, nx0 x nx0/2 (default 2048 x 1024), up to
             three levels, regrid every 4 coarse steps on the device, 4000
             steps on the persistent schedule (default): conservation audited
             exactly across every regrid, throughput including regrids
"""
import json
import math
import sys
import time

import numpy as np

from . import autotune
from . import inputs as I
from . import vlbm as V


def now():
    return time.perf_counter()


def emit(d):
    print(json.dumps(d), flush=True)


def run_pulse():
    cs = I.pulse2l()
    h = V.Hierarchy.from_case(cs)
    h.set_step_totals(True)
    t0 = now()
    h.advance(cs.steps)
    rows = h.step_totals()
    el = now() - t0
    drift = np.abs(rows[:, :4] - rows[0, :4]) / rows[0, 4:]
    # uniform state through the interface
    u = I.pulse2l(amp=0.0)
    hu = V.Hierarchy.from_case(u)
    hu.advance(u.steps)
    dev = 0.0
    for l in range(u.nlev):
        W, act = hu.get_conserved(l)
        for k in range(4):
            ref = u.W[0][k, 0, 0]
            dev = max(dev, float(np.max(np.abs(W[k][act] - ref))) / max(abs(ref), 1.0))
    emit({"run": "pulse2l", "steps": cs.steps, "lups_per_step": h.info()["lups_per_step"],
          "wall_s": el, "max_rel_drift_per_step": float(drift.max()),
          "uniform_state_max_dev": dev})


def l2_errors(h, case, exact_levels):
    """L2 norms (over the domain, finest data at each point) of the error in
    rho and |u| against the exact state on each level's cell centres."""
    e_rho = e_u = 0.0
    dx0 = case.dx0
    for l in range(case.nlev):
        W, act = h.get_conserved(l)
        Ex = exact_levels[l]
        a = dx0 / 2 ** l
        e_rho += float(np.sum((W[0][act] - Ex[0][act]) ** 2)) * a * a
        sp = np.hypot(W[1][act] / W[0][act], W[2][act] / W[0][act])  # W is meaningful on `act` only
        se = np.hypot(Ex[1][act] / Ex[0][act], Ex[2][act] / Ex[0][act])
        e_u += float(np.sum((sp - se) ** 2)) * a * a
    return math.sqrt(e_rho), math.sqrt(e_u)


def vortex_exact(cs):
    """The exact solution at the end of the run, t_end = steps * dt: the
    initial vortex carried by the free stream (1, 1) over t_end, periodically.
    The step count is t = 10 / dt rounded, so t_end differs from one period by
    up to dt / 2; comparing with the initial state instead would add an error
    of order dt * |grad W| that does not converge at second order."""
    t_end = cs.steps * cs.dx0 / cs.c
    xc = (5.0 + t_end) % 10.0
    return I.fill_levels(cs.nx0, cs.ny0, cs.nlev, cs.dx0,
                         lambda X, Y: I.vortex_state(X, Y, xc=xc, yc=xc, gamma=cs.gamma))


def run_vortex():
    res = {}
    for patch in (True, False):
        for N in (128, 256, 512):
            cs = I.vortex(N=N, patch=patch)
            h = V.Hierarchy.from_case(cs)
            h.set_step_totals(True)
            t0 = now()
            h.advance(cs.steps)
            rows = h.step_totals()
            el = now() - t0
            er, eu = l2_errors(h, cs, vortex_exact(cs))
            drift = float((np.abs(rows[:, :4] - rows[0, :4]) / rows[0, 4:]).max())
            res[(patch, N)] = (er, eu)
            emit({"run": "vortex", "N": N, "patch": patch, "steps": cs.steps, "t_end": cs.steps * cs.dx0 / cs.c,
                  "lups_per_step": h.info()["lups_per_step"], "wall_s": el,
                  "mlups": h.info()["lups_per_step"] * cs.steps / el / 1e6,
                  "l2_rho": er, "l2_speed": eu, "max_rel_drift_per_step": drift})
            h.close()
    for patch in (True, False):
        e = [res[(patch, N)] for N in (128, 256, 512)]
        emit({"run": "vortex-order", "patch": patch,
              "order_rho": [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)],
              "order_speed": [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]})
    # a uniform grid at twice the base resolution, for the refined runs' comparison
    for N in (256, 512, 1024):
        cs = I.vortex(N=N, patch=False)
        h = V.Hierarchy.from_case(cs)
        t0 = now()
        h.advance(cs.steps)
        h.sync()
        el = now() - t0
        er, eu = l2_errors(h, cs, vortex_exact(cs))
        emit({"run": "vortex-uniform-2N", "N": N, "steps": cs.steps, "wall_s": el,
              "mlups": h.info()["lups_per_step"] * cs.steps / el / 1e6, "l2_rho": er, "l2_speed": eu})
        h.close()


def run_riemann():
    cs = I.riemann3(N=1024, nlev=3)
    h = V.Hierarchy.from_case(cs)
    lups = h.info()["lups_per_step"]
    h.advance(8)
    h.sync()
    t0 = now()
    h.advance(cs.steps - 8)
    h.sync()
    el = now() - t0
    sym = True
    for l in range(cs.nlev):
        f = h.get_populations(l).reshape(4, 4, *h.shapes[l])
        a, b = h.layout(l)
        act = (a == 1) & (b == 0)
        ft = f.transpose(0, 1, 3, 2)[[2, 3, 0, 1]][:, [0, 2, 1, 3]]
        sym = sym and bool(np.array_equal(f[:, :, act], ft[:, :, act]))
    W, act = h.get_conserved(0)
    info = h.info()
    emit({"run": "riemann3", "N": 1024, "levels": 3, "steps": cs.steps, "t_end": cs.steps * cs.dx0 / cs.c,
          "active_cells": info["active_cells"], "lups_per_step": lups, "wall_s": el,
          "mlups": lups * (cs.steps - 8) / el / 1e6, "transpose_symmetric_bitwise": sym,
          "rho_min": float(W[0][act].min()), "rho_max": float(W[0][act].max())})


def run_riemann_sensor(N=1024, nlev=3, beta_max_permille=1000, c_sensor=64):
    """Lax-Liu 3 with the sensor-driven relaxation (beta between 0.5 and
    beta_max, gain C): constant beta = 0.9 or 1 loses positivity on this
    problem; the sensor lowers beta only at compressions."""
    bmax = beta_max_permille / 1000.0
    cs = I.riemann3(N=N, nlev=nlev, beta=bmax)

    def make():
        g = V.Hierarchy.from_case(cs)
        g.set_sensor(True, beta_min=0.5, c_sensor=float(c_sensor))
        return g

    h = make()
    best, _ = autotune.tune(make, target=h, steps=32, candidates=autotune.SENSOR_CANDIDATES)
    lups = h.info()["lups_per_step"]
    h.advance(4)
    h.sync()
    t0 = now()
    done = 4
    try:
        while done < cs.steps:
            n = min(100, cs.steps - done)
            h.advance(n)
            h.sync()
            done += n
    except V.VlbmError as err:
        emit({"run": "riemann3-sensor", "N": N, "levels": nlev, "beta": [0.5, bmax], "c_sensor": c_sensor,
              "physical_to_end": False, "failed_by_step": done + 100, "error": str(err)})
        return
    el = now() - t0
    W, act = h.get_conserved(0)
    p = 0.4 * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])
    sym = True
    for l in range(cs.nlev):
        f = h.get_populations(l).reshape(4, 4, *h.shapes[l])
        a, b = h.layout(l)
        act_l = (a == 1) & (b == 0)
        ft = f.transpose(0, 1, 3, 2)[[2, 3, 0, 1]][:, [0, 2, 1, 3]]
        sym = sym and bool(np.array_equal(f[:, :, act_l], ft[:, :, act_l]))
    emit({"run": "riemann3-sensor", "N": N, "levels": nlev, "steps": cs.steps, "lups_per_step": lups, "tuning": best,
          "wall_s": el, "mlups": lups * (cs.steps - 4) / el / 1e6, "transpose_symmetric_bitwise": sym,
          "rho_min": float(W[0][act].min()), "rho_max": float(W[0][act].max()), "p_min": float(p[act].min()),
          "beta": [0.5, bmax], "c_sensor": c_sensor, "physical_to_end": True})


def run_shockbubble(steps=4000, every=4, schedule=1, nx0=2048):
    """The adaptive run (nx0 x nx0/2 coarse cells, three levels, a regrid
    every `every` coarse steps, all on the device); the totals are audited
    exactly before and after every regrid, on the device, and read back at
    the end."""
    cs = I.shockbubble(nx0=nx0, ny0=nx0 // 2, steps=steps)
    h = V.Hierarchy.from_case(cs)
    h.set_tuning(schedule=schedule, graph_steps=every, persist_after=0)
    for _ in range(cs.nlev - 1):
        h.regrid()
    h.set_regrid_audit(True)
    start = h.lups_done()
    per_step0 = h.info()["lups_per_step"]
    t0 = now()
    done = 0
    while done < steps:
        n = min(every, steps - done)
        h.advance(n)
        done += n
        if done < steps:
            h.regrid()
    h.sync()
    el = now() - t0
    rows = h.regrid_audits()
    worst = 0.0
    if len(rows):
        d = np.abs(rows[:, 8:12] - rows[:, 0:4])
        a = rows[:, 4:8]
        worst = float(np.max(np.where(a > 0, d / np.where(a > 0, a, 1), d)))
    emit({"run": "shockbubble", "coarse": [cs.nx0, cs.ny0], "levels": cs.nlev, "steps": steps, "schedule": schedule,
          "regrids": (steps - 1) // every, "wall_s": el, "mlups_incl_regrid": (h.lups_done() - start) / el / 1e6,
          "max_rel_change_across_regrid": worst, "lups_per_step_at_start": per_step0,
          "active_cells_at_end": h.info()["active_cells"],
          "host_ms": h.host_times()})
    h.close()


def main(argv=None):
    which = (argv if argv is not None else sys.argv[1:]) or ["pulse", "vortex", "riemann", "shockbubble"]
    for w in which:
        name, _, arg = w.partition("=")
        fn = {"pulse": run_pulse, "vortex": run_vortex, "riemann": run_riemann, "riemann_sensor": run_riemann_sensor,
              "shockbubble": run_shockbubble}[name]
        fn(*[int(a) for a in arg.split(",")]) if arg else fn()


if __name__ == "__main__":
    main()
