"""ORACLE -- test infrastructure, not product code.

ctypes wrapper around liboracle.so, the plain FP64 C rendering of the
conservative locally refined VLBM (Hosseini, Strassle & Karlin).  Only the
test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this module.  It shares no code with the CUDA path;
the only thing both sides consume is the input recipes of
``paper_2609_35529_b300.inputs`` (initial states and layouts, no method
arithmetic).

Every array is numpy, C order, x fastest: per-level populations are
``f[16, ny, nx]`` with population index ``q = 4*i + k`` (direction i in
+x, -x, +y, -y; field k in rho, rho*u, rho*v, rho*E); conserved fields are
``W[4, ny, nx]``; refinement masks are ``uint8[ny, nx]`` on the level they
refine.
"""
import ctypes as C
import os

import numpy as np

from . import build_oracle

BC_PERIODIC, BC_OUTFLOW, BC_INFLOW, BC_REFLECT = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.ora_create.restype = C.c_void_p
        L.ora_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), dp,
                                 C.c_double, C.c_double, C.c_double]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_set_layout.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
        L.ora_set_layout.restype = C.c_int
        L.ora_set_state.argtypes = [C.c_void_p, C.c_int, dp]
        L.ora_set_f.argtypes = [C.c_void_p, C.c_int, dp]
        L.ora_get_f.argtypes = [C.c_void_p, C.c_int, dp]
        L.ora_get_W.argtypes = [C.c_void_p, C.c_int, dp, C.c_void_p]
        L.ora_get_layout.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.ora_advance.argtypes = [C.c_void_p, C.c_int]
        L.ora_regrid.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
        L.ora_regrid.restype = C.c_int
        L.ora_regrid_tagged.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.ora_regrid_tagged.restype = C.c_int
        L.ora_layout_from_tags.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                                           C.POINTER(C.c_void_p)]
        L.ora_tags.argtypes = [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_void_p)]
        L.ora_flux_max.argtypes = [C.c_void_p, dp]
        L.ora_set_sensor.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double]
        L.ora_sensor_beta.argtypes = [C.c_void_p, C.c_int, dp]
        L.ora_feq.argtypes = [C.c_double, C.c_double, dp, dp]
        L.ora_collide.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
        L.ora_minmod.argtypes = [C.c_double, C.c_double]
        L.ora_minmod.restype = C.c_double
        L.ora_recon.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int]
        L.ora_recon.restype = C.c_double
        L.ora_merge4.argtypes = [C.c_double] * 4
        L.ora_merge4.restype = C.c_double
        L.ora_split_child.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int]
        L.ora_split_child.restype = C.c_double
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---- single-cell operators (Sec. 2.2, Sec. 3.3, Sec. 3.4) ----

def feq(gamma, c, W):
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(16)
    lib().ora_feq(gamma, c, _dp(W), _dp(out))
    return out


def collide(gamma, c, beta, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(16)
    lib().ora_collide(gamma, c, beta, _dp(f), _dp(out))
    return out


def minmod(a, b):
    return lib().ora_minmod(a, b)


def recon(a, a_prev, sigma, r, k, j):
    return lib().ora_recon(a, a_prev, sigma, r, k, j)


def merge4(c00, c10, c01, c11):
    return lib().ora_merge4(c00, c10, c01, c11)


def split_child(fc, sx, sy, r, a, b):
    return lib().ora_split_child(fc, sx, sy, r, a, b)


class Hierarchy:
    """An oracle hierarchy: levels 0..nlev-1 at refinement ratio r."""

    def __init__(self, nx0, ny0, nlev, r, bc, gamma, c, beta, inflow=None):
        self.nx0, self.ny0, self.nlev, self.r = nx0, ny0, nlev, r
        self.shapes = [(ny0 * r ** l, nx0 * r ** l) for l in range(nlev)]
        bcs = (C.c_int * 4)(*bc)
        wb = np.zeros((4, 4)) if inflow is None else np.ascontiguousarray(inflow, dtype=np.float64)
        self._h = lib().ora_create(nx0, ny0, nlev, r, bcs, _dp(wb), gamma, c, beta)
        if not self._h:
            raise ValueError("oracle: invalid hierarchy arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_destroy(h)
            self._h = None

    def _masks(self, refs):
        keep = []
        arr = (C.c_void_p * self.nlev)()
        for l in range(self.nlev):
            if l < self.nlev - 1 and refs is not None and refs[l] is not None:
                m = np.ascontiguousarray(refs[l], dtype=np.uint8)
                assert m.shape == self.shapes[l]
            else:
                m = np.zeros(self.shapes[l], dtype=np.uint8)
            keep.append(m)
            arr[l] = m.ctypes.data
        return arr, keep

    def set_layout(self, refs):
        arr, keep = self._masks(refs)
        err = lib().ora_set_layout(self._h, arr)
        if err:
            raise ValueError(f"oracle: layout not nested (code {err})")

    def set_state(self, l, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (4,) + self.shapes[l]
        lib().ora_set_state(self._h, l, _dp(W))

    def set_f(self, l, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (16,) + self.shapes[l]
        lib().ora_set_f(self._h, l, _dp(f))

    def get_f(self, l):
        f = np.zeros((16,) + self.shapes[l])
        lib().ora_get_f(self._h, l, _dp(f))
        return f

    def get_W(self, l):
        """Returns (W[4,ny,nx], flags) with flags bit0 = on level, bit1 = covered."""
        W = np.zeros((4,) + self.shapes[l])
        fl = np.zeros(self.shapes[l], dtype=np.uint8)
        lib().ora_get_W(self._h, l, _dp(W), fl.ctypes.data)
        return W, fl

    def layout(self, l):
        a = np.zeros(self.shapes[l], dtype=np.uint8)
        b = np.zeros(self.shapes[l], dtype=np.uint8)
        lib().ora_get_layout(self._h, l, a.ctypes.data, b.ctypes.data)
        return a, b

    def advance(self, nsteps):
        lib().ora_advance(self._h, int(nsteps))

    def regrid(self, refs):
        arr, keep = self._masks(refs)
        err = lib().ora_regrid(self._h, arr)
        if err:
            raise ValueError(f"oracle: layout not nested (code {err})")

    def regrid_tagged(self, tol, buffer, block, sensor=0):
        """Tag-driven regrid; sensor 0 = normalised density gradient, 1 =
        flux jump with max norm (Sec. 3.4)."""
        outs = [np.zeros(s, dtype=np.uint8) for s in self.shapes]
        arr = (C.c_void_p * self.nlev)(*[o.ctypes.data for o in outs])
        err = lib().ora_regrid_tagged(self._h, int(sensor), tol, buffer, block, arr)
        if err:
            raise ValueError(f"oracle: regrid failed (code {err})")
        return outs[: self.nlev - 1]

    def tags(self, tol, sensor=0):
        outs = [np.zeros(s, dtype=np.uint8) for s in self.shapes]
        arr = (C.c_void_p * self.nlev)(*[o.ctypes.data for o in outs])
        lib().ora_tags(self._h, int(sensor), tol, arr)
        return outs[: self.nlev - 1]

    def set_sensor(self, on=True, beta_min=0.5, c_sensor=1.0, eps=1e-30):
        """Sensor-driven relaxation (Sec. 2.2): beta_max is the hierarchy's
        beta; the flux maxima are fixed from the current state."""
        lib().ora_set_sensor(self._h, int(on), beta_min, c_sensor, eps)

    def sensor_beta(self, level):
        out = np.zeros(self.shapes[level])
        lib().ora_sensor_beta(self._h, level, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def flux_max(self):
        q = (C.c_double * 4)()
        lib().ora_flux_max(self._h, q)
        return np.array(q[:])

    def layout_from_tags(self, tags, buffer, block):
        tg = [np.ascontiguousarray(t, dtype=np.uint8) for t in tags] + \
             [np.zeros(s, dtype=np.uint8) for s in self.shapes[len(tags):]]
        outs = [np.zeros(s, dtype=np.uint8) for s in self.shapes]
        a = (C.c_void_p * self.nlev)(*[t.ctypes.data for t in tg])
        b = (C.c_void_p * self.nlev)(*[o.ctypes.data for o in outs])
        lib().ora_layout_from_tags(self._h, a, buffer, block, b)
        return outs[: self.nlev - 1]

    # ---- diagnostics ----

    def active_masks(self):
        out = []
        for l in range(self.nlev):
            a, b = self.layout(l)
            out.append((a == 1) & (b == 0))
        return out

    def totals(self):
        """Exact (math.fsum) totals of sum_l 4^-l sum_active W_k, and of |W_k|."""
        import math
        tot = [[] for _ in range(4)]
        ab = [[] for _ in range(4)]
        for l in range(self.nlev):
            W, fl = self.get_W(l)
            act = fl == 1
            s = 0.25 ** l if self.r == 2 else (1.0 / self.r ** 2) ** l
            for k in range(4):
                v = W[k][act] * s
                tot[k].append(v)
                ab[k].append(np.abs(v))
        return (np.array([math.fsum(np.concatenate(t)) for t in tot]),
                np.array([math.fsum(np.concatenate(t)) for t in ab]))
