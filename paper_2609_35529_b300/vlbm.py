"""Thin ctypes binding of libvlbm.so (include/vlbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The library must be built (``paper_2609_35529_b300/build.py``)
and a CUDA device must be present; there is no CPU fallback, and a missing
library raises immediately.

PyTorch is optional plumbing: when a ``torch.cuda.Stream`` is given the
library runs on it, and ``allocator="torch"`` routes the library's device
allocations through PyTorch's caching allocator.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvlbm.so")

VLBM_MAX_LEVELS = 4
VLBM_BLOCK = 8
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_NESTING", 3: "ERR_OOM", 4: "ERR_CUDA", 5: "ERR_NONPHYSICAL",
          6: "ERR_TIMEOUT", 7: "ERR_STATE"}
BC_PERIODIC, BC_OUTFLOW, BC_INFLOW, BC_REFLECT = 0, 1, 2, 3


class VlbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class vlbm_box(C.Structure):
    _fields_ = [("level", C.c_int32), ("i0", C.c_int32), ("j0", C.c_int32), ("ni", C.c_int32), ("nj", C.c_int32)]


class vlbm_config(C.Structure):
    _fields_ = [("nx0", C.c_int32), ("ny0", C.c_int32), ("dx0", C.c_double), ("max_levels", C.c_int32),
                ("bc", C.c_int32 * 4), ("inflow_W", (C.c_double * 4) * 4), ("gamma", C.c_double),
                ("c", C.c_double), ("beta", C.c_double), ("boxes", C.POINTER(vlbm_box)), ("nboxes", C.c_int32),
                ("tag_tol", C.c_double), ("tag_buffer", C.c_int32), ("tag_sensor", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class vlbm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class vlbm_kernel_time(C.Structure):
    _fields_ = [("kind", C.c_int32), ("level", C.c_int32), ("launches", C.c_int64), ("cells", C.c_int64),
                ("ms", C.c_double)]


class vlbm_tuning(C.Structure):
    _fields_ = [("variant", C.c_int32), ("max_ctas", C.c_int32), ("graph_steps", C.c_int32), ("schedule", C.c_int32),
                ("persist_after", C.c_int64)]


class vlbm_info(C.Structure):
    _fields_ = [("nlev", C.c_int32), ("nx", C.c_int32 * 4), ("ny", C.c_int32 * 4),
                ("active_cells", C.c_int64 * 4), ("lups_per_step", C.c_int64), ("device_bytes", C.c_int64),
                ("steps", C.c_int64), ("c", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("dx0", C.c_double)]


_lib = None


def lib():
    """Loads libvlbm.so; raises when it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libvlbm.so not built ({LIB_PATH}); run paper_2609_35529_b300/build.py")
    L = C.CDLL(LIB_PATH)
    vp, dp, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
    sig = {
        "vlbm_create_hierarchy": [C.POINTER(vlbm_config), C.POINTER(vlbm_allocator), vp, C.POINTER(vp)],
        "vlbm_set_state": [vp, i32, vp, i64, i32],
        "vlbm_set_populations": [vp, i32, vp, i64, i32],
        "vlbm_get_populations": [vp, i32, vp, i64, i32],
        "vlbm_advance": [vp, i64],
        "vlbm_regrid": [vp, C.POINTER(vlbm_box), i32],
        "vlbm_regrid_masks": [vp, C.POINTER(vp)],
        "vlbm_get_layout": [vp, i32, vp, vp],
        "vlbm_get_conserved": [vp, i32, vp, i64, vp, dp, dp],
        "vlbm_audit": [vp, dp, dp],
        "vlbm_sync": [vp],
        "vlbm_get_info": [vp, C.POINTER(vlbm_info)],
        "vlbm_lups_done": [vp, C.POINTER(i64)],
        "vlbm_lups_mark": [vp, vp],
        "vlbm_kernels_launched": [vp, C.POINTER(i64)],
        "vlbm_set_regrid_audit": [vp, i32],
        "vlbm_get_regrid_audits": [vp, dp, i64, C.POINTER(i64)],
        "vlbm_host_times": [vp, dp],
        "vlbm_set_sensor": [vp, i32, C.c_double, C.c_double, C.c_double],
        "vlbm_profile": [vp, i64, C.POINTER(vlbm_kernel_time), i32, C.POINTER(i32)],
        "vlbm_set_step_totals": [vp, i32],
        "vlbm_checkpoint_size": [vp, C.POINTER(C.c_size_t)],
        "vlbm_checkpoint_save": [vp, vp, C.c_size_t],
        "vlbm_checkpoint_load": [vp, vp, C.c_size_t],
        "vlbm_get_step_totals": [vp, dp, i64, C.POINTER(i64)],
        "vlbm_engine_create": [C.c_size_t, C.POINTER(vlbm_allocator), vp, C.POINTER(vp)],
        "vlbm_engine_admit": [vp, vp, i64, i32, C.POINTER(i32)],
        "vlbm_engine_step": [vp, C.POINTER(i32), C.POINTER(i32)],
        "vlbm_engine_set_schedule": [vp, i32],
        "vlbm_engine_advance": [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)],
        "vlbm_engine_release": [vp, i32],
        "vlbm_engine_usage": [vp, C.POINTER(i32), C.POINTER(i64)],
        "vlbm_engine_host_times": [vp, dp],
        "vlbm_engine_slot_stats": [vp, i32, C.POINTER(i64), C.POINTER(i64)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.vlbm_num_variants.argtypes = []
    L.vlbm_num_variants.restype = C.c_int32
    L.vlbm_set_tuning.argtypes = [vp, C.POINTER(vlbm_tuning)]
    L.vlbm_set_tuning.restype = C.c_int
    L.vlbm_get_tuning.argtypes = [vp, C.POINTER(vlbm_tuning)]
    L.vlbm_get_tuning.restype = C.c_int
    L.vlbm_selftest_timeout.argtypes = [dp, C.POINTER(i32)]
    L.vlbm_selftest_timeout.restype = C.c_int
    L.vlbm_selftest_rcp.argtypes = [C.c_uint64, i64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), dp]
    L.vlbm_selftest_rcp.restype = C.c_int
    L.vlbm_selftest_div.argtypes = [C.c_uint64, i64, C.POINTER(C.c_uint64), dp]
    L.vlbm_selftest_div.restype = C.c_int
    L.vlbm_selftest_layout.argtypes = [C.c_uint64, i32, C.POINTER(i64), C.POINTER(i64), C.c_char_p, i32]
    L.vlbm_selftest_layout.restype = C.c_int
    L.vlbm_totals_static.argtypes = [vp, i64, i32, i32, C.c_double, vp, vp]
    L.vlbm_totals_static.restype = C.c_int
    L.vlbm_last_error.argtypes = [vp]
    L.vlbm_last_error.restype = C.c_char_p
    L.vlbm_destroy.argtypes = [vp]
    L.vlbm_destroy.restype = None
    L.vlbm_engine_destroy.argtypes = [vp]
    L.vlbm_engine_destroy.restype = None
    _lib = L
    return L


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)
        self.struct = vlbm_allocator(self.c_alloc, self.c_free, None)

    def _alloc(self, n, stream, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(n), self.dev, stream or 0)
        except Exception:
            return None

    def _free(self, p, stream, ctx):
        self.torch.cuda.caching_allocator_delete(p)


def _check(h, st):
    if st != 0:
        msg = lib().vlbm_last_error(h).decode() if h else ""
        raise VlbmError(st, msg)


class Hierarchy:
    """A refined VLBM hierarchy on the GPU (vlbm_hier)."""

    def __init__(self, nx0, ny0, nlev, bc, gamma, c, beta, boxes=(), dx0=1.0, inflow=None, tag_tol=0.0,
                 tag_buffer=0, stream=None, allocator=None, tag_sensor=0):
        L = lib()
        cfg = vlbm_config()
        cfg.nx0, cfg.ny0, cfg.dx0, cfg.max_levels = nx0, ny0, dx0, nlev
        for s in range(4):
            cfg.bc[s] = int(bc[s])
        if inflow is not None:
            for s in range(4):
                for k in range(4):
                    cfg.inflow_W[s][k] = float(inflow[s][k])
        cfg.gamma, cfg.c, cfg.beta = gamma, c, beta
        self._boxes = (vlbm_box * max(1, len(boxes)))(*[vlbm_box(*b) for b in boxes])
        cfg.boxes = self._boxes if boxes else None
        cfg.nboxes = len(boxes)
        cfg.tag_tol, cfg.tag_buffer, cfg.tag_sensor = tag_tol, tag_buffer, int(tag_sensor)
        self._alloc = _TorchAllocator() if allocator == "torch" else None
        h = C.c_void_p()
        st = L.vlbm_create_hierarchy(C.byref(cfg), C.byref(self._alloc.struct) if self._alloc else None,
                                     _stream_handle(stream), C.byref(h))
        if st != 0:
            raise VlbmError(st, "vlbm_create_hierarchy")
        self._h = h
        self.nlev = nlev
        self.shapes = [(ny0 << l, nx0 << l) for l in range(nlev)]

    @classmethod
    def from_case(cls, case, boxes=None, stream=None, allocator=None, refs=True):
        """Creates a hierarchy for an inputs.Case and loads its initial state."""
        h = cls(case.nx0, case.ny0, case.nlev, case.bc, case.gamma, case.c, case.beta, boxes=boxes or (),
                dx0=case.dx0, inflow=case.inflow, tag_tol=(case.amr or {}).get("tol", 0.0),
                tag_buffer=(case.amr or {}).get("buffer", 0), stream=stream, allocator=allocator,
                tag_sensor=(case.amr or {}).get("sensor", 0))
        if refs and case.nlev > 1 and not boxes and any(r.any() for r in case.refs):
            h.regrid_masks(case.refs)
        for l in range(case.nlev):
            h.set_state(l, case.W[l])
        return h

    # --- life cycle ---
    def close(self):
        if getattr(self, "_h", None):
            lib().vlbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # --- state ---
    def set_state(self, level, W):
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert W.shape == (4,) + self.shapes[level], W.shape
        _check(self._h, lib().vlbm_set_state(self._h, level, W.ctypes.data, W.shape[2], 0))

    def set_state_device(self, level, W_ptr, ld):
        _check(self._h, lib().vlbm_set_state(self._h, level, W_ptr, ld, 1))

    def set_populations(self, level, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (16,) + self.shapes[level]
        _check(self._h, lib().vlbm_set_populations(self._h, level, f.ctypes.data, f.shape[2], 0))

    def get_populations(self, level):
        f = np.zeros((16,) + self.shapes[level])
        _check(self._h, lib().vlbm_get_populations(self._h, level, f.ctypes.data, f.shape[2], 0))
        return f

    def advance(self, n):
        _check(self._h, lib().vlbm_advance(self._h, int(n)))

    def sync(self):
        _check(self._h, lib().vlbm_sync(self._h))

    def regrid(self, boxes=None):
        if boxes is None:
            _check(self._h, lib().vlbm_regrid(self._h, None, 0))
        else:
            arr = (vlbm_box * max(1, len(boxes)))(*[vlbm_box(*b) for b in boxes])
            _check(self._h, lib().vlbm_regrid(self._h, arr, len(boxes)))

    def regrid_masks(self, refs):
        keep = []
        arr = (C.c_void_p * self.nlev)()
        for l in range(self.nlev - 1):
            m = np.ascontiguousarray(refs[l], dtype=np.uint8)
            assert m.shape == self.shapes[l]
            keep.append(m)
            arr[l] = m.ctypes.data
        _check(self._h, lib().vlbm_regrid_masks(self._h, arr))

    def layout(self, level):
        a = np.zeros(self.shapes[level], dtype=np.uint8)
        b = np.zeros(self.shapes[level], dtype=np.uint8)
        _check(self._h, lib().vlbm_get_layout(self._h, level, a.ctypes.data, b.ctypes.data))
        return a, b

    def get_conserved(self, level, totals=False, out=None, valid=True):
        """W of every cell of `level` (shape (4, ny, nx)) and the mask of the
        cells whose W is meaningful.  `out`: a caller-owned float64 array of
        that shape to fill (C-contiguous; pinned host memory makes the copy
        run at full PCIe speed); valid=False skips the mask (returned as
        None)."""
        shape = (4,) + self.shapes[level]
        if out is None:
            W = np.zeros(shape)
        else:
            W = out
            if W.shape != shape or W.dtype != np.float64 or not W.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a C-contiguous float64 array of shape %s" % (shape,))
        v = np.zeros(self.shapes[level], dtype=np.uint8) if valid else None
        t = (C.c_double * 4)()
        a = (C.c_double * 4)()
        _check(self._h, lib().vlbm_get_conserved(self._h, level, W.ctypes.data, W.shape[2],
                                                 v.ctypes.data if valid else None,
                                                 t if totals else None, a if totals else None))
        vm = v.astype(bool) if valid else None
        if totals:
            return W, vm, np.array(t[:]), np.array(a[:])
        return W, vm

    def audit(self):
        t = (C.c_double * 4)()
        a = (C.c_double * 4)()
        _check(self._h, lib().vlbm_audit(self._h, t, a))
        return np.array(t[:]), np.array(a[:])

    def info(self):
        i = vlbm_info()
        _check(self._h, lib().vlbm_get_info(self._h, C.byref(i)))
        return {"nlev": i.nlev, "nx": list(i.nx[: i.nlev]), "ny": list(i.ny[: i.nlev]),
                "active_cells": list(i.active_cells[: i.nlev]), "lups_per_step": i.lups_per_step,
                "device_bytes": i.device_bytes, "steps": i.steps, "c": i.c, "beta": i.beta}

    def lups_done(self):
        """Cell updates done since creation, counted on the device at the
        layout each step ran on (vlbm_lups_done; synchronises)."""
        v = C.c_int64()
        _check(self._h, lib().vlbm_lups_done(self._h, C.byref(v)))
        return int(v.value)

    def kernels_launched(self):
        """Kernels the library has queued for this hierarchy so far."""
        v = C.c_int64()
        _check(self._h, lib().vlbm_kernels_launched(self._h, C.byref(v)))
        return int(v.value)

    def lups_mark(self, dst_ptr):
        """Queues a copy of the cell-update counter into host memory at
        dst_ptr (an int64; pinned for a truly asynchronous copy)."""
        _check(self._h, lib().vlbm_lups_mark(self._h, C.c_void_p(dst_ptr)))

    def set_regrid_audit(self, on=True):
        """Record exact totals before and after every device regrid."""
        _check(self._h, lib().vlbm_set_regrid_audit(self._h, int(on)))

    def regrid_audits(self, cap=4096):
        """Rows recorded since the last read: [n, 16] = totals, |W| totals
        before the regrid, then after (synchronises)."""
        out = np.zeros((cap, 16))
        n = C.c_int64()
        _check(self._h, lib().vlbm_get_regrid_audits(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                                     C.byref(n)))
        return out[: n.value]

    def set_sensor(self, on=True, beta_min=0.5, c_sensor=16.0, eps=1e-30):
        """Sensor-driven relaxation (vlbm_set_sensor): beta_max is the
        hierarchy's beta; the flux maxima are fixed from the current state."""
        _check(self._h, lib().vlbm_set_sensor(self._h, int(on), beta_min, c_sensor, eps))
        self.sensor_on = bool(on)

    HOST_TIMERS = ("tag", "layout", "regrid", "build", "tasks", "capture", "regrids", "task_lists")

    def host_times(self):
        """Cumulative host-side milliseconds by activity and the regrid and
        task-list counts (vlbm_host_times)."""
        out = (C.c_double * len(self.HOST_TIMERS))()
        _check(self._h, lib().vlbm_host_times(self._h, out))
        return dict(zip(self.HOST_TIMERS, out[:]))

    def profile(self, steps):
        """Per-kernel device times over `steps` eagerly launched coarse steps:
        list of dicts (kind: sweep/close/end_step, level, launches, cells, ms)."""
        recs = (vlbm_kernel_time * 16)()
        n = C.c_int32()
        _check(self._h, lib().vlbm_profile(self._h, int(steps), recs, 16, C.byref(n)))
        kinds = {0: "sweep", 1: "close", 2: "end_step"}
        return [{"kind": kinds[r.kind], "level": r.level, "launches": r.launches, "cells": r.cells, "ms": r.ms}
                for r in recs[: n.value]]

    def checkpoint(self):
        """The hierarchy's state as a bytes blob (vlbm_checkpoint_save)."""
        n = C.c_size_t()
        _check(self._h, lib().vlbm_checkpoint_size(self._h, C.byref(n)))
        buf = (C.c_char * n.value)()
        _check(self._h, lib().vlbm_checkpoint_save(self._h, buf, n.value))
        return bytes(buf)

    def restore(self, blob):
        """Resumes from a blob made by checkpoint() under the same configuration."""
        buf = C.create_string_buffer(blob, len(blob))
        _check(self._h, lib().vlbm_checkpoint_load(self._h, buf, len(blob)))

    def set_step_totals(self, on=True):
        _check(self._h, lib().vlbm_set_step_totals(self._h, 1 if on else 0))

    def step_totals(self, cap=4096):
        """Per-step totals recorded since the last call: array [n, 8]
        (sum W_k, then sum |W_k|, of the state at the start of each step)."""
        out = np.zeros((cap, 8))
        n = C.c_int64()
        _check(self._h, lib().vlbm_get_step_totals(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), cap,
                                                   C.byref(n)))
        return out[: n.value]

    def set_tuning(self, variant=1, max_ctas=0, graph_steps=8, schedule=1, persist_after=2):
        """schedule: 0 per-phase launches, 1 persistent task kernel, 2 auto
        (per-phase until the layout has lived persist_after coarse steps)."""
        t = vlbm_tuning(variant, max_ctas, graph_steps, schedule, persist_after)
        _check(self._h, lib().vlbm_set_tuning(self._h, C.byref(t)))

    def get_tuning(self):
        t = vlbm_tuning()
        _check(self._h, lib().vlbm_get_tuning(self._h, C.byref(t)))
        return {"variant": t.variant, "max_ctas": t.max_ctas, "graph_steps": t.graph_steps, "schedule": t.schedule,
                "persist_after": t.persist_after}

    def last_error(self):
        return lib().vlbm_last_error(self._h).decode()


def totals_static(f_ptr, ld, nx, ny, weight, out_ptr, stream=None):
    """vlbm_totals_static: conservation totals of a caller-owned device
    population array [16][ny][ld] into a caller-owned device array of 8
    doubles, with no device allocation (for callers that cannot allocate)."""
    st = lib().vlbm_totals_static(f_ptr, int(ld), int(nx), int(ny), float(weight), out_ptr, _stream_handle(stream))
    if st != 0:
        raise VlbmError(st, "vlbm_totals_static")


def num_variants():
    return lib().vlbm_num_variants()


def selftest_rcp(seed, n):
    """Bitwise check of the integer-pipe reciprocal against the FP64
    division on n seeded values; returns (mismatches, inputs whose exact
    correction did not settle, first offending (x, result))."""
    bad = C.c_uint64()
    uns = C.c_uint64()
    first = (C.c_double * 2)()
    st = lib().vlbm_selftest_rcp(int(seed), int(n), C.byref(bad), C.byref(uns), first)
    if st != 0:
        raise VlbmError(st, "vlbm_selftest_rcp")
    return int(bad.value), int(uns.value), tuple(first)


def selftest_div(seed, n):
    """Bitwise check of the sensor's division (integer-pipe reciprocal and
    two remainder corrections) against the FP64 division on n seeded pairs;
    returns (mismatches, first offending (a, b, result))."""
    bad = C.c_uint64()
    first = (C.c_double * 3)()
    st = lib().vlbm_selftest_div(int(seed), int(n), C.byref(bad), first)
    if st != 0:
        raise VlbmError(st, "vlbm_selftest_div")
    return int(bad.value), tuple(first)


def selftest_layout(seed, cases):
    """Device-resident layouts against the host's layout rule, tile lists and
    task builder on seeded random hierarchies; returns (mismatches, tasks
    stored in the overflow area, first difference)."""
    bad = C.c_int64()
    big = C.c_int64()
    buf = C.create_string_buffer(512)
    st = lib().vlbm_selftest_layout(int(seed), int(cases), C.byref(bad), C.byref(big), buf, 512)
    if st != 0:
        raise VlbmError(st, "vlbm_selftest_layout")
    return int(bad.value), int(big.value), buf.value.decode()


def selftest_timeout():
    """Bounded-wait self-test of the persistent kernel: returns (status code,
    kernel milliseconds, raw status bits); the expected status is
    VLBM_ERR_TIMEOUT (the wait on a mark nothing sets gives up)."""
    ms = C.c_double()
    word = C.c_int32()
    st = lib().vlbm_selftest_timeout(C.byref(ms), C.byref(word))
    return st, ms.value, word.value


class Engine:
    """Continuous-batching engine (vlbm_engine): each call advances every
    resident hierarchy by the same coarse steps, on per-phase launches shared
    by all residents (schedule 0) or in one persistent launch over their
    device-built task lists merged phase-major (schedule 1)."""

    def __init__(self, mem_budget=0, stream=None, allocator=None, schedule=0):
        """allocator="torch" routes the engine's own device memory (its launch
        tables) through torch's caching allocator."""
        e = C.c_void_p()
        self._alloc = _TorchAllocator() if allocator == "torch" else None
        st = lib().vlbm_engine_create(int(mem_budget), C.byref(self._alloc.struct) if self._alloc else None,
                                      _stream_handle(stream), C.byref(e))
        if st != 0:
            raise VlbmError(st, "vlbm_engine_create")
        self._e = e
        self.cap = 0
        self.set_schedule(schedule)

    def set_schedule(self, schedule):
        """0: per-phase launches; 1: one persistent launch per call (phase-major)."""
        st = lib().vlbm_engine_set_schedule(self._e, int(schedule))
        if st != 0:
            raise VlbmError(st, "vlbm_engine_set_schedule")

    def admit(self, hier, steps, regrid_every=0):
        slot = C.c_int32()
        st = lib().vlbm_engine_admit(self._e, hier.handle, int(steps), int(regrid_every), C.byref(slot))
        if st == 3:
            return None  # not admitted now (memory budget)
        if st != 0:
            raise VlbmError(st, "vlbm_engine_admit")
        self.cap = max(self.cap, slot.value + 1)
        return slot.value

    def step(self):
        buf = (C.c_int32 * max(1, self.cap))()
        n = C.c_int32()
        st = lib().vlbm_engine_step(self._e, buf, C.byref(n))
        if st != 0:
            raise VlbmError(st, "vlbm_engine_step")
        return [buf[i] for i in range(n.value)]

    def advance(self, max_steps):
        """Up to max_steps coarse steps of every resident (see
        vlbm_engine_advance): (finished slots, steps taken)."""
        buf = (C.c_int32 * max(1, self.cap))()
        n = C.c_int32()
        k = C.c_int32()
        st = lib().vlbm_engine_advance(self._e, int(max_steps), buf, C.byref(n), C.byref(k))
        if st != 0:
            raise VlbmError(st, "vlbm_engine_advance")
        return [buf[i] for i in range(n.value)], k.value

    def release(self, slot):
        st = lib().vlbm_engine_release(self._e, int(slot))
        if st != 0:
            raise VlbmError(st, "vlbm_engine_release")

    def slot_stats(self, slot):
        """(coarse steps done, cell updates done) of a resident."""
        a, b = C.c_int64(), C.c_int64()
        st = lib().vlbm_engine_slot_stats(self._e, int(slot), C.byref(a), C.byref(b))
        if st != 0:
            raise VlbmError(st, "vlbm_engine_slot_stats")
        return a.value, b.value

    def usage(self):
        n = C.c_int32()
        b = C.c_int64()
        lib().vlbm_engine_usage(self._e, C.byref(n), C.byref(b))
        return n.value, b.value

    def host_times(self):
        """Host milliseconds of the engine's calls by activity, and the call
        and step counts (vlbm_engine_host_times)."""
        out = (C.c_double * 8)()
        st = lib().vlbm_engine_host_times(self._e, out)
        if st != 0:
            raise VlbmError(st, "vlbm_engine_host_times")
        names = ["regrid_finish", "finish", "rebuild", "launch", "lead", "regrid_begin", "calls", "steps"]
        return {k: out[i] for i, k in enumerate(names)}

    def close(self):
        if getattr(self, "_e", None):
            lib().vlbm_engine_destroy(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
