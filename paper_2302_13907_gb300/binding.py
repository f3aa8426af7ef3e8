"""Thin ctypes binding of the C-ABI in include/cwell.h (argument marshalling only).

Every step of the simulation runs in libcwell.so's CUDA kernels; this module
only converts numpy arrays and workload objects into the C structs and back.
Importing it loads the library and raises if it is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_EUNSTABLE, SIM_ETIMEOUT, SIM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
FIELDS = ("vr", "vp", "vz", "srr", "spp", "szz", "srp", "spz", "srz")
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
KERNEL = {"auto": 0, "split": 1, "fused": 2}


class SimGrid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("nth", ctypes.c_int), ("nz", ctypes.c_int), ("pml_r", ctypes.c_int),
                ("pml_z", ctypes.c_int), ("dr", ctypes.c_double), ("dz", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double)]


class SimMedium(ctypes.Structure):
    _fields_ = [("n_mat", ctypes.c_int), ("rho", ctypes.POINTER(ctypes.c_double)),
                ("vp", ctypes.POINTER(ctypes.c_double)), ("vs", ctypes.POINTER(ctypes.c_double)),
                ("cell_id", ctypes.c_void_p)]


class SimSource(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("r", ctypes.c_double), ("theta", ctypes.c_double), ("z", ctypes.c_double),
                ("f0", ctypes.c_double), ("amplitude", ctypes.c_double)]


class SimReceivers(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("r", ctypes.POINTER(ctypes.c_double)), ("theta", ctypes.POINTER(ctypes.c_double)),
                ("z", ctypes.POINTER(ctypes.c_double)), ("quantity", ctypes.c_int)]


class SimOpts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("pml_off", ctypes.c_int), ("graph_chunk", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("mem_cap", ctypes.c_size_t), ("max_steps", ctypes.c_int),
                ("kernel", ctypes.c_int), ("timing", ctypes.c_int), ("device", ctypes.c_int)]


_lib = None


def lib(path: str | None = None):
    """Load libcwell.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        path = path or os.environ.get("CWELL_LIB") or _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libcwell.so not found at {path}: build it with paper_2302_13907_gb300.build")
        L = ctypes.CDLL(path)
        p, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        L.sim_create.argtypes = [ctypes.POINTER(SimGrid), ctypes.POINTER(SimMedium), ctypes.POINTER(SimSource),
                                 ctypes.POINTER(SimReceivers), ctypes.POINTER(SimOpts), ctypes.POINTER(p)]
        L.sim_create.restype = i
        L.sim_step.argtypes = [p, i]
        L.sim_step.restype = i
        L.sim_sync.argtypes = [p]
        L.sim_sync.restype = i
        L.sim_traces.argtypes = [p, ctypes.POINTER(ctypes.c_float), sz, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.sim_traces.restype = i
        L.sim_read_field.argtypes = [p, i, ctypes.POINTER(ctypes.c_float), sz]
        L.sim_read_field.restype = i
        L.sim_write_field.argtypes = [p, i, ctypes.POINTER(ctypes.c_float), sz]
        L.sim_write_field.restype = i
        L.sim_dt.argtypes = [p]
        L.sim_dt.restype = d
        L.sim_steps_done.argtypes = [p]
        L.sim_steps_done.restype = i
        L.sim_device_bytes.argtypes = [p]
        L.sim_device_bytes.restype = sz
        L.sim_config.argtypes = [p, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.sim_config.restype = i
        L.sim_kernel_time.argtypes = [p, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_long)]
        L.sim_kernel_time.restype = i
        L.sim_save.argtypes = [p, ctypes.c_char_p]
        L.sim_save.restype = i
        L.sim_load.argtypes = [p, ctypes.c_char_p]
        L.sim_load.restype = i
        L.sim_destroy.argtypes = [p]
        L.sim_destroy.restype = None
        L.sim_last_error.argtypes = [p]
        L.sim_last_error.restype = ctypes.c_char_p
        L.sim_error_string.argtypes = [i]
        L.sim_error_string.restype = ctypes.c_char_p
        L.simb_create.argtypes = [i, ctypes.POINTER(SimGrid), ctypes.POINTER(SimMedium), ctypes.POINTER(SimSource),
                                  ctypes.POINTER(SimReceivers), ctypes.POINTER(SimOpts), ctypes.POINTER(p)]
        L.simb_create.restype = i
        L.simb_run.argtypes = [p, i]
        L.simb_run.restype = i
        L.simb_sync.argtypes = [p]
        L.simb_sync.restype = i
        L.simb_traces.argtypes = [p, i, ctypes.POINTER(ctypes.c_float), sz, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.simb_traces.restype = i
        L.simb_read_field.argtypes = [p, i, i, ctypes.POINTER(ctypes.c_float), sz]
        L.simb_read_field.restype = i
        L.simb_config.argtypes = [p, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i)]
        L.simb_config.restype = i
        L.simb_destroy.argtypes = [p]
        L.simb_destroy.restype = None
        L.simb_last_error.argtypes = [p]
        L.simb_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(L, h, rc):
    if rc != SIM_OK:
        raise SimError(rc, L.sim_last_error(h).decode())
    return rc


def make_structs(scenario, *, storage="f32", pml_on=None, graph_chunk=0, stream=None, mem_cap=0, max_steps=None,
                 kernel="auto", timing=False, device=0, dt=0.0):
    """C structs for a workload Scenario; returns (structs, keepalive)."""
    m = scenario.medium
    g = m.grid
    keep = dict(rho=np.ascontiguousarray(m.rho, np.float64), vp=np.ascontiguousarray(m.vp, np.float64),
                vs=np.ascontiguousarray(m.vs, np.float64), cid=np.ascontiguousarray(m.cell_id, np.uint16),
                rr=np.ascontiguousarray(scenario.receivers.r, np.float64),
                rt=np.ascontiguousarray(scenario.receivers.theta, np.float64),
                rz=np.ascontiguousarray(scenario.receivers.z, np.float64))
    grid = SimGrid(g.nr, g.nth, g.nz, g.pml_r, g.pml_z, g.dr, g.dz, float(scenario.cfl), float(dt))
    med = SimMedium(len(keep["rho"]), _dp(keep["rho"]), _dp(keep["vp"]), _dp(keep["vs"]), keep["cid"].ctypes.data)
    s = scenario.source
    src = SimSource(int(s.kind), float(s.r), float(s.theta), float(s.z), float(s.f0), float(s.amplitude))
    rec = SimReceivers(len(keep["rz"]), _dp(keep["rr"]), _dp(keep["rt"]), _dp(keep["rz"]),
                       int(scenario.receivers.quantity))
    on = scenario.pml_on if pml_on is None else pml_on
    cap = scenario.steps if max_steps is None else max_steps
    opts = SimOpts(STORAGE[storage] if isinstance(storage, str) else int(storage), 0 if on else 1, int(graph_chunk),
                   ctypes.c_void_p(stream) if stream else None, int(mem_cap), int(cap),
                   KERNEL[kernel] if isinstance(kernel, str) else int(kernel), int(bool(timing)), int(device))
    return (grid, med, src, rec, opts), keep


class Simulation:
    """One simulator handle (sim_create ... sim_destroy)."""

    def __init__(self, scenario, **kw):
        self.L = lib()
        (grid, med, src, rec, opts), self._keep = make_structs(scenario, **kw)
        self.grid = scenario.medium.grid
        self.n_rec = rec.n
        h = ctypes.c_void_p()
        rc = self.L.sim_create(ctypes.byref(grid), ctypes.byref(med), ctypes.byref(src), ctypes.byref(rec),
                               ctypes.byref(opts), ctypes.byref(h))
        if rc != SIM_OK:
            raise SimError(rc, self.L.sim_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def dt(self) -> float:
        return float(self.L.sim_dt(self.h))

    @property
    def steps_done(self) -> int:
        return int(self.L.sim_steps_done(self.h))

    @property
    def device_bytes(self) -> int:
        return int(self.L.sim_device_bytes(self.h))

    def step(self, n: int):
        _check(self.L, self.h, self.L.sim_step(self.h, int(n)))
        return self

    def sync(self):
        _check(self.L, self.h, self.L.sim_sync(self.h))

    def traces(self) -> np.ndarray:
        nr, ns = ctypes.c_int(), ctypes.c_int()
        _check(self.L, self.h, self.L.sim_traces(self.h, None, 0, ctypes.byref(nr), ctypes.byref(ns)))
        out = np.zeros((nr.value, ns.value), np.float32)
        _check(self.L, self.h, self.L.sim_traces(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 out.size, ctypes.byref(nr), ctypes.byref(ns)))
        return out

    def field(self, name: str) -> np.ndarray:
        out = np.zeros(self.grid.shape, np.float32)
        _check(self.L, self.h, self.L.sim_read_field(self.h, FIELDS.index(name),
                                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def set_field(self, name: str, a: np.ndarray):
        a = np.ascontiguousarray(a, np.float32)
        assert a.shape == self.grid.shape
        _check(self.L, self.h, self.L.sim_write_field(self.h, FIELDS.index(name),
                                                      a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def config(self):
        """(kernel, tile_rows): kernel 1 = split, 2 = fused; tile rows chosen by the autotuner."""
        k, t = ctypes.c_int(), ctypes.c_int()
        _check(self.L, self.h, self.L.sim_config(self.h, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def kernel_time(self, q: int):
        ms, n = ctypes.c_double(), ctypes.c_long()
        _check(self.L, self.h, self.L.sim_kernel_time(self.h, q, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def save(self, path: str):
        _check(self.L, self.h, self.L.sim_save(self.h, path.encode()))

    def load(self, path: str):
        _check(self.L, self.h, self.L.sim_load(self.h, path.encode()))


class BatchSimulation:
    """Many wells advanced together (simb_create ... simb_destroy)."""

    def __init__(self, scenarios, **kw):
        self.L = lib()
        n = len(scenarios)
        if n == 0:
            raise SimError(SIM_EINVAL, "a batch needs at least one scenario")
        parts = [make_structs(sc, **kw) for sc in scenarios]
        self._keep = [k for _, k in parts]
        G = (SimGrid * n)(*[p[0][0] for p in parts])
        M = (SimMedium * n)(*[p[0][1] for p in parts])
        S = (SimSource * n)(*[p[0][2] for p in parts])
        R = (SimReceivers * n)(*[p[0][3] for p in parts])
        opts = parts[0][0][4]
        self._arrays = (G, M, S, R, opts)
        self.grids = [sc.medium.grid for sc in scenarios]
        h = ctypes.c_void_p()
        rc = self.L.simb_create(n, G, M, S, R, ctypes.byref(opts), ctypes.byref(h))
        if rc != SIM_OK:
            raise SimError(rc, self.L.simb_last_error(None).decode())
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            self.L.simb_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, rc):
        if rc != SIM_OK:
            raise SimError(rc, self.L.simb_last_error(self.h).decode())

    def run(self, n: int):
        self._chk(self.L.simb_run(self.h, int(n)))
        return self

    def sync(self):
        self._chk(self.L.simb_sync(self.h))

    def traces(self, which: int) -> np.ndarray:
        nr, ns = ctypes.c_int(), ctypes.c_int()
        self._chk(self.L.simb_traces(self.h, int(which), None, 0, ctypes.byref(nr), ctypes.byref(ns)))
        out = np.zeros((nr.value, ns.value), np.float32)
        self._chk(self.L.simb_traces(self.h, int(which), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size,
                                     ctypes.byref(nr), ctypes.byref(ns)))
        return out

    def field(self, which: int, name: str) -> np.ndarray:
        out = np.zeros(self.grids[which].shape, np.float32)
        self._chk(self.L.simb_read_field(self.h, int(which), FIELDS.index(name),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def config(self):
        """(cases, work items per launch, persistent blocks per launch)."""
        n, w, g = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        self._chk(self.L.simb_config(self.h, ctypes.byref(n), ctypes.byref(w), ctypes.byref(g)))
        return n.value, w.value, g.value
