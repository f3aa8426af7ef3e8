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
STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "f16sr": 3}
KERNEL = {"auto": 0, "split": 1, "fused": 2, "fused4": 3, "march": 4, "sweep": 5}


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
                ("kernel", ctypes.c_int), ("timing", ctypes.c_int), ("device", ctypes.c_int), ("tile", ctypes.c_int),
                ("watchdog_every", ctypes.c_int)]


class SimZones(ctypes.Structure):
    _fields_ = [("n_zones", ctypes.c_int), ("row0", ctypes.POINTER(ctypes.c_int))]


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
        L.sim_read_field_noalloc.argtypes = [p, i, ctypes.POINTER(ctypes.c_float), sz]
        L.sim_read_field_noalloc.restype = i
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
        L.sim_set_wait_test.argtypes = [p, ctypes.c_longlong, i]
        L.sim_set_wait_test.restype = i
        L.sim_time_step.argtypes = [p, p, ctypes.POINTER(ctypes.c_double)]
        L.sim_time_step.restype = i
        L.sim_watchdog.argtypes = [p, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(i)]
        L.sim_watchdog.restype = i
        L.sim_round_f16_sr.argtypes = [p, p, p, ctypes.c_longlong, p]
        L.sim_round_f16_sr.restype = i
        L.sim_create_slab.argtypes = [p, p, p, p, p, i, i, ctypes.POINTER(p)]
        L.sim_create_slab.restype = i
        L.sim_half_step.argtypes = [p, i]
        L.sim_half_step.restype = i
        L.sim_slab_info.argtypes = [p] + [ctypes.POINTER(i)] * 4
        L.sim_slab_info.restype = i
        L.sim_get_planes.argtypes = [p, i, i, i, p]
        L.sim_get_planes.restype = i
        L.sim_put_planes.argtypes = [p, i, i, i, p]
        L.sim_put_planes.restype = i
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
        L.simb_layout.argtypes = [p, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.simb_layout.restype = i
        L.simb_destroy.argtypes = [p]
        L.simb_destroy.restype = None
        L.simb_last_error.argtypes = [p]
        L.simb_last_error.restype = ctypes.c_char_p
        L.simr_create.argtypes = [ctypes.POINTER(SimGrid), ctypes.POINTER(SimZones), ctypes.POINTER(SimMedium),
                                  ctypes.POINTER(SimSource), ctypes.POINTER(SimReceivers), ctypes.POINTER(SimOpts),
                                  ctypes.POINTER(p)]
        L.simr_create.restype = i
        L.simr_step.argtypes = [p, i]
        L.simr_step.restype = i
        L.simr_sync.argtypes = [p]
        L.simr_sync.restype = i
        L.simr_traces.argtypes = [p, ctypes.POINTER(ctypes.c_float), sz, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.simr_traces.restype = i
        L.simr_zone.argtypes = [p, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.simr_zone.restype = i
        L.simr_read_field.argtypes = [p, i, i, ctypes.POINTER(ctypes.c_float), sz]
        L.simr_read_field.restype = i
        L.simr_dt.argtypes = [p]
        L.simr_dt.restype = d
        L.simr_steps_done.argtypes = [p]
        L.simr_steps_done.restype = i
        L.simr_cells.argtypes = [p]
        L.simr_cells.restype = sz
        L.simr_destroy.argtypes = [p]
        L.simr_destroy.restype = None
        L.simr_last_error.argtypes = [p]
        L.simr_last_error.restype = ctypes.c_char_p
        L.simr_interface_matrix.argtypes = [i, i, i, ctypes.POINTER(ctypes.c_double)]
        L.simr_interface_matrix.restype = i
        _lib = L
    return _lib


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _ptr(a):
    """Data pointer of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return ctypes.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return ctypes.c_void_p(a.data_ptr())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(L, h, rc):
    if rc != SIM_OK:
        raise SimError(rc, L.sim_last_error(h).decode())
    return rc


def make_structs(scenario, *, storage="f32", pml_on=None, graph_chunk=0, stream=None, mem_cap=0, max_steps=None,
                 kernel="auto", timing=False, device=0, dt=0.0, tile=0, watchdog_every=0):
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
                   KERNEL[kernel] if isinstance(kernel, str) else int(kernel), int(bool(timing)), int(device),
                   int(tile), int(watchdog_every))
    return (grid, med, src, rec, opts), keep


def time_step(scenario, dt=0.0) -> float:
    """The time step sim_create takes for `scenario` (host only, sim_time_step)."""
    L = lib()
    (grid, med, _, _, _), keep = make_structs(scenario, dt=dt)
    out = ctypes.c_double()
    rc = L.sim_time_step(ctypes.byref(grid), ctypes.byref(med), ctypes.byref(out))
    if rc != SIM_OK:
        raise SimError(rc, L.sim_last_error(None).decode())
    return out.value


def round_f16_sr(x, dither, out, stream=None):
    """sim_round_f16_sr on CUDA tensors: x float32, dither int32 (13 bits
    used), out int16 (FP16 bit patterns), all contiguous and of one length."""
    L = lib()
    n = x.numel()
    if dither.numel() != n or out.numel() != n:
        raise ValueError("x, dither and out need the same length")
    rc = L.sim_round_f16_sr(_ptr(x), _ptr(dither), _ptr(out), n, stream)
    if rc != SIM_OK:
        raise SimError(rc, L.sim_last_error(None).decode())
    return out


class Simulation:
    """One simulator handle (sim_create ... sim_destroy)."""

    def __init__(self, scenario, slab=None, **kw):
        """slab = (s0, s1): the z slab of stored cells s0 <= k < s1 of the
        well (sim_create_slab); fields then cover the cells the handle holds."""
        self.L = lib()
        (grid, med, src, rec, opts), self._keep = make_structs(scenario, **kw)
        self.grid = scenario.medium.grid
        self.n_rec = rec.n
        h = ctypes.c_void_p()
        if slab is None:
            rc = self.L.sim_create(ctypes.byref(grid), ctypes.byref(med), ctypes.byref(src), ctypes.byref(rec),
                                   ctypes.byref(opts), ctypes.byref(h))
        else:
            rc = self.L.sim_create_slab(ctypes.byref(grid), ctypes.byref(med), ctypes.byref(src), ctypes.byref(rec),
                                        ctypes.byref(opts), int(slab[0]), int(slab[1]), ctypes.byref(h))
        if rc != SIM_OK:
            raise SimError(rc, self.L.sim_last_error(None).decode())
        self.h = h
        l0, s0, s1, nz = (ctypes.c_int() for _ in range(4))
        _check(self.L, self.h, self.L.sim_slab_info(self.h, ctypes.byref(l0), ctypes.byref(s0), ctypes.byref(s1),
                                                    ctypes.byref(nz)))
        self.l0, self.s0, self.s1 = l0.value, s0.value, s1.value
        self.shape = (self.grid.nth, self.grid.NR, nz.value)

    def half_step(self, which: int):
        """0: velocity half-step (and point forces); 1: stress half-step,
        source and receivers (sim_half_step)."""
        _check(self.L, self.h, self.L.sim_half_step(self.h, int(which)))

    def get_planes(self, group: int, k0: int, k1: int, out):
        """Planes k0 <= k < k1 of group 0 (velocities) / 1 (stresses) into
        `out` (a float32 numpy array or a CUDA torch tensor of
        [fields][nth * NR][k1 - k0]); asynchronous on the handle's stream."""
        _check(self.L, self.h, self.L.sim_get_planes(self.h, int(group), int(k0), int(k1), _ptr(out)))
        return out

    def put_planes(self, group: int, k0: int, k1: int, buf):
        _check(self.L, self.h, self.L.sim_put_planes(self.h, int(group), int(k0), int(k1), _ptr(buf)))

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
        out = np.zeros(self.shape, np.float32)
        _check(self.L, self.h, self.L.sim_read_field(self.h, FIELDS.index(name),
                                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def field_noalloc(self, name: str) -> np.ndarray:
        """As field(), staged in the library's fixed device scratch (no device allocation)."""
        out = np.zeros(self.shape, np.float32)
        _check(self.L, self.h, self.L.sim_read_field_noalloc(self.h, FIELDS.index(name),
                                                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                             out.size))
        return out

    def set_field(self, name: str, a: np.ndarray):
        a = np.ascontiguousarray(a, np.float32)
        assert a.shape == self.shape
        _check(self.L, self.h, self.L.sim_write_field(self.h, FIELDS.index(name),
                                                      a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def config(self):
        """(kernel, tile code): kernel 1 = split, 2 = fused, 4 = marching, 5 = sweep; the tile code
        the autotuner chose (0 split; r or 100 + r fused; 1000 + 100 r + J marching)."""
        k, t = ctypes.c_int(), ctypes.c_int()
        _check(self.L, self.h, self.L.sim_config(self.h, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def watchdog(self):
        """(energy proxy of the last check, reference, step of that check)
        of the device watchdog (opts.watchdog_every > 0; sim_watchdog)."""
        e, r, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(self.L, self.h, self.L.sim_watchdog(self.h, ctypes.byref(e), ctypes.byref(r), ctypes.byref(n)))
        return e.value, r.value, n.value

    def set_wait_test(self, wait_cycles: int, withhold_chunk: int):
        """Test hook of the sweep kernel's bounded waits (sim_set_wait_test)."""
        _check(self.L, self.h, self.L.sim_set_wait_test(self.h, int(wait_cycles), int(withhold_chunk)))

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

    def layout(self):
        """(cases on their own launches, parallel streams they run on)."""
        o, b = ctypes.c_int(), ctypes.c_int()
        self._chk(self.L.simb_layout(self.h, ctypes.byref(o), ctypes.byref(b)))
        return o.value, b.value


def interface_matrix(n_coarse: int, half: bool, fine_to_coarse: bool) -> np.ndarray:
    """The refined grid's interface map (simr_interface_matrix), FP64."""
    L = lib()
    shape = (n_coarse, 2 * n_coarse) if fine_to_coarse else (2 * n_coarse, n_coarse)
    out = np.zeros(shape)
    rc = L.simr_interface_matrix(int(n_coarse), int(bool(half)), int(bool(fine_to_coarse)), _dp(out))
    if rc != SIM_OK:
        raise SimError(rc, "simr_interface_matrix")
    return out


class RefinedSimulation:
    """One well on the azimuthally refined grid (simr_create ... simr_destroy):
    zones 1 .. M-1 start at `rows`; zone m has nth / 2^(M-1-m) azimuthal nodes."""

    def __init__(self, scenario, rows, **kw):
        self.L = lib()
        (grid, med, src, rec, opts), self._keep = make_structs(scenario, **kw)
        self._rows = (ctypes.c_int * max(1, len(rows)))(*[int(r) for r in rows])
        zones = SimZones(len(rows) + 1, self._rows)
        self.grid = scenario.medium.grid
        h = ctypes.c_void_p()
        rc = self.L.simr_create(ctypes.byref(grid), ctypes.byref(zones), ctypes.byref(med), ctypes.byref(src),
                                ctypes.byref(rec), ctypes.byref(opts), ctypes.byref(h))
        if rc != SIM_OK:
            raise SimError(rc, self.L.simr_last_error(None).decode())
        self.h = h
        self.M = len(rows) + 1
        self.zones = []
        for z in range(self.M):
            a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            self._chk(self.L.simr_zone(self.h, z, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
            self.zones.append((a.value, b.value, c.value))  # first row, rows, nth

    def close(self):
        if getattr(self, "h", None):
            self.L.simr_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, rc):
        if rc != SIM_OK:
            raise SimError(rc, self.L.simr_last_error(self.h).decode())

    @property
    def dt(self) -> float:
        return float(self.L.simr_dt(self.h))

    @property
    def cells(self) -> int:
        return int(self.L.simr_cells(self.h))

    def step(self, n: int):
        self._chk(self.L.simr_step(self.h, int(n)))
        return self

    def sync(self):
        self._chk(self.L.simr_sync(self.h))

    def traces(self) -> np.ndarray:
        nr, ns = ctypes.c_int(), ctypes.c_int()
        self._chk(self.L.simr_traces(self.h, None, 0, ctypes.byref(nr), ctypes.byref(ns)))
        out = np.zeros((nr.value, ns.value), np.float32)
        self._chk(self.L.simr_traces(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size,
                                     ctypes.byref(nr), ctypes.byref(ns)))
        return out

    def field(self, name: str, zone: int) -> np.ndarray:
        """[nth_zone][rows][NZ] of one zone."""
        row, rows, nth = self.zones[zone]
        out = np.zeros((nth, rows, self.grid.NZ), np.float32)
        self._chk(self.L.simr_read_field(self.h, FIELDS.index(name), int(zone),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out


# ------------------------------------------------------------------ surrogate
class SurCfg(ctypes.Structure):
    _fields_ = [("in_dim", ctypes.c_int), ("h1", ctypes.c_int), ("h2", ctypes.c_int), ("l0", ctypes.c_int),
                ("n_up", ctypes.c_int), ("chans", ctypes.c_int * 9), ("out_ch", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


SURROGATE_DEFAULT = dict(in_dim=6, h1=256, h2=512, l0=64, chans=(64, 64, 64, 32, 32, 16), out_ch=8)


def _sur_sigs(L):
    if getattr(L, "_sur_ready", False):
        return
    p, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    fp = ctypes.POINTER(ctypes.c_float)
    L.sur_create.argtypes = [ctypes.POINTER(SurCfg), ctypes.POINTER(SimOpts), ctypes.POINTER(p)]
    L.sur_create.restype = i
    L.sur_param_count.argtypes = [p, ctypes.POINTER(ctypes.c_longlong)]
    L.sur_param_count.restype = i
    L.sur_get_params.argtypes = [p, fp, sz]
    L.sur_get_params.restype = i
    L.sur_set_params.argtypes = [p, fp, sz]
    L.sur_set_params.restype = i
    L.sur_set_normalization.argtypes = [p, fp, fp, ctypes.c_float]
    L.sur_set_normalization.restype = i
    L.sur_forward.argtypes = [p, fp, i, fp]
    L.sur_forward.restype = i
    L.sur_loss_grad.argtypes = [p, fp, fp, i, fp, fp, sz]
    L.sur_loss_grad.restype = i
    L.sur_train.argtypes = [p, fp, fp, i, i, i, ctypes.c_float, ctypes.c_ulonglong, fp]
    L.sur_train.restype = i
    L.sur_gate_fit.argtypes = [p, fp, fp, i]
    L.sur_gate_fit.restype = i
    L.sur_gate.argtypes = [p, fp, i, i, ctypes.c_float, ctypes.POINTER(i)]
    L.sur_sensitivity.argtypes = [p, fp, i, ctypes.c_float, fp]
    L.sur_sensitivity.restype = i
    L.sur_gate.restype = i
    L.sur_destroy.argtypes = [p]
    L.sur_destroy.restype = None
    L.sur_last_error.argtypes = [p]
    L.sur_last_error.restype = ctypes.c_char_p
    u16p = ctypes.POINTER(ctypes.c_uint16)
    L.cw_gemm_bf16.argtypes = [i, i, i, i, i, u16p, i, u16p, i, fp, i]
    L.cw_gemm_bf16.restype = i
    L.cw_gemm_bf16_path.argtypes = [i, i, i, i, i, i, u16p, i, u16p, i, fp, i]
    L.cw_gemm_bf16_path.restype = i
    L._sur_ready = True


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


GEMM_PATH = {"auto": 0, "mma": 1, "tcgen05": 2}


def gemm_bf16(A16: np.ndarray, B16: np.ndarray, trans_a=False, trans_b=False, path="auto") -> np.ndarray:
    """Tensor-core GEMM on BF16 bit patterns (uint16 arrays), FP32 result;
    path "auto" (by shape, as in training), "mma" or "tcgen05"."""
    L = lib()
    _sur_sigs(L)
    A16 = np.ascontiguousarray(A16, np.uint16)
    B16 = np.ascontiguousarray(B16, np.uint16)
    M, K = (A16.shape[1], A16.shape[0]) if trans_a else A16.shape
    N = B16.shape[0] if trans_b else B16.shape[1]
    C = np.zeros((M, N), np.float32)
    u16p = ctypes.POINTER(ctypes.c_uint16)
    rc = L.cw_gemm_bf16_path(GEMM_PATH[path], int(trans_a), int(trans_b), M, N, K, A16.ctypes.data_as(u16p),
                             A16.shape[1], B16.ctypes.data_as(u16p), B16.shape[1], _fp(C), N)
    if rc != SIM_OK:
        raise SimError(rc, "cw_gemm_bf16_path failed")
    return C


class Surrogate:
    """Trace surrogate handle (sur_create ... sur_destroy)."""

    def __init__(self, max_batch=32, seed=1, stream=None, device=0, **arch):
        self.L = lib()
        _sur_sigs(self.L)
        a = dict(SURROGATE_DEFAULT)
        a.update(arch)
        ch = list(a["chans"])
        cfg = SurCfg(a["in_dim"], a["h1"], a["h2"], a["l0"], len(ch) - 1, (ctypes.c_int * 9)(*(ch + [0] * (9 - len(ch)))),
                     a["out_ch"], int(max_batch), int(seed))
        opts = SimOpts(0, 0, 0, ctypes.c_void_p(stream) if stream else None, 0, 0, 0, 0, int(device))
        h = ctypes.c_void_p()
        rc = self.L.sur_create(ctypes.byref(cfg), ctypes.byref(opts), ctypes.byref(h))
        if rc != SIM_OK:
            raise SimError(rc, self.L.sur_last_error(None).decode())
        self.h = h
        self.arch = a
        self.out_len = a["l0"] * 2 ** (len(ch) - 1)
        n = ctypes.c_longlong()
        self._chk(self.L.sur_param_count(self.h, ctypes.byref(n)))
        self.n_params = n.value

    def _chk(self, rc):
        if rc != SIM_OK:
            raise SimError(rc, self.L.sur_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.sur_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *e):
        self.close()

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._chk(self.L.sur_get_params(self.h, _fp(out), out.size))
        return out

    def set_params(self, th):
        th = np.ascontiguousarray(th, np.float32)
        self._chk(self.L.sur_set_params(self.h, _fp(th), th.size))

    def set_normalization(self, mean, scale, y_scale=1.0):
        m = np.ascontiguousarray(mean, np.float32)
        s = np.ascontiguousarray(scale, np.float32)
        self._chk(self.L.sur_set_normalization(self.h, _fp(m), _fp(s), float(y_scale)))

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        Y = np.zeros((X.shape[0], self.arch["out_ch"], self.out_len), np.float32)
        self._chk(self.L.sur_forward(self.h, _fp(X), X.shape[0], _fp(Y)))
        return Y

    def loss_grad(self, X, Y):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_float()
        self._chk(self.L.sur_loss_grad(self.h, _fp(X), _fp(Y), X.shape[0], ctypes.byref(loss), _fp(g), g.size))
        return loss.value, g

    def train(self, X, Y, epochs, batch=32, lr=1e-3, seed=0):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        hist = np.zeros(max(epochs, 1), np.float32)
        self._chk(self.L.sur_train(self.h, _fp(X), _fp(Y), X.shape[0], int(epochs), int(batch), float(lr), int(seed),
                                   _fp(hist)))
        return hist[:epochs]

    def gate_fit(self, X, err):
        X = np.ascontiguousarray(X, np.float32)
        e = np.ascontiguousarray(err, np.float32)
        self._chk(self.L.sur_gate_fit(self.h, _fp(X), _fp(e), X.shape[0]))

    def sensitivity(self, X, step=0.1) -> np.ndarray:
        """sur_sensitivity: the largest relative output change over unit
        moves of `step` (normalised units) along each input dimension."""
        X = np.ascontiguousarray(X, np.float32)
        out = np.zeros(X.shape[0], np.float32)
        self._chk(self.L.sur_sensitivity(self.h, _fp(X), X.shape[0], float(step), _fp(out)))
        return out

    def gate(self, X, k=3, tol=0.05) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        acc = np.zeros(X.shape[0], np.int32)
        self._chk(self.L.sur_gate(self.h, _fp(X), X.shape[0], int(k), float(tol),
                                  acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return acc.astype(bool)
