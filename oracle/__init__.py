"""FP64 CPU oracle of the cased-well velocity-stress scheme (test infrastructure).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
use this package; the CUDA simulator never imports, links or runs it.  The
numerical work lives in `cwell_oracle.c` (plain loops, FP64) and, for the
azimuthally refined grid, `cwell_refine.c`; this module compiles them with gcc
and exposes them through ctypes, plus the few closed forms the tests pin them
with.

Field order (Sec. 2 of the paper): v_r, v_phi, v_z, s_rr, s_phiphi, s_zz,
s_rphi, s_phiz, s_rz; each is a float64 array [theta][r][z], z fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "cwell_oracle.c"), os.path.join(_HERE, "cwell_refine.c")]
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = ("vr", "vp", "vz", "srr", "spp", "szz", "srp", "spz", "srz")
PSI = ("vr_r", "vp_r", "vz_r", "vr_z", "vp_z", "vz_z", "err_r", "grp_r", "grz_r", "ezz_z", "grz_z", "gpz_z",
       "vr_q", "vp_q", "vz_q", "epp_q", "grp_q", "gpz_q")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i, p, sz = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_create.restype = p
            L.or_create.argtypes = [i, i, i, i, i, d, d, i, dp, dp, dp, p, d, d, i,
                                    i, d, d, d, d, d, i, dp, dp, dp, i, ctypes.POINTER(i)]
            L.or_step.argtypes = [p, i]
            L.or_step.restype = i
            L.or_destroy.argtypes = [p]
            L.or_dt.argtypes = [p]
            L.or_dt.restype = d
            L.or_steps_done.argtypes = [p]
            L.or_steps_done.restype = i
            L.or_field.argtypes = [p, i]
            L.or_field.restype = dp
            L.or_psi.argtypes = [p, i]
            L.or_psi.restype = dp
            L.or_traces.argtypes = [p]
            L.or_traces.restype = dp
            L.or_trace_capacity.argtypes = [p]
            L.or_trace_capacity.restype = i
            L.or_set_threads.argtypes = [p, i]
            L.or_max_threads.restype = i
            L.or_ricker.argtypes = [d, d]
            L.or_ricker.restype = d
            L.or_cfl_dt.argtypes = [i, i, i, d, d, p, dp, d]
            L.or_cfl_dt.restype = d
            L.or_round_storage.argtypes = [d, i]
            L.or_round_storage.restype = d
            L.or_set_storage.argtypes = [p, i, d, d]
            L.or_set_storage.restype = i
            L.or_round_stochastic_f16.argtypes = [d, ctypes.c_uint]
            L.or_round_stochastic_f16.restype = d
            L.or_splitmix64.argtypes = [ctypes.c_uint64]
            L.or_splitmix64.restype = ctypes.c_uint64
            L.or_sr_dither.argtypes = [i, i, i, i, i, i, i, i]
            L.or_sr_dither.restype = ctypes.c_uint
            L.or_pml_table.argtypes = [p, i]
            L.or_pml_table.restype = dp
            L.or_set_zrange.argtypes = [p, i, i]
            L.or_set_zrange.restype = i
            L.or_set_steps_done.argtypes = [p, i]
            L.or_velocity_update.argtypes = [p]
            L.or_stress_update.argtypes = [p]
            L.or_inject_source.argtypes = [p, i]
            L.or_sample.argtypes = [p, i]
            ip = ctypes.POINTER(i)
            L.or_ref_create.restype = p
            L.or_ref_create.argtypes = [i, i, i, i, i, d, d, i, ip, i, dp, dp, dp, p, d, d, i,
                                        i, d, d, d, d, d, i, dp, dp, dp, i, ip]
            L.or_ref_step.argtypes = [p, i]
            L.or_ref_step.restype = i
            L.or_ref_destroy.argtypes = [p]
            L.or_ref_dt.argtypes = [p]
            L.or_ref_dt.restype = d
            L.or_ref_steps_done.argtypes = [p]
            L.or_ref_steps_done.restype = i
            L.or_ref_field.argtypes = [p, i]
            L.or_ref_field.restype = dp
            L.or_ref_traces.argtypes = [p]
            L.or_ref_traces.restype = dp
            L.or_ref_set_threads.argtypes = [p, i]
            L.or_ref_zone.argtypes = [p, i, ip, ip, ip, ctypes.POINTER(ctypes.c_longlong)]
            L.or_ref_matrix.argtypes = [p, i, i]
            L.or_ref_matrix.restype = dp
            L.or_ref_interp.argtypes = [dp, i, i, i, dp]
            L.or_ref_velocity_update.argtypes = [p]
            L.or_ref_stress_update.argtypes = [p]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ricker(t, f0: float):
    """Ricker pulse of the paper (Sec. 2) with delay 2/f0, evaluated by the oracle."""
    L = lib()
    t = np.asarray(t, dtype=np.float64)
    return np.vectorize(lambda x: L.or_ricker(float(x), float(f0)))(t)


def max_threads() -> int:
    return int(lib().or_max_threads())


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle run: a medium, a source, receivers, FP64 leapfrog steps.

    `scenario` is any object with `.medium` (grid, cell_id, rho, vp, vs),
    `.source` (kind, r, theta, z, f0, amplitude), `.receivers` (r, theta, z),
    `.cfl` and `.pml_on` attributes.
    """

    def __init__(self, scenario, *, max_steps: int | None = None, dt: float = 0.0,
                 pml_on: bool | None = None, threads: int = 0, storage: str = "f64",
                 scales: tuple = (1.0, 1.0)):
        """`storage` "bf16" / "f16" rounds every field to that 16-bit format
        where the reduced-precision variant stores it (values first rounded
        to FP32, the variant's arithmetic precision; "f16sr": FP16 with
        stochastic rounding); `scales` = (velocity, stress) factors of the
        stored representation round(value * scale)."""
        L = lib()
        m = scenario.medium
        g = m.grid
        src = scenario.source
        rec = scenario.receivers
        self.grid = g
        self._rho = np.ascontiguousarray(m.rho, dtype=np.float64)
        self._vp = np.ascontiguousarray(m.vp, dtype=np.float64)
        self._vs = np.ascontiguousarray(m.vs, dtype=np.float64)
        self._id = np.ascontiguousarray(m.cell_id, dtype=np.uint16)
        self._rr = np.ascontiguousarray(rec.r, dtype=np.float64)
        self._rt = np.ascontiguousarray(rec.theta, dtype=np.float64)
        self._rz = np.ascontiguousarray(rec.z, dtype=np.float64)
        on = scenario.pml_on if pml_on is None else pml_on
        cap = int(scenario.steps if max_steps is None else max_steps)
        err = ctypes.c_int(0)
        h = L.or_create(g.nr, g.nth, g.nz, g.pml_r, g.pml_z, g.dr, g.dz, len(self._rho),
                        _dp(self._rho), _dp(self._vp), _dp(self._vs), self._id.ctypes.data,
                        float(scenario.cfl), float(dt), int(bool(on)),
                        int(src.kind), float(src.r), float(src.theta), float(src.z), float(src.f0),
                        float(src.amplitude), len(self._rr), _dp(self._rr), _dp(self._rt), _dp(self._rz),
                        cap, ctypes.byref(err))
        if not h:
            raise OracleError(f"or_create failed with code {err.value}")
        self._h = ctypes.c_void_p(h)
        self._L = L
        self.n_rec = len(self._rr)
        self.cap = cap
        if threads:
            L.or_set_threads(self._h, int(threads))
        mode = STORAGE_MODES[storage]
        if mode:
            rc = L.or_set_storage(self._h, mode, float(scales[0]), float(scales[1]))
            if rc != 0:
                raise OracleError(f"or_set_storage failed with code {rc}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    @property
    def dt(self) -> float:
        return float(self._L.or_dt(self._h))

    @property
    def steps_done(self) -> int:
        return int(self._L.or_steps_done(self._h))

    def step(self, n: int = 1):
        rc = self._L.or_step(self._h, int(n))
        if rc != 0:
            raise OracleError(f"or_step failed with code {rc}")
        return self

    def velocity_update(self):
        self._L.or_velocity_update(self._h)

    def stress_update(self):
        self._L.or_stress_update(self._h)

    def inject_source(self, n: int):
        """The source of step n (point forces after the velocity update, the
        volumetric source and the torsion ring after the stress update)."""
        self._L.or_inject_source(self._h, int(n))

    def sample(self, n: int):
        self._L.or_sample(self._h, int(n))

    def set_zrange(self, k_lo: int, k_hi: int):
        """Update, inject and sample only stored z cells k_lo <= k < k_hi."""
        if self._L.or_set_zrange(self._h, int(k_lo), int(k_hi)) != 0:
            raise OracleError("bad z range")

    def set_steps_done(self, n: int):
        self._L.or_set_steps_done(self._h, int(n))

    def field(self, name: str) -> np.ndarray:
        """Writable view of a field, shape [nth][NR][NZ]."""
        q = FIELDS.index(name)
        ptr = self._L.or_field(self._h, q)
        g = self.grid
        return np.ctypeslib.as_array(ptr, shape=(g.nth, g.NR, g.NZ))

    def psi(self, name: str) -> np.ndarray:
        q = PSI.index(name)
        ptr = self._L.or_psi(self._h, q)
        g = self.grid
        return np.ctypeslib.as_array(ptr, shape=(g.nth, g.NR, g.NZ))

    def fields(self) -> dict:
        return {n: self.field(n).copy() for n in FIELDS}

    def pml_table(self, q: int) -> np.ndarray:
        n = self.grid.NR if q < 8 else self.grid.NZ
        return np.ctypeslib.as_array(self._L.or_pml_table(self._h, q), shape=(n,)).copy()

    def traces(self) -> np.ndarray:
        """[n_rec][steps_done] pressure traces; sample m is p after step m."""
        n = min(self.steps_done, self.cap)
        if self.n_rec == 0 or self.cap == 0:
            return np.zeros((self.n_rec, n))
        full = np.ctypeslib.as_array(self._L.or_traces(self._h), shape=(self.n_rec, self.cap))
        return full[:, :n].copy()


STORAGE_MODES = {"f64": 0, "bf16": 1, "f16": 2, "f16sr": 3}


def round_storage(x, storage: str) -> np.ndarray:
    """The oracle's rounding of values to a storage format (via FP32, round
    to nearest even), element by element."""
    L = lib()
    mode = STORAGE_MODES[storage]
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(lambda v: L.or_round_storage(float(v), mode), otypes=[np.float64])(x)


def round_stochastic_f16(x, dither) -> np.ndarray:
    """The oracle's stochastic rounding to FP16 with the given 13-bit dithers."""
    L = lib()
    x = np.asarray(x, dtype=np.float64)
    d = np.broadcast_to(np.asarray(dither, dtype=np.uint32), x.shape)
    return np.vectorize(lambda v, r: L.or_round_stochastic_f16(float(v), int(r)), otypes=[np.float64])(x, d)


def splitmix64(key: int) -> int:
    return int(lib().or_splitmix64(int(key)))


def sr_dither(n, q, j, i, k, nth, NR, NZ) -> int:
    return int(lib().or_sr_dither(n, q, j, i, k, nth, NR, NZ))


def cfl_dt(medium, cfl: float) -> float:
    g = medium.grid
    vp = np.ascontiguousarray(medium.vp, dtype=np.float64)
    cid = np.ascontiguousarray(medium.cell_id, dtype=np.uint16)
    return float(lib().or_cfl_dt(g.nth, g.NR, g.NZ, g.dr, g.dz, cid.ctypes.data, _dp(vp), float(cfl)))


def fft_interp(a, nb: int, half: bool) -> np.ndarray:
    """The coarse-to-fine azimuthal interpolation of the refined grid (the
    paper's three FFT steps, Sec. 3), applied by the oracle to samples `a`."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros(nb)
    lib().or_ref_interp(_dp(a), len(a), int(nb), int(bool(half)), _dp(out))
    return out


class RefinedOracle:
    """One oracle run on the azimuthally refined grid: `rows` are the rows
    where zones 1 .. M-1 start; zone m has nth / 2^(M-1-m) azimuthal nodes.
    The medium is given on the finest azimuthal grid (the scenario's)."""

    def __init__(self, scenario, rows, *, max_steps: int | None = None, dt: float = 0.0,
                 pml_on: bool | None = None, threads: int = 0):
        L = lib()
        m = scenario.medium
        g = m.grid
        src = scenario.source
        rec = scenario.receivers
        self.grid = g
        self.rows = [int(r) for r in rows]
        self.M = len(self.rows) + 1
        self._row0 = (ctypes.c_int * max(1, len(self.rows)))(*self.rows)
        self._rho = np.ascontiguousarray(m.rho, dtype=np.float64)
        self._vp = np.ascontiguousarray(m.vp, dtype=np.float64)
        self._vs = np.ascontiguousarray(m.vs, dtype=np.float64)
        self._id = np.ascontiguousarray(m.cell_id, dtype=np.uint16)
        self._rr = np.ascontiguousarray(rec.r, dtype=np.float64)
        self._rt = np.ascontiguousarray(rec.theta, dtype=np.float64)
        self._rz = np.ascontiguousarray(rec.z, dtype=np.float64)
        on = scenario.pml_on if pml_on is None else pml_on
        cap = int(scenario.steps if max_steps is None else max_steps)
        err = ctypes.c_int(0)
        h = L.or_ref_create(g.nr, g.nth, g.nz, g.pml_r, g.pml_z, g.dr, g.dz, self.M, self._row0,
                            len(self._rho), _dp(self._rho), _dp(self._vp), _dp(self._vs), self._id.ctypes.data,
                            float(scenario.cfl), float(dt), int(bool(on)),
                            int(src.kind), float(src.r), float(src.theta), float(src.z), float(src.f0),
                            float(src.amplitude), len(self._rr), _dp(self._rr), _dp(self._rt), _dp(self._rz),
                            cap, ctypes.byref(err))
        if not h:
            raise OracleError(f"or_ref_create failed with code {err.value}")
        self._h = ctypes.c_void_p(h)
        self._L = L
        self.n_rec = len(self._rr)
        self.cap = cap
        self.zones = []  # (first row, rows, nth, element offset)
        for z in range(self.M):
            row, rows, nth, off = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
            L.or_ref_zone(self._h, z, ctypes.byref(row), ctypes.byref(rows), ctypes.byref(nth), ctypes.byref(off))
            self.zones.append((row.value, rows.value, nth.value, off.value))
        if threads:
            L.or_ref_set_threads(self._h, int(threads))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_ref_destroy(h)
            self._h = None

    @property
    def dt(self) -> float:
        return float(self._L.or_ref_dt(self._h))

    @property
    def steps_done(self) -> int:
        return int(self._L.or_ref_steps_done(self._h))

    def step(self, n: int = 1):
        rc = self._L.or_ref_step(self._h, int(n))
        if rc != 0:
            raise OracleError(f"or_ref_step failed with code {rc}")
        return self

    def velocity_update(self):
        self._L.or_ref_velocity_update(self._h)

    def stress_update(self):
        self._L.or_ref_stress_update(self._h)

    def field(self, name: str, zone: int) -> np.ndarray:
        """Writable view of a field on one zone, shape [nth_zone][rows][NZ]."""
        q = FIELDS.index(name)
        row, rows, nth, off = self.zones[zone]
        NZ = self.grid.NZ
        last = self.zones[-1]
        total = last[3] + last[1] * last[2] * NZ
        full = np.ctypeslib.as_array(self._L.or_ref_field(self._h, q), shape=(total,))
        return full[off:off + rows * nth * NZ].reshape(rows, nth, NZ).transpose(1, 0, 2)

    def matrix(self, interface: int, half: bool) -> np.ndarray:
        """Coarse-to-fine matrix of interface m (zone m-1 -> zone m)."""
        nb, na = self.zones[interface][2], self.zones[interface - 1][2]
        ptr = self._L.or_ref_matrix(self._h, int(interface), int(bool(half)))
        return np.ctypeslib.as_array(ptr, shape=(nb, na)).copy()

    def traces(self) -> np.ndarray:
        n = min(self.steps_done, self.cap)
        if self.n_rec == 0 or self.cap == 0:
            return np.zeros((self.n_rec, n))
        full = np.ctypeslib.as_array(self._L.or_ref_traces(self._h), shape=(self.n_rec, self.cap))
        return full[:, :n].copy()
