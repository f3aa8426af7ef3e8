"""The C-ABI library loads and exports every declared symbol; host-side
argument validation runs without a GPU (no compute calls here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2302_13907_gb300 import binding as B
from paper_2302_13907_gb300 import build as Bld
from paper_2302_13907_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:sim|simb|simr|sur|cw)_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = Bld.build()
    L = ctypes.CDLL(path)
    names = declared_symbols()
    assert "sim_create" in names and "sim_step" in names and "sim_traces" in names and "simr_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _create(sc, **kw):
    L = B.lib()
    (g, m, s, r, o), keep = B.make_structs(sc, **kw)
    h = ctypes.c_void_p()
    rc = L.sim_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(s), ctypes.byref(r), ctypes.byref(o),
                      ctypes.byref(h))
    return rc, h, L


def _tiny():
    g = W.Grid(nr=8, nth=4, nz=16, pml_r=2, pml_z=2, dr=0.005, dz=0.005)
    return W.Scenario("tiny", W.cased_well(g, z_top=0.04, casing_in=0.02, casing_t=0.005, cement_out=0.03),
                      W.Source(z=0.03), W.on_axis_receivers([0.05]), steps=10)


@pytest.mark.parametrize("mutate,code", [
    (lambda sc: setattr(sc.medium, "grid", W.Grid(8, 5, 16, 2, 2, 0.005, 0.005)), B.SIM_EINVAL),  # odd nth
    (lambda sc: setattr(sc.source, "z", 5.0), B.SIM_EINVAL),  # source outside
    (lambda sc: setattr(sc.receivers, "z", np.array([-1.0])), B.SIM_EINVAL),  # receiver outside
    (lambda sc: setattr(sc.source, "kind", 3), B.SIM_EINVAL),  # torsion ring on the axis
    (lambda sc: (setattr(sc.source, "kind", 3), setattr(sc.source, "r", 0.01)), B.SIM_EUNSUPPORTED),  # ring in liquid
    (lambda sc: setattr(sc.source, "kind", 4), B.SIM_EINVAL),  # no such kind
    (lambda sc: sc.medium.cell_id.__setitem__((0, 0, 3), 99), B.SIM_EINVAL),  # id out of range
    (lambda sc: setattr(sc.medium, "vs", np.full_like(sc.medium.vs, 100.0)), B.SIM_EUNSUPPORTED),  # solid axis
    (lambda sc: setattr(sc.medium, "rho", -sc.medium.rho), B.SIM_EINVAL),
])
def test_host_validation_rejects_bad_input(mutate, code):
    sc = _tiny()
    mutate(sc)
    rc, h, L = _create(sc)
    assert rc == code, L.sim_last_error(None)
    assert not h.value
    assert L.sim_last_error(None)


@pytest.mark.parametrize("kw", [dict(kernel="split", tile=1416), dict(kernel="march", tile=-3), dict(kernel=7),
                                dict(kernel="fused", source_kind=2), dict(watchdog_every=-1)])
def test_host_validation_rejects_bad_kernel_options(kw):
    """Kernel / tile options are checked on the host before any device call
    (point forces cannot run on the fused kernels)."""
    sc = _tiny()
    kind = kw.pop("source_kind", 0)
    sc.source.kind = kind
    rc, h, L = _create(sc, **kw)
    assert rc == (B.SIM_EUNSUPPORTED if kind else B.SIM_EINVAL), L.sim_last_error(None)
    assert not h.value


def test_error_strings():
    L = B.lib()
    for c in (0, -1, -2, -3, -4, -5, -6):
        assert L.sim_error_string(c)


def _refined(nth=16, nr=16):
    g = W.Grid(nr=nr, nth=nth, nz=16, pml_r=2, pml_z=2, dr=0.005, dz=0.005)
    return W.Scenario("tiny", W.cased_well(g, z_top=0.04, casing_in=0.02, casing_t=0.005, cement_out=0.03),
                      W.Source(z=0.03), W.on_axis_receivers([0.05]), steps=10)


@pytest.mark.parametrize("rows,kw,code", [
    ([4, 8], dict(storage="bf16"), B.SIM_EUNSUPPORTED),   # FP32 only
    ([4, 8], dict(kernel="fused"), B.SIM_EUNSUPPORTED),   # split kernels only
    ([8, 4], {}, B.SIM_EINVAL),                           # interface rows not increasing
    ([1, 8], {}, B.SIM_EINVAL),                           # one-row zone
    ([4, 15], {}, B.SIM_EINVAL),                          # interface inside the radial PML
    ([2, 4, 8], {}, B.SIM_EINVAL),                        # 16 / 2^3 = 2 nodes in zone 0
    ([4, 8], dict(source_kind=3, source_r=0.02), B.SIM_EUNSUPPORTED),  # torsion ring on a zone's first row
    ([4, 8], dict(nth=24), B.SIM_EINVAL),                 # nth not a power of two
    ([4, 8], dict(source_kind=1, source_r=0.02), B.SIM_EUNSUPPORTED),  # force node on a zone's first row
    ([4, 8], dict(watchdog_every=10), B.SIM_EUNSUPPORTED),  # no watchdog on the refined grid
    ([4, 8], dict(tile=2004), B.SIM_EINVAL),              # zones run 22xx / 23xx split codes only
])
def test_refined_grid_host_validation(rows, kw, code):
    """simr_create checks its zones, storage, kernel and source on the host
    before any device call."""
    kw = dict(kw)
    sc = _refined(nth=kw.pop("nth", 16))
    sc.source.kind = kw.pop("source_kind", 0)
    sc.source.r = kw.pop("source_r", 0.0)
    L = B.lib()
    (g, m, s, r, o), keep = B.make_structs(sc, **kw)
    arr = (ctypes.c_int * len(rows))(*rows)
    z = B.SimZones(len(rows) + 1, arr)
    h = ctypes.c_void_p()
    rc = L.simr_create(ctypes.byref(g), ctypes.byref(z), ctypes.byref(m), ctypes.byref(s), ctypes.byref(r),
                       ctypes.byref(o), ctypes.byref(h))
    assert rc == code, L.simr_last_error(None)
    assert not h.value
    assert L.simr_last_error(None)
