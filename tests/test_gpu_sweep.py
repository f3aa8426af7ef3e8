"""The single-pass sweep kernel (one persistent launch per step that sweeps
z in chunks of 32 or 64 cells spanning every (theta, r) row: the velocity
items of chunk c + L and the stress items of chunk c alternate, so the stress
items find their inputs in L2) against the FP64 oracle, and its bounded waits.

* Every tile code, element by element on every field, on grids whose NZ
  (a ragged last chunk, fewer chunks than the lag, a single chunk), row count
  nth x NR (items of 16 or 8 rows straddling theta) and PML are uneven.
* The cased well with PML: traces and fields.
* The give-up path: a chunk whose velocity items never report makes the
  stress items that need it wait out a short limit; the step reports
  SIM_ETIMEOUT, no fault, and a fresh handle on the same device matches the
  oracle again.
"""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import rel_l2
from tests.test_gpu_parity import TRACE_TOL, _ragged_scenario, sim

pytestmark = pytest.mark.gpu

SWEEP_TILES = (3043, 3024, 3143, 3124, 3243, 3224, 3343, 3324, 3443, 3424, 3543, 3524)


def _fields_match(s, o, tol=2e-5):
    for n in oracle.FIELDS:
        a, b = s.field(n), o.field(n)
        scale = np.abs(b).max()
        assert scale > 0, n
        assert np.abs(a - b).max() <= tol * scale, (n, np.abs(a - b).max() / scale)


@pytest.mark.parametrize("tile", SWEEP_TILES)
@pytest.mark.parametrize("seed,nth,nr,nz", [(6, 12, 14, 301), (9, 6, 5, 250), (10, 10, 4, 77), (11, 4, 21, 130),
                                            (14, 8, 9, 20)])
def test_sweep_every_tile_fields_elementwise(tile, seed, nth, nr, nz):
    sc = _ragged_scenario(seed=seed, nth=nth, nr=nr, nz=nz)
    if nz < 30:  # a short well (one 32-cell chunk): source and receivers inside
        sc.source.z = 0.03
        sc.receivers = W.Receivers(r=np.array([0.0, 0.013]), theta=np.array([0.0, 1.1]), z=np.array([0.01, 0.05]))
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="sweep", tile=tile) as s:
        assert s.config() == (5, tile)
        s.step(sc.steps)
        _fields_match(s, o)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL


@pytest.mark.parametrize("tile", SWEEP_TILES)
def test_sweep_two_rows(tile):
    """NR = 2 (no PML), 44 z cells: two chunks of 32 (one of 64), fewer
    chunks than the lag, so every velocity item precedes every stress item."""
    g = W.Grid(nr=2, nth=4, nz=40, pml_r=0, pml_z=2, dr=0.004, dz=0.003)
    med = W.layered_radial(g, [0.004], [W.FLUID, W.STEEL])
    sc = W.Scenario("two rows", med, W.Source(z=0.05, f0=60e3), W.on_axis_receivers([0.03, 0.09]), steps=150)
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="sweep", tile=tile) as s:
        s.step(sc.steps)
        for n in ("vr", "vz", "srr", "spp", "szz"):
            a, b = s.field(n), o.field(n)
            scale = np.abs(b).max()
            assert scale > 0, n
            assert np.abs(a - b).max() <= 2e-5 * scale, (n, np.abs(a - b).max() / scale)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL


@pytest.mark.parametrize("tile", SWEEP_TILES)
def test_sweep_on_config1(tile):
    sc = W.config1(steps=500)
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="sweep", tile=tile) as s:
        s.step(sc.steps)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL
        for n in ("vr", "vz", "srr", "srz", "spp"):
            assert rel_l2(s.field(n), o.field(n)) <= TRACE_TOL, n


def test_sweep_equals_split_and_is_deterministic():
    """The sweep and split kernels run the same cell bodies: fields agree to
    FP32 rounding, and two sweep runs agree bit for bit (no item's result
    depends on the order blocks run in)."""
    sc = _ragged_scenario(seed=12, nth=16, nr=20, nz=400)
    with sim(sc, kernel="split", tile=2004) as a, sim(sc, kernel="sweep", tile=3043) as b, \
            sim(sc, kernel="sweep", tile=3043) as c:
        for h in (a, b, c):
            h.step(150)
        for n in oracle.FIELDS:
            x, y, z = a.field(n), b.field(n), c.field(n)
            assert np.array_equal(y, z), n
            assert rel_l2(y, x) <= 1e-6, n


def test_sweep_wait_gives_up_and_reports_timeout():
    """Withhold the velocity reports of one z chunk with a short wait limit:
    the stress items of the three chunks around it give up, the step ends (no
    hang, no fault) and sim_sync reports SIM_ETIMEOUT.  A new handle on the
    same device then matches the oracle."""
    from paper_2302_13907_gb300.binding import SIM_ETIMEOUT, SimError
    sc = _ragged_scenario(seed=13, nth=8, nr=12, nz=200)
    with sim(sc, kernel="sweep", tile=3043, graph_chunk=-1) as s:
        s.step(3)
        s.sync()
        s.set_wait_test(200000, 3)  # chunk 3 of 7 (cells 96 .. 127); ~0.1 ms per wait
        s.step(2)
        with pytest.raises(SimError) as ei:
            s.sync()
        assert ei.value.code == SIM_ETIMEOUT
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="sweep", tile=3043) as s2:
        s2.step(sc.steps)
        _fields_match(s2, o)
