"""GPU parity of the azimuthally refined grid (Sec. 3; reading R14) through
the C-ABI (simr_*), against the refined FP64 oracle: every field of every
zone element by element, and the receiver traces.

Cases: an uneven heterogeneous grid (random materials outside a liquid ring
0, NZ not a multiple of 4 or 32, NR not a multiple of the 4-row tiles) with
two and three interfaces, the volumetric source on and off the axis and the
transverse force on and off the axis; a one-zone grid against the uniform
simulator; and the 20 m well's full radius and azimuth (zones 4 / 8 / 16 / 32
/ 64 nodes by the paper's rule) on a z-crop the oracle finishes in seconds.
"""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4
FIELD_TOL = 2e-5


def _ragged(seed=0, nth=16, nr=14, nz=61, kind=0, src_r=0.0, steps=200):
    g = W.Grid(nr=nr, nth=nth, nz=nz, pml_r=3, pml_z=3, dr=0.004, dz=0.003)
    rng = np.random.default_rng(seed)
    mats = [W.FLUID, W.STEEL, W.CEMENT, W.ROCK, (2000.0, 2500.0, 0.0)]
    cid = rng.integers(0, len(mats), size=g.shape).astype(np.uint16)
    cid[:, 0, :] = 0
    med = W.Medium(g, cid, np.array([m[0] for m in mats]), np.array([m[1] for m in mats]),
                   np.array([m[2] for m in mats]))
    rec = W.Receivers(r=np.array([0.0, 0.013, 0.0255, 0.045]), theta=np.array([0.0, 1.1, 4.0, 2.2]),
                      z=np.array([0.02, 0.05, 0.09, 0.12]))
    src = W.Source(r=src_r, theta=2.0, z=0.06, f0=60e3, kind=kind)
    return W.Scenario("ragged-refined", med, src, rec, steps=steps)


def _compare(sc, rows, steps, tile=0):
    from paper_2302_13907_gb300.binding import RefinedSimulation
    o = oracle.RefinedOracle(sc, rows=rows)
    o.step(steps)
    with RefinedSimulation(sc, rows, graph_chunk=32, tile=tile) as s:
        assert s.dt == pytest.approx(o.dt, rel=1e-15)
        assert [z[:3] for z in o.zones] == s.zones
        s.step(steps)
        got = s.traces()
        ref = o.traces()
        assert got.shape == ref.shape
        if np.abs(ref).max() == 0:  # a torsion field has no pressure at all
            assert np.abs(got).max() == 0
        else:
            assert rel_l2(got, ref) <= TRACE_TOL, rel_l2(got, ref)
        # each field against the largest magnitude of its kind (velocities,
        # stresses): a monopole leaves v_phi, s_rphi, s_phiz at rounding level
        kind_scale = {}
        for n in oracle.FIELDS:
            kind = n[0]
            kind_scale[kind] = max(kind_scale.get(kind, 0.0), max(np.abs(o.field(n, z)).max() for z in range(o.M)))
        for n in oracle.FIELDS:
            scale = kind_scale[n[0]]
            for z in range(o.M):
                a, b = s.field(n, z), o.field(n, z)
                assert np.abs(a - b).max() <= FIELD_TOL * scale, (n, z, np.abs(a - b).max() / scale)
        return s.cells


@pytest.mark.parametrize("rows", [[4, 8], [3, 6, 10]])
@pytest.mark.parametrize("kind,src_r", [(0, 0.0), (0, 0.0305), (1, 0.0), (1, 0.0205)])
def test_refined_fields_elementwise(rows, kind, src_r):
    nth = 16 if len(rows) == 2 else 32
    sc = _ragged(seed=4, nth=nth, kind=kind, src_r=src_r)
    cells = _compare(sc, rows, steps=160)
    g = sc.medium.grid
    row0 = [0] + rows + [g.NR]
    M = len(rows) + 1
    assert cells == sum((nth >> (M - 1 - m)) * (row0[m + 1] - row0[m]) * g.NZ for m in range(M))


@pytest.mark.parametrize("tile", [2204, 22852324, 23342305])
def test_refined_zones_on_other_split_codes(tile):
    """opts.tile of a refined handle: every zone's halves on the split code(s)
    named (interior / edge and three-way, one code or a pair), against the
    oracle as above."""
    sc = _ragged(seed=5, nth=16, kind=0, src_r=0.0305)
    _compare(sc, [4, 8], steps=120, tile=tile)


def test_single_zone_equals_uniform_simulator():
    from paper_2302_13907_gb300.binding import RefinedSimulation, Simulation
    sc = _ragged(seed=9, nth=12, kind=1, src_r=0.0205)
    with Simulation(sc, kernel="split", tile=2004) as u, RefinedSimulation(sc, []) as r:
        u.step(150)
        r.step(150)
        assert rel_l2(r.traces(), u.traces()) < 1e-6
        for n in ("vr", "vp", "srr", "srz"):
            assert rel_l2(r.field(n, 0), u.field(n)) < 1e-6, n


def test_refined_20m_well_full_radius_on_a_z_crop():
    """The 20 m well's full radius and azimuth, zones by the paper's rule,
    on a 192-cell z-crop around the source: GPU against the oracle."""
    full = W.config2()
    g = full.medium.grid
    rows = W.refinement_rows(g)
    assert rows == [12, 24, 49, 98]
    ks = int(round(full.source.z / g.dz))
    k0 = ks - 96
    crop = W.crop_z(full.medium, k0, 192)
    zs = full.source.z - k0 * g.dz
    sc = W.Scenario("crop", crop, W.Source(z=zs, f0=full.source.f0),
                    W.Receivers(r=np.array([0.0, 0.1, 0.3]), theta=np.array([0.0, 1.0, 2.5]),
                                z=np.array([zs - 0.1, zs, zs + 0.15])), cfl=full.cfl, steps=300)
    u = oracle.Oracle(sc, max_steps=1)
    o_dt = oracle.RefinedOracle(sc, rows=rows, max_steps=1).dt
    assert o_dt > 3 * u.dt  # the axis no longer sets the step: ~3.6x
    _compare(sc, rows, steps=300)


@pytest.mark.parametrize("kind,r0", [(2, 0.0), (2, 0.0305), (3, 0.046)])
def test_refined_longitudinal_force_and_torsion_ring(kind, r0):
    """The longitudinal force (on and off the axis) and the torsion ring in
    the casing of a cased well on a refined grid: every field of every zone
    against the refined oracle."""
    g = W.Grid(nr=24, nth=16, nz=61, pml_r=4, pml_z=4, dr=0.004, dz=0.003)
    med = W.cased_well(g, z_top=0.08, casing_in=0.04, casing_t=0.012, cement_out=0.06)
    rec = W.Receivers(r=np.array([0.0, 0.021, 0.061]), theta=np.array([0.0, 0.4, 2.0]),
                      z=np.array([0.05, 0.1, 0.12]))
    sc = W.Scenario("refined-sources", med, W.Source(r=r0, theta=0.7, z=0.08, f0=60e3, kind=kind), rec, steps=160)
    _compare(sc, [4, 8], steps=160)
