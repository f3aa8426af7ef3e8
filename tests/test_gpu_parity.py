"""GPU parity: the CUDA simulator (through the C-ABI) against the FP64 oracle.

Bar (FP32 arithmetic against FP64): receiver-trace relative L2 <= 1e-4 over
all receivers and steps concatenated; fields compared element by element on
small grids that span several kernel tiles and a ragged z tail.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import energy, node_coefficients, random_admissible_state, rel_l2

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4


def sim(sc, **kw):
    from paper_2302_13907_gb300.binding import Simulation
    return Simulation(sc, **kw)


def _ragged_scenario(seed=0, nth=6, nr=9, pml_r=3, nz=37, pml_z=3):
    """Random heterogeneous medium (liquid ring 0) on a grid whose NZ is not a
    multiple of 4 or 32, with an off-axis source and off-axis receivers."""
    g = W.Grid(nr=nr, nth=nth, nz=nz, pml_r=pml_r, pml_z=pml_z, dr=0.004, dz=0.003)
    rng = np.random.default_rng(seed)
    mats = [W.FLUID, W.STEEL, W.CEMENT, W.ROCK, (2000.0, 2500.0, 0.0)]
    cid = rng.integers(0, len(mats), size=g.shape).astype(np.uint16)
    cid[:, 0, :] = 0
    med = W.Medium(g, cid, np.array([m[0] for m in mats]), np.array([m[1] for m in mats]),
                   np.array([m[2] for m in mats]))
    rec = W.Receivers(r=np.array([0.0, 0.013, 0.0155]), theta=np.array([0.0, 1.1, 4.0]),
                      z=np.array([0.02, 0.05, 0.09]))
    return W.Scenario("ragged", med, W.Source(r=0.014, theta=2.0, z=0.06, f0=60e3), rec, steps=200)


@pytest.mark.parametrize("kernel", ["split", "fused", "fused4", "march", "sweep"])
def test_config1_traces_match_oracle(kernel):
    sc = W.config1()
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    ref = o.traces()
    with sim(sc, kernel=kernel) as s:
        assert s.dt == pytest.approx(o.dt, rel=1e-15)
        s.step(sc.steps)
        got = s.traces()
        assert got.shape == ref.shape
        err = rel_l2(got, ref)
        assert err <= TRACE_TOL, err
        for n in ("vr", "vz", "srr", "srz"):
            assert rel_l2(s.field(n), o.field(n)) <= TRACE_TOL, n


def test_config1_long_window_traces_match_oracle():
    """4000 steps: the cement-top reflection is inside the window."""
    sc = W.config1_long()
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    ref = o.traces()
    with sim(sc) as s:
        s.step(sc.steps)
        got = s.traces()
    assert rel_l2(got, ref) <= TRACE_TOL
    for q in range(ref.shape[0]):
        if np.abs(ref[q]).max() > 1e-6 * np.abs(ref).max():
            assert rel_l2(got[q], ref[q]) <= 10 * TRACE_TOL, q


@pytest.mark.parametrize("kernel", ["split", "fused", "fused4", "march", "sweep"])
@pytest.mark.parametrize("seed,nth,nr,nz", [(0, 6, 9, 37), (1, 4, 5, 70), (2, 8, 13, 2), (3, 4, 40, 131),
                                            (4, 10, 29, 190)])
def test_ragged_grid_fields_elementwise(kernel, seed, nth, nr, nz):
    sc = _ragged_scenario(seed=seed, nth=nth, nr=nr, nz=nz)
    if nz < 20:  # tiny z: keep source / receivers inside
        sc.source.z = 0.0
        sc.receivers = W.Receivers(r=np.array([0.0]), theta=np.array([0.0]), z=np.array([0.0]))
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel=kernel) as s:
        s.step(sc.steps)
        for n in oracle.FIELDS:
            a, b = s.field(n), o.field(n)
            scale = np.abs(b).max()
            if scale == 0:
                assert np.abs(a).max() == 0, n
                continue
            assert np.abs(a - b).max() <= 2e-5 * scale, (n, np.abs(a - b).max() / scale)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL


def _torsion_scenario():
    """Small cased section (liquid, steel, rock) with the torsion ring in the steel."""
    g = W.Grid(nr=12, nth=6, nz=40, pml_r=3, pml_z=3, dr=0.004, dz=0.003)
    med = W.layered_radial(g, [0.016, 0.032], [W.FLUID, W.STEEL, W.ROCK])
    rec = W.Receivers(r=np.array([0.0, 0.026]), theta=np.array([0.0, 1.0]), z=np.array([0.03, 0.06]))
    return W.Scenario("torsion", med, W.Source(kind=W.SOURCE_TORSION, r=0.024, z=0.05, f0=60e3), rec, steps=200)


@pytest.mark.parametrize("kernel", ["split", "march", "sweep"])
@pytest.mark.parametrize("kind,r,theta", [(1, 0.0, 0.7), (1, 0.013, 1.1), (2, 0.0, 0.0), (2, 0.014, 2.0),
                                          (3, 0.024, 0.0)])
def test_point_forces_and_torsion_fields_elementwise(kernel, kind, r, theta):
    """The transverse and longitudinal point forces (on and off the axis)
    and the torsion ring, injected between the half-steps, against the
    oracle element by element on every field (the sweep kernel fuses the
    half-steps: the torsion ring only, the forces are refused)."""
    if kernel == "sweep" and kind != 3:
        from paper_2302_13907_gb300.binding import SIM_EUNSUPPORTED, SimError
        sc = _ragged_scenario(seed=7, nth=8, nr=11, nz=45)
        sc.source = W.Source(kind=kind, r=r, theta=theta, z=0.06, f0=60e3)
        with pytest.raises(SimError) as ei:
            sim(sc, kernel=kernel)
        assert ei.value.code == SIM_EUNSUPPORTED
        return
    if kind == 3:
        sc = _torsion_scenario()
    else:
        sc = _ragged_scenario(seed=7, nth=8, nr=11, nz=45)
        sc.source = W.Source(kind=kind, r=r, theta=theta, z=0.06, f0=60e3)
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel=kernel) as s:
        s.step(sc.steps)
        for n in oracle.FIELDS:
            a, b = s.field(n), o.field(n)
            scale = np.abs(b).max()
            if scale == 0:
                assert np.abs(a).max() == 0, n
                continue
            assert np.abs(a - b).max() <= 2e-5 * scale, (n, np.abs(a - b).max() / scale)
        tr, ref = s.traces(), o.traces()
        if np.abs(ref).max() > 0:
            assert rel_l2(tr, ref) <= TRACE_TOL


def test_energy_conserved_fp32_pml_off():
    g = W.Grid(nr=40, nth=8, nz=60, pml_r=0, pml_z=0, dr=0.005, dz=0.005)
    med = W.cased_well(g, z_top=0.15)
    f, coef = random_admissible_state(med, seed=7)
    sc = W.Scenario("e", med, W.Source(z=0.1, amplitude=0.0), W.on_axis_receivers([0.1]), steps=2000, pml_on=False)
    with sim(sc, pml_on=False, graph_chunk=-1) as s:
        for n, a in f.items():
            s.set_field(n, a)
        E = []
        v_old = {n: s.field(n).astype(np.float64) for n in ("vr", "vp", "vz")}
        for it in range(6):
            s_now = {n: s.field(n).astype(np.float64) for n in ("srr", "spp", "szz", "srp", "spz", "srz")}
            s.step(1)
            v_new = {n: s.field(n).astype(np.float64) for n in ("vr", "vp", "vz")}
            E.append(energy(coef, g, v_old, v_new, s_now))
            s.step(399)
            v_old = {n: s.field(n).astype(np.float64) for n in ("vr", "vp", "vz")}
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-5, E


def test_axisymmetric_theta_independent_bitwise():
    sc = W.config1(steps=300)
    with sim(sc) as s:
        s.step(300)
        for n in ("vp", "srp", "spz"):
            assert np.all(s.field(n) == 0), n
        for n in ("vr", "vz", "srr", "spp", "szz", "srz"):
            a = s.field(n)
            assert np.abs(a).max() > 0
            assert np.array_equal(a, np.broadcast_to(a[:1], a.shape)), n


def test_graph_chunks_equal_single_steps_and_deterministic():
    sc = W.config1(steps=200)
    with sim(sc, graph_chunk=64) as a:
        a.step(200)
        ta = a.traces()
        fa = a.field("srr")
    with sim(sc, graph_chunk=-1) as b:
        for _ in range(200):
            b.step(1)
        tb = b.traces()
        fb = b.field("srr")
    assert np.array_equal(ta, tb) and np.array_equal(fa, fb)
    with sim(sc, graph_chunk=37) as c:
        c.step(13)
        c.step(0)
        c.step(187)
        assert np.array_equal(c.traces(), ta)


def test_zero_steps_and_empty_receivers():
    sc = W.config1(steps=10)
    sc.receivers = W.Receivers(r=np.zeros(0), theta=np.zeros(0), z=np.zeros(0))
    with sim(sc) as s:
        s.step(0)
        assert s.traces().shape == (0, 0)
        s.step(10)
        assert s.traces().shape == (0, 10)
        assert s.steps_done == 10


def test_checkpoint_resume_bitwise():
    sc = W.config1(steps=120)
    with sim(sc) as a:
        a.step(120)
        ref = a.traces()
        ref_f = a.field("vz")
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        with sim(sc) as b:
            b.step(50)
            b.save(path)
        with sim(sc) as c:
            c.load(path)
            assert c.steps_done == 50
            c.step(70)
            assert np.array_equal(c.traces(), ref)
            assert np.array_equal(c.field("vz"), ref_f)


def test_checkpoint_resume_bitwise_with_stochastic_rounding_and_watchdog():
    """FP16 storage with stochastic rounding: the dithers are keyed on the
    device step counter, which the checkpoint carries, so the resumed run
    repeats the uninterrupted one bit for bit, and the watchdog's energy
    proxy after it equals the uninterrupted run's."""
    sc = W.config1(steps=120)
    kw = dict(storage="f16sr", watchdog_every=10)
    with sim(sc, **kw) as a:
        a.step(120)
        ref, ref_f, ref_w = a.traces(), a.field("srr"), a.watchdog()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        with sim(sc, **kw) as b:
            b.step(50)
            b.save(path)
        with sim(sc, **kw) as c:
            c.load(path)
            c.step(70)
            assert np.array_equal(c.traces(), ref)
            assert np.array_equal(c.field("srr"), ref_f)
            e, r, n = c.watchdog()
            assert n == 120 and e == pytest.approx(ref_w[0], rel=1e-12)
            c.sync()


def test_trace_capacity_and_stepping_beyond():
    sc = W.config1(steps=800)
    o = oracle.Oracle(sc)
    o.step(300)
    with sim(sc, max_steps=100) as s:
        s.step(300)
        t = s.traces()
        assert t.shape == (4, 100)
        assert rel_l2(s.field("srr"), o.field("srr")) <= TRACE_TOL


def test_unstable_dt_is_reported_not_faulted():
    from paper_2302_13907_gb300.binding import SimError, SIM_EUNSTABLE
    sc = W.config1(steps=3000)
    sc.cfl = 3.0
    with sim(sc) as s:
        s.step(3000)
        with pytest.raises(SimError) as ei:
            s.sync()
        assert ei.value.code == SIM_EUNSTABLE


def test_memory_cap_is_enforced():
    from paper_2302_13907_gb300.binding import SimError, SIM_ENOMEM
    with pytest.raises(SimError) as ei:
        sim(W.config1(), mem_cap=1 << 20)
    assert ei.value.code == SIM_ENOMEM


def test_full_size_well_sampled_against_oracle_crop():
    """The 196 x 64 x 8224 well in the benchmark's launch configuration:
    after 32 steps the field is confined within 64 cells of the source, so
    the oracle on a z crop around the source computes those outputs exactly."""
    sc = W.config2()
    g = sc.grid
    n = 32  # two cells of reach per step: 64 < 96-cell margin
    with sim(sc, max_steps=n, graph_chunk=16) as s:
        s.step(n)
        full = {q: s.field(q) for q in ("vz", "srr", "srz", "vr")}
        dt = s.dt
    ks = int(round(sc.source.z / g.dz)) + g.pml_z
    lo, hi = ks - 96, ks + 96
    crop = W.crop_z(sc.medium, lo, hi - lo - 2 * g.pml_z)
    sc_c = W.Scenario("crop", crop, W.Source(z=sc.source.z - lo * g.dz, f0=sc.source.f0),
                      W.on_axis_receivers([sc.source.z - lo * g.dz]), steps=n)
    o = oracle.Oracle(sc_c, dt=dt)
    o.step(n)
    for q, a in full.items():
        b = o.field(q)
        sub = a[:, :, lo + 8:hi - 8]
        ref = b[:, :, 8:-8]
        assert np.abs(a[:, :, : lo]).max() == 0 and np.abs(a[:, :, hi:]).max() == 0, q
        if np.abs(ref).max() == 0:  # e.g. shear stress next to the source, all liquid
            assert np.abs(sub).max() == 0, q
            continue
        assert rel_l2(sub, ref) <= TRACE_TOL, (q, rel_l2(sub, ref))


MARCH_TILES = (1216, 1232, 1264, 1416, 1432, 1464, 1816, 1832, 1864)


@pytest.mark.parametrize("tile", MARCH_TILES)
def test_march_every_tile_fields_elementwise(tile):
    """The marching kernels at every tile code the autotuner may pick, on a
    grid where neither Ntheta (runs of 16 / 32 / 64 planes), NR (tiles of
    2 / 4 / 8 rows) nor NZ (tiles of 128) divides evenly, with an off-axis
    source: every field against the oracle element by element."""
    sc = _ragged_scenario(seed=5, nth=40, nr=14, nz=150)
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="march", tile=tile) as s:
        assert s.config() == (4, tile)
        s.step(sc.steps)
        for n in oracle.FIELDS:
            a, b = s.field(n), o.field(n)
            scale = np.abs(b).max()
            assert scale > 0, n
            assert np.abs(a - b).max() <= 2e-5 * scale, (n, np.abs(a - b).max() / scale)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL


SPLIT_TILES = (2000, 2003, 2004, 2005, 2013, 2014, 2106, 2108, 2204, 2205, 2216, 2218, 2224, 2225, 2234, 2235,
               2244, 2245, 2256, 2258, 2264, 2265, 2274, 2275, 2284, 2285, 2294, 2295,
               2304, 2305, 2314, 2315, 2324, 2325, 2334, 2335)


@pytest.mark.parametrize("tile", SPLIT_TILES)
def test_split_variants_fields_elementwise(tile):
    """The split kernels and their load-first variants (every register
    budget, cells per thread and interior / edge split the autotuner may
    pick) on an uneven grid: every field against the oracle element by
    element.  NZ = 307 and NR = 17 leave interior tiles for both the
    four- and the two-cells-per-thread split launches, edge tiles in the
    radial PML, at both z ends and in a ragged z tail."""
    sc = _ragged_scenario(seed=6, nth=12, nr=14, nz=301)
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="split", tile=tile) as s:
        assert s.config() == (1, tile)
        s.step(sc.steps)
        for n in oracle.FIELDS:
            a, b = s.field(n), o.field(n)
            scale = np.abs(b).max()
            assert scale > 0, n
            assert np.abs(a - b).max() <= 2e-5 * scale, (n, np.abs(a - b).max() / scale)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL


@pytest.mark.parametrize("tile", (2204, 2205, 2216, 2218, 2224, 2235, 2244, 2258, 2264, 2275, 2285, 2294, 2305, 2314))
def test_interior_edge_split_on_config1(tile):
    """The interior / edge split launches on the cased-well geometry, where
    most tiles are interior: traces and fields against the oracle."""
    sc = W.config1(steps=300)
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with sim(sc, kernel="split", tile=tile) as s:
        assert s.config() == (1, tile)
        s.step(sc.steps)
        assert rel_l2(s.traces(), o.traces()) <= TRACE_TOL
        for n in ("vr", "vz", "srr", "srz", "spp"):
            assert rel_l2(s.field(n), o.field(n)) <= TRACE_TOL, n


def test_split_pair_code_runs_two_variants():
    """A pair code v * 10000 + s runs the velocity kernel of split code v and
    the stress kernel of split code s; the scheme is the same, so the fields
    agree with a single code to FP32 rounding."""
    sc = _ragged_scenario(seed=8, nth=10, nr=14, nz=301)
    with sim(sc, kernel="split", tile=2004) as a, sim(sc, kernel="split", tile=22052204) as b:
        assert b.config() == (1, 22052204)
        a.step(150)
        b.step(150)
        for n in ("vr", "vp", "vz", "srr", "srz", "spz"):
            x = a.field(n)
            assert rel_l2(b.field(n), x) <= 1e-6, n
    from paper_2302_13907_gb300.binding import SIM_EINVAL, SimError
    with pytest.raises(SimError) as ei:
        sim(sc, kernel="split", tile=22072204)  # 2207 is not a split code
    assert ei.value.code == SIM_EINVAL


def test_march_rejects_a_tile_it_does_not_have():
    from paper_2302_13907_gb300.binding import SIM_EINVAL, SimError
    with pytest.raises(SimError) as ei:
        sim(W.config1(steps=4), kernel="march", tile=1234)
    assert ei.value.code == SIM_EINVAL


def test_fused_matches_split_and_autotuner_choice():
    """The fused (time-skewed, TMA-staged) kernel and the split kernels
    compute the same scheme: traces agree to FP32 rounding; every tile
    height the autotuner may pick gives the same answer."""
    sc = W.config1(steps=400)
    with sim(sc, kernel="split", tile=2000) as a:
        a.step(400)
        ta = a.traces()
        fa = {n: a.field(n) for n in ("vr", "srr", "srz")}
    for kern, kind_want, tiles in (("fused", 2, (2, 4, 6, 8)), ("fused4", 2, (106, 110, 114)),
                                   ("march", 4, MARCH_TILES), ("split", 1, SPLIT_TILES),
                                   ("sweep", 5, (3043, 3024, 3143, 3124, 3243, 3224, 3343, 3324, 3443, 3424, 3543, 3524))):
        with sim(sc, kernel=kern) as b:
            kind, tile = b.config()
            halves = (tile // 10000, tile % 10000) if tile >= 10000 else (tile, tile)
            assert kind == kind_want and all(t in tiles for t in halves), (kern, kind, tile)
            b.step(400)
            tb = b.traces()
            assert rel_l2(tb, ta) <= 1e-6, kern
            for n, x in fa.items():
                assert rel_l2(b.field(n), x) <= 1e-6, (kern, n)
