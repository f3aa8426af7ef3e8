"""Pins of the oracle's azimuthally refined grid (Sec. 3, "Azimuth grid
refinement"; reading R14), each against something other than the oracle's
own code:

* the interpolation reproduces band-limited trigonometric polynomials
  exactly at the fine nodes, for both azimuthal staggerings (the exactness
  the paper cites FFT interpolation for);
* its matrix keeps constants and the coarse values at coinciding nodes;
* a grid of one zone is the uniform grid: the pinned uniform oracle's
  fields, to rounding;
* an axisymmetric problem does not depend on the azimuthal step at all, so
  the refined grid reproduces the uniform one at every node it has;
* the discrete energy of the scheme (tests/helpers.py, written from the
  definition) stays constant across interfaces: the fine-to-coarse map is
  the adjoint of the coarse-to-fine one;
* a dipole (m = 1) source on a refined grid stays close to the uniform
  fine grid.
"""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import energy_refined, refined_coefficients, rel_l2

FIELDS = oracle.FIELDS
HALF = ("vp", "srp", "spz")


@pytest.mark.parametrize("na", [4, 8, 16, 32])
@pytest.mark.parametrize("half", [False, True])
def test_interpolation_exact_on_trig_polynomials(na, half):
    nb = 2 * na
    rng = np.random.default_rng(na + 100 * half)
    off = 0.5 if half else 0.0
    ta = (np.arange(na) + off) * 2 * np.pi / na
    tb = (np.arange(nb) + off) * 2 * np.pi / nb
    for m in range(0, na // 2):
        a0, b0 = rng.standard_normal(2)
        f = lambda t: a0 * np.cos(m * t) + b0 * np.sin(m * t)
        got = oracle.fft_interp(f(ta), nb, half)
        assert np.abs(got - f(tb)).max() < 1e-12 * max(1.0, abs(a0) + abs(b0)), (m, half)


def test_interpolation_nyquist_mode_is_the_cosine():
    """The Nyquist coefficient is split evenly, so the coarse grid-scale
    oscillation (-1)^j interpolates to cos(N/2 theta)."""
    na = 8
    got = oracle.fft_interp((-1.0) ** np.arange(na), 2 * na, False)
    want = np.cos(na / 2 * np.arange(2 * na) * 2 * np.pi / (2 * na))
    assert np.abs(got - want).max() < 1e-13


def _scenario(nr=24, nth=16, nz=40, pml_r=4, pml_z=4, kind=0, axis=True, seed=None, steps=120):
    g = W.Grid(nr=nr, nth=nth, nz=nz, pml_r=pml_r, pml_z=pml_z, dr=0.004, dz=0.004)
    med = W.cased_well(g, z_top=0.08)
    if seed is not None:  # a non-axisymmetric medium outside ring 0
        rng = np.random.default_rng(seed)
        mats = [W.FLUID, W.STEEL, W.CEMENT, W.ROCK]
        cid = rng.integers(0, len(mats), size=g.shape).astype(np.uint16)
        cid[:, 0, :] = 0
        med = W.Medium(g, cid, np.array([m[0] for m in mats]), np.array([m[1] for m in mats]),
                       np.array([m[2] for m in mats]))
    src = W.Source(r=0.0 if axis else 0.0305, theta=0.7, z=0.08, f0=60e3, kind=kind)
    rec = W.Receivers(r=np.array([0.0, 0.021, 0.061]), theta=np.array([0.0, 0.4, 2.0]),
                      z=np.array([0.05, 0.1, 0.12]))
    return W.Scenario("refine", med, src, rec, steps=steps)


def test_matrix_keeps_constants_and_coinciding_nodes():
    o = oracle.RefinedOracle(_scenario(), rows=[6, 12])
    for m in (1, 2):
        Pi, Ph = o.matrix(m, False), o.matrix(m, True)
        assert np.abs(Pi.sum(axis=1) - 1).max() < 1e-13
        assert np.abs(Ph.sum(axis=1) - 1).max() < 1e-13
        na = Pi.shape[1]
        assert np.abs(Pi[0::2] - np.eye(na)).max() < 1e-13  # even fine nodes are coarse nodes


@pytest.mark.parametrize("kind,axis", [(0, False), (1, True), (1, False)])
def test_single_zone_is_the_uniform_oracle(kind, axis):
    sc = _scenario(kind=kind, axis=axis, seed=3)
    u = oracle.Oracle(sc)
    r = oracle.RefinedOracle(sc, rows=[])
    assert r.dt == u.dt
    u.step(80)
    r.step(80)
    for n in FIELDS:
        a, b = r.field(n, 0), u.field(n)
        assert np.abs(a - b).max() <= 1e-13 * max(np.abs(b).max(), 1e-300), n
    assert np.abs(r.traces() - u.traces()).max() <= 1e-13 * np.abs(u.traces()).max()


def test_axisymmetric_problem_reproduced_on_every_zone():
    """Monopole on the axis in an axisymmetric well: nothing depends on theta,
    so the coarse zones must carry exactly the uniform grid's values."""
    sc = _scenario(kind=0, axis=True)
    dt = oracle.Oracle(sc).dt
    u = oracle.Oracle(sc, dt=dt)
    r = oracle.RefinedOracle(sc, rows=[6, 12], dt=dt)
    u.step(150)
    r.step(150)
    vscale = max(np.abs(u.field(n)).max() for n in ("vr", "vz"))
    sscale = max(np.abs(u.field(n)).max() for n in ("srr", "spp", "szz", "srz"))
    for n in FIELDS:
        b = u.field(n)
        scale = vscale if n in ("vr", "vp", "vz") else sscale  # v_phi, s_rphi, s_phiz vanish
        for z, (row, rows, nth, _) in enumerate(r.zones):
            a = r.field(n, z)
            want = b[:: sc.medium.grid.nth // nth, row:row + rows, :]
            assert np.abs(a - want).max() <= 1e-11 * scale, (n, z, np.abs(a - want).max() / scale)
    assert rel_l2(r.traces(), u.traces()) < 1e-11


def test_cfl_uses_each_zone_azimuthal_step():
    """64 azimuthal nodes: the axis cells set the uniform grid's dt; with 8
    nodes in the innermost zone the steel casing sets it."""
    sc = _scenario(nth=64)
    u = oracle.Oracle(sc)
    r = oracle.RefinedOracle(sc, rows=[3, 6, 12])
    assert r.dt > 1.5 * u.dt, (r.dt, u.dt)
    assert r.dt == oracle.RefinedOracle(sc, rows=[3, 6, 12], pml_on=False).dt


def _admissible_zones(o, zcoef, seed):
    rng = np.random.default_rng(seed)
    NZ = o.grid.NZ
    for z, (row, n, nth, c) in enumerate(zcoef):
        f = {k: rng.standard_normal((nth, n, NZ)) for k in FIELDS}
        for k in ("vr", "vp", "vz"):
            f[k] *= 1e-3
        if row == 0:
            f["vr"][:, 0, :] = 0
        f["vz"][:, :, -1] = 0
        fluid = c["mu"] == 0
        f["spp"][fluid] = f["srr"][fluid]
        f["szz"][fluid] = f["srr"][fluid]
        f["srp"][c["mu_rp"] == 0] = 0
        f["srz"][c["mu_rz"] == 0] = 0
        f["spz"][c["mu_pz"] == 0] = 0
        for k in FIELDS:
            o.field(k, z)[...] = f[k]


@pytest.mark.parametrize("rows,nth", [([4, 10], 16), ([3, 7, 14], 32)])
def test_energy_conserved_across_interfaces(rows, nth):
    """PML off, random admissible state in every zone, 800 leapfrog steps:
    the discrete energy is constant to rounding."""
    sc = _scenario(nr=24, nth=nth, nz=40, pml_r=0, pml_z=0, seed=5)
    o = oracle.RefinedOracle(sc, rows=rows, max_steps=0, pml_on=False)
    zcoef = refined_coefficients(sc.medium, rows)
    _admissible_zones(o, zcoef, seed=11)
    M = o.M
    get = lambda names: {n: [o.field(n, z).copy() for z in range(M)] for n in names}
    E = []
    v_old = get(("vr", "vp", "vz"))
    for it in range(800):
        s_now = get(("srr", "spp", "szz", "srp", "spz", "srz"))
        o.velocity_update()
        v_new = get(("vr", "vp", "vz"))
        if it % 100 == 0 or it == 799:
            E.append(energy_refined(sc.medium.grid, zcoef, v_old, v_new, s_now))
        o.stress_update()
        v_old = v_new
    E = np.array(E)
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12, np.max(np.abs(E - E[0])) / E[0]


def test_dipole_on_refined_grid_close_to_uniform():
    """Transverse force on the axis (an m = 1 field): the refined grid's
    traces at off-axis receivers stay within a few per cent of the uniform
    fine grid's (the coarse zones have fewer azimuthal nodes near the axis)."""
    sc = _scenario(nr=30, nth=32, nz=60, kind=1, axis=True, steps=400)
    u = oracle.Oracle(sc)
    r = oracle.RefinedOracle(sc, rows=[4, 8, 16], dt=u.dt)
    u.step(400)
    r.step(400)
    tu, tr = u.traces(), r.traces()
    for q in (1, 2):
        assert rel_l2(tr[q], tu[q]) < 0.08, (q, rel_l2(tr[q], tu[q]))


def _dirichlet(n, t):
    """Textbook periodic interpolation kernel of n (even) samples, Nyquist
    term halved: (1/n) [1 + 2 sum_{m=1}^{n/2-1} cos(m t) + cos(n t / 2)]."""
    m = np.arange(1, n // 2)
    return (1.0 + 2.0 * np.cos(np.outer(t, m)).sum(axis=1) + np.cos(0.5 * n * t)) / n


@pytest.mark.parametrize("na", [4, 8, 16, 32])
def test_interpolation_matrix_is_the_closed_form_kernel(na):
    """The oracle builds its coarse-to-fine matrix by running the three DFT
    steps on unit vectors; it must equal the closed-form interpolation kernel
    evaluated at the node offsets (integer nodes: (j' - 2j) h_B; half-integer
    nodes: (j' - 2j - 1/2) h_B)."""
    nb = 2 * na
    hb = 2 * np.pi / nb
    for half in (False, True):
        got = np.stack([oracle.fft_interp(np.eye(na)[j], nb, half) for j in range(na)], axis=1)
        jb, ja = np.meshgrid(np.arange(nb), np.arange(na), indexing="ij")
        want = _dirichlet(na, ((jb - 2 * ja - (0.5 if half else 0.0)) * hb).ravel()).reshape(nb, na)
        assert np.abs(got - want).max() < 1e-13, (na, half)


def test_zoning_rule_halves_the_step_each_time_the_radius_doubles():
    """workloads.refinement_rows: going inward from the outer radius, zone
    boundaries where the radius halves, node counts halving down to 4."""
    g = W.Grid(nr=180, nth=64, nz=8, pml_r=16, pml_z=2, dr=0.0025, dz=0.0025)
    rows = W.refinement_rows(g)
    assert rows == [12, 24, 49, 98]
    edges = [0] + rows + [g.NR]
    nths = [g.nth >> (len(rows) - m) for m in range(len(rows) + 1)]
    assert nths == [4, 8, 16, 32, 64]
    for m in range(1, len(rows)):
        assert abs(edges[m + 1] / edges[m] - 2.0) < 0.1  # each zone spans one doubling of the radius
    # every zone's azimuthal cell size at its outer edge is within 2x of the
    # outer zone's at its inner edge (the purpose of the rule)
    size = [(edges[m + 1] * g.dr) * 2 * np.pi / nths[m] for m in range(len(nths))]
    assert max(size) / min(size) < 2.2
    assert W.refinement_rows(W.Grid(nr=20, nth=8, nz=8, pml_r=4, pml_z=2, dr=0.003, dz=0.003)) == [12]


@pytest.mark.parametrize("kind,r0", [(2, 0.0), (2, 0.0305), (3, 0.046)])
def test_axisymmetric_force_and_torsion_reproduced_on_every_zone(kind, r0):
    """The longitudinal force on the axis and the torsion ring (R12, R13) in an
    axisymmetric well excite axisymmetric fields, so every zone must carry
    the uniform grid's values at its nodes; the off-axis force is checked
    for running on its zone's nodes (finite, non-zero)."""
    g = W.Grid(nr=24, nth=16, nz=40, pml_r=4, pml_z=4, dr=0.004, dz=0.004)
    med = W.cased_well(g, z_top=0.08, casing_in=0.04, casing_t=0.012, cement_out=0.06)
    src = W.Source(r=r0, theta=0.7, z=0.08, f0=60e3, kind=kind)
    rec = W.Receivers(r=np.array([0.0, 0.021, 0.061]), theta=np.array([0.0, 0.4, 2.0]),
                      z=np.array([0.05, 0.1, 0.12]))
    sc = W.Scenario("refine-src", med, src, rec, steps=200)
    dt = oracle.Oracle(sc).dt
    u = oracle.Oracle(sc, dt=dt)
    r = oracle.RefinedOracle(sc, rows=[4, 8], dt=dt)
    u.step(200)
    r.step(200)
    if r0 > 0 and kind == 2:  # a point off the axis is not axisymmetric
        assert np.all(np.isfinite(r.field("vz", 1))) and np.abs(r.field("vz", 1)).max() > 0
        return
    vscale = max(np.abs(u.field(n)).max() for n in ("vr", "vp", "vz"))
    sscale = max(np.abs(u.field(n)).max() for n in ("srr", "spp", "szz", "srp", "spz", "srz"))
    assert vscale > 0 and sscale > 0
    for n in FIELDS:
        scale = vscale if n[0] == "v" else sscale
        for z, (row, rows, nth, _) in enumerate(r.zones):
            want = u.field(n)[:: g.nth // nth, row:row + rows, :]
            assert np.abs(r.field(n, z) - want).max() <= 1e-11 * scale, (kind, n, z)


def test_torsion_ring_on_a_zone_first_row_is_refused():
    g = W.Grid(nr=24, nth=16, nz=40, pml_r=4, pml_z=4, dr=0.004, dz=0.004)
    med = W.cased_well(g, z_top=0.08, casing_in=0.04, casing_t=0.012, cement_out=0.06)
    sc = W.Scenario("t", med, W.Source(r=0.046, z=0.08, f0=60e3, kind=3), W.on_axis_receivers([0.1]), steps=10)
    with pytest.raises(oracle.OracleError):
        oracle.RefinedOracle(sc, rows=[6, 12])  # s_rphi row 12 starts zone 2


def test_refined_cfl_step_is_inside_the_discrete_stability_limit():
    """The refined grid's dt (R7 with each row's own azimuthal step) must lie
    inside the leapfrog stability limit 2 / sqrt(lambda_max) of the coupled
    zones, interfaces included.  Power iteration on the refined oracle's own
    half-steps (dt = 1, PML off) on the 20 m well's full radius and azimuth,
    zoned by the paper's rule, on a 40-cell z-crop: dt <= 0.6 of the limit
    (the uniform grid's pin; measured 0.49)."""
    import math
    full = W.config2()
    g = full.medium.grid
    rows = W.refinement_rows(g)
    ks = int(round(full.source.z / g.dz))
    crop = W.crop_z(full.medium, ks - 20, 40)
    sc = W.Scenario("crop", crop, W.Source(z=0.05, f0=8e3), W.on_axis_receivers([0.05]), cfl=0.5, steps=0)
    dt = oracle.RefinedOracle(sc, rows, max_steps=0).dt
    assert dt > 3 * oracle.Oracle(sc, max_steps=0).dt
    o = oracle.RefinedOracle(sc, rows, max_steps=0, dt=1.0, pml_on=False)
    rng = np.random.default_rng(1)
    V, S = ("vr", "vp", "vz"), ("srr", "spp", "szz", "srp", "spz", "srz")
    x = {(n, z): rng.standard_normal(o.field(n, z).shape) for n in V for z in range(o.M)}
    for z in range(o.M):
        x[("vz", z)][:, :, -1] = 0.0
    x[("vr", 0)][:, 0, :] = 0.0
    lam = 0.0
    for it in range(150):
        nrm = math.sqrt(sum(np.sum(a * a) for a in x.values()))
        for k in x:
            x[k] /= nrm
        for z in range(o.M):
            for n in S:
                o.field(n, z)[...] = 0.0
        for (n, z), a in x.items():
            o.field(n, z)[...] = a
        o.stress_update()  # stress from v = x
        for (n, z) in x:
            o.field(n, z)[...] = 0.0
        o.velocity_update()  # the velocity that stress drives from v = 0
        y = {(n, z): -o.field(n, z).copy() for (n, z) in x}
        lam = sum(np.sum(y[k] * x[k]) for k in x)
        x = y
    assert lam > 0
    assert dt <= 0.6 * 2.0 / math.sqrt(lam), (dt, 2.0 / math.sqrt(lam))


def test_refined_pml_long_run_does_not_grow():
    """20000 steps of a cased well on a refined grid with the PML on: nothing
    grows (the interfaces add no instability to the PML's)."""
    g = W.Grid(nr=24, nth=16, nz=48, pml_r=10, pml_z=10, dr=0.005, dz=0.005)
    med = W.cased_well(g, z_top=0.12, casing_in=0.05, casing_t=0.01, cement_out=0.08)
    sc = W.Scenario("long", med, W.Source(r=0.03, theta=1.0, z=0.1, f0=20e3, kind=1), W.on_axis_receivers([0.15]),
                    steps=20000)
    o = oracle.RefinedOracle(sc, rows=[4, 8])
    peaks = []
    for blk in range(20):
        o.step(1000)
        peaks.append(max(np.abs(o.field(n, z)).max() for n in FIELDS for z in range(o.M)))
    peaks = np.array(peaks)
    assert np.all(np.isfinite(peaks))
    assert peaks[10:].max() <= peaks[:10].max(), peaks



def test_refined_dipole_converges_to_the_uniform_grid():
    """Fewer halvings toward the axis (coarse zones of 4, then 8, then 16
    nodes against the uniform 32) bring the transverse dipole's traces closer
    to the uniform grid's at every off-axis receiver: the refinement's error
    is the coarse zones' azimuthal resolution, and it vanishes with it
    (measured 4.3 / 4.1 / 0.27 % and 0.40 / 0.20 / 0.05 %)."""
    sc = _scenario(nr=30, nth=32, nz=60, kind=1, axis=True, steps=400)
    u = oracle.Oracle(sc)
    u.step(400)
    tu = u.traces()
    errs = []
    for rows in ([4, 8, 16], [8, 16], [16]):
        r = oracle.RefinedOracle(sc, rows=rows, dt=u.dt)
        r.step(400)
        tr = r.traces()
        errs.append([rel_l2(tr[q], tu[q]) for q in (1, 2)])
    errs = np.array(errs)
    assert np.all(np.diff(errs, axis=0) < 0), errs
    assert errs[-1].max() < 0.005
