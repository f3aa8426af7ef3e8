"""The seeded workload generator: geometry, grading, noise statistics."""
import math

import numpy as np
import pytest

from paper_2302_13907_gb300 import workloads as W


def _mat(med, j, i, k):
    m = med.cell_id[j, i, k]
    return (med.rho[m], med.vp[m], med.vs[m])


def test_config1_geometry_by_cell_centre():
    sc = W.config1()
    g = sc.grid
    med = sc.medium
    assert g.shape == (16, 70, 320)
    rc = g.r_centre()
    zc = g.z_centre()
    k_below = int(np.searchsorted(zc, 0.75))  # first cell with z >= 0.75
    k_above = k_below - 1
    for i in range(g.NR):
        r = rc[i]
        if r < 0.10:
            exp_b = exp_a = W.FLUID
        elif r < 0.11:
            exp_b = exp_a = W.STEEL
        elif r < 0.15:
            exp_b, exp_a = W.CEMENT, W.FLUID
        else:
            exp_b = exp_a = W.ROCK
        assert _mat(med, 3, i, k_below) == exp_b
        assert _mat(med, 3, i, k_above) == exp_a
    # medium continues into the z-PML: fluid annulus above, cement below
    assert _mat(med, 0, 25, 0) == W.FLUID and _mat(med, 0, 25, g.NZ - 1) == W.CEMENT
    assert np.all(med.cell_id == med.cell_id[:1])  # axisymmetric


def test_receiver_and_source_positions_config1():
    sc = W.config1()
    k = np.rint(sc.receivers.z / sc.grid.dz).astype(int)
    assert list(k) == [80, 133, 187, 240]
    assert round(sc.source.z / sc.grid.dz) == 60


def test_graded_cement_ramp():
    g = W.Grid(nr=60, nth=4, nz=400, pml_r=0, pml_z=0, dr=0.0025, dz=0.0025)
    med = W.cased_well(g, z_top=0.3, ramp=0.3, top_frac=0.25)
    i = int(0.13 / g.dr)
    rho_c, vp_c, vs_c = W.CEMENT
    mu_full = rho_c * vs_c ** 2
    K = rho_c * vp_c ** 2 - 4 * mu_full / 3
    for k in range(g.NZ):
        z = k * g.dz
        rho, vp, vs = _mat(med, 0, i, k)
        if z < 0.3 - 1e-12:
            assert (rho, vp, vs) == W.FLUID
            continue
        lev = min(max((z - 0.3) / 0.3, 0.0), 1.0)
        mu = rho * vs ** 2
        assert mu == pytest.approx(mu_full * (0.25 + 0.75 * lev), rel=1e-12)
        assert rho * vp ** 2 - 4 * mu / 3 == pytest.approx(K, rel=1e-12)  # bulk fixed


def test_straddle_cell_volume_fraction():
    g = W.Grid(nr=60, nth=4, nz=40, pml_r=0, pml_z=0, dr=0.0025, dz=0.0025)
    t = 0.0093
    med = W.cased_well(g, z_top=0.0, casing_t=t)
    ro = 0.10 + t
    i = int(ro / g.dr)
    ra, rb = i * g.dr, (i + 1) * g.dr
    f = (ro ** 2 - ra ** 2) / (rb ** 2 - ra ** 2)
    rho, vp, vs = _mat(med, 0, i, 5)
    assert rho == pytest.approx(f * W.STEEL[0] + (1 - f) * W.CEMENT[0], rel=1e-12)
    ms, mc = W.STEEL[0] * W.STEEL[2] ** 2, W.CEMENT[0] * W.CEMENT[2] ** 2
    assert rho * vs ** 2 == pytest.approx(1 / (f / ms + (1 - f) / mc), rel=1e-12)
    assert _mat(med, 0, i - 1, 5) == W.STEEL and _mat(med, 0, i + 1, 5) == W.CEMENT


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0 (published test vector of the generator)
    out = W.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rock_noise_statistics():
    # a long box so that the sample correlation averages ~250 correlation lengths
    g = W.Grid(nr=100, nth=8, nz=20000, pml_r=0, pml_z=0, dr=0.0025, dz=0.0025)
    nz = W.Noise(seed=11)
    d = W.rock_noise(g, 60, nz)
    assert np.abs(d).max() == pytest.approx(0.05, abs=1e-4)
    q = d / 1e-4
    assert np.allclose(q, np.round(q), atol=1e-6)
    # correlation along z: exp(-dz^2/corr^2) -> e^-1 at 0.2 m = 80 cells
    a = d - d.mean()
    c0 = np.mean(a * a)
    c80 = np.mean(a[:, :, :-80] * a[:, :, 80:])
    assert c80 / c0 == pytest.approx(math.exp(-1.0), abs=0.1)
    c40 = np.mean(a[:, :, :-40] * a[:, :, 40:])
    assert c40 / c0 == pytest.approx(math.exp(-0.25), abs=0.1)
    # same seed, same field; other seed, other field
    g2 = W.Grid(nr=70, nth=8, nz=300, pml_r=0, pml_z=0, dr=0.0025, dz=0.0025)
    d2 = W.rock_noise(g2, 60, nz)
    assert np.array_equal(d2, W.rock_noise(g2, 60, nz))
    assert not np.array_equal(d2, W.rock_noise(g2, 60, W.Noise(seed=12)))


def test_case_draw_ranges():
    for seed in range(1, 9):
        p = W.scenario_case(seed, surrogate_inputs=True).params
        L = p["nz"] * 0.0025
        assert p["nz"] in (2048, 3072, 4096, 6144)
        assert 0.3 * L <= p["z_top"] <= 0.7 * L
        assert 0 <= p["ramp"] <= 0.5 and 0 <= p["top_frac"] <= 1
        assert 0.008 <= p["casing_t"] <= 0.012
        assert 0.9 * 1700 <= p["cement_vs"] <= 1.1 * 1700 and 0.9 * 2300 <= p["rock_vs"] <= 1.1 * 2300


def test_full_scale_well_medium_is_valid():
    """A shortened variant of the 20 m well (same radial grid, noise and
    grading): every cell ID indexes the table; noisy rock spans +-5 %."""
    sc = W.config2(nz=256)
    med = sc.medium
    assert med.cell_id.max() < med.n_mat
    g = sc.grid
    rock = med.cell_id[:, int(0.15 / g.dr) + 1:, :]
    vp = med.vp[rock]
    # normalised by max|g|: one extreme reaches exactly 5 %, none exceeds it
    assert np.abs(vp / 4000 - 1).max() == pytest.approx(0.05, rel=1e-9)
    assert len(np.unique(rock)) > 500
    full = W.config2.__doc__
    assert "20000 steps" in full


def test_small_cement_case_draws_and_geometry():
    """Miniature cement cases: inputs inside their ranges, source 0.075 m
    above the cement top, every cell of ring 0 a liquid."""
    for seed in range(6):
        sc = W.small_cement_case(seed)
        x = W.surrogate_features(sc)
        assert 0.55 <= x[0] <= 0.65 and 0.0 <= x[1] <= 0.2 and 0.0 <= x[2] <= 1.0 and 0.008 <= x[3] <= 0.012
        assert 0.9 * W.CEMENT[2] <= x[4] <= 1.1 * W.CEMENT[2] and 0.9 * W.ROCK[2] <= x[5] <= 1.1 * W.ROCK[2]
        assert sc.source.z == pytest.approx(x[0] - 0.075)
        assert np.all(sc.medium.vs[sc.medium.cell_id[:, 0, :]] == 0)


def _paper_well():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_realistic_well.json")))


def test_realistic_well_defaults_are_the_printed_dimensions():
    import inspect
    P = _paper_well()
    d = {k: v.default for k, v in inspect.signature(W.realistic_well).parameters.items()}
    for key in ("H_target", "ID_prev", "H_toc", "H_spacer", "L_joint", "L_collar", "OD_target", "OD_collar"):
        assert d[key] == P[key + "_m"], key
    assert W.PAPER_STEEL[2] == P["torsion_wave_speed_m_s"]


def test_realistic_well_matches_the_printed_dimensions():
    """The paper's realistic well (Sec. 6) at the printed dimensions: interior
    casing OD 0.1778 m to 202 m, collars OD 0.1945 m, 0.184 m long at every
    12 m joint boundary, exterior casing ID 0.22916 m, spacer (liquid) above
    200 m and cement below in the annulus, casing Vs 3220 m/s."""
    g = W.Grid(nr=64, nth=4, nz=2000, pml_r=4, pml_z=4, dr=0.0025, dz=0.0025)
    med = W.realistic_well(g, z0=11.0)  # depths 11 .. 16 m: the collar at 12 m
    vs = med.vs[med.cell_id[0]]  # [NR][NZ]
    rc = g.r_centre()
    depth = 11.0 + g.z_centre()

    def col(d):
        return vs[:, int(np.argmin(np.abs(depth - d)))]

    plain, collar = col(13.0), col(12.0)
    steel = np.flatnonzero(plain == 3220.0)
    inner = steel[rc[steel] < 0.1]
    outer = steel[rc[steel] > 0.1]
    assert rc[inner[0]] >= 0.1778 / 2 - 0.00919 - 1e-12 and rc[inner[-1]] < 0.1778 / 2
    assert rc[outer[0]] >= 0.22916 / 2 and rc[outer[-1]] < 0.22916 / 2 + 0.01105
    assert np.all(plain[rc < 0.1778 / 2 - 0.00919] == 0)  # liquid inside
    assert np.all(plain[(rc >= 0.1778 / 2) & (rc < 0.22916 / 2)] == 0)  # spacer
    on_collar = (rc >= 0.1778 / 2) & (rc < 0.1945 / 2)
    assert np.all(collar[on_collar] == 3220.0) and np.all(plain[on_collar] == 0)
    at = np.flatnonzero(vs[on_collar.nonzero()[0][0]] == 3220.0)
    assert abs(depth[at].mean() - 12.0) < g.dz and abs(len(at) * g.dz - 0.184) <= g.dz
    deep = W.realistic_well(g, z0=199.0)
    dv = deep.vs[deep.cell_id[0]]
    ann = (rc >= 0.1778 / 2 + 0.01) & (rc < 0.22916 / 2)  # away from collars
    ddepth = 199.0 + g.z_centre()
    assert np.all(dv[ann][:, ddepth < 200.0] == 0) and np.all(dv[ann][:, ddepth >= 200.0] > 0)
    assert np.all(med.vs[med.cell_id[:, 0, :]] == 0)  # ring 0 liquid
