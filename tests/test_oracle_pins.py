"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of the Ricker pulse (Sec. 2), the compliance matrix M printed in Sec. 2,
the analytic cylindrical operators of Eq. 1 applied to smooth fields, the
exact discrete energy invariant of the staggered scheme, the azimuthal
symmetry of an axisymmetric problem, the liquid invariant (mu = 0, Sec. 2),
the point-source closed form in a homogeneous liquid and its second-order
convergence, second-order convergence in a solid under refinement by three,
the discrete stability limit (power iteration) against the CFL formula, the
low-frequency tube-wave speed of an open hole, and the PML's reflected-energy
bound.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import energy, lame, node_coefficients, random_admissible_state, rel_l2


# ---------------------------------------------------------------- Ricker (Sec. 2)
def test_ricker_closed_forms():
    f0 = 10e3
    t0 = 2.0 / f0
    assert oracle.ricker(t0, f0) == pytest.approx(1.0, abs=1e-15)
    # zeros of (1 - 2 a) with a = (pi f0 tau)^2: tau = +-1/(pi f0 sqrt 2) = +-22.5 us at 10 kHz
    tz = 1.0 / (math.pi * f0 * math.sqrt(2.0))
    assert tz == pytest.approx(22.5079e-6, rel=1e-5)
    assert abs(oracle.ricker(t0 + tz, f0)) < 1e-14
    assert abs(oracle.ricker(t0 - tz, f0)) < 1e-14
    # minima -2 exp(-3/2) at tau = +-sqrt(3/2)/(pi f0)
    tm = math.sqrt(1.5) / (math.pi * f0)
    assert oracle.ricker(t0 + tm, f0) == pytest.approx(-2 * math.exp(-1.5), rel=1e-13)
    # even about the delay and zero mean
    tt = np.linspace(0, 4 / f0, 4001)
    f = oracle.ricker(tt, f0)
    assert np.allclose(f, f[::-1], atol=1e-14)
    assert abs(np.trapezoid(f, tt)) < 1e-9 / f0


# ---------------------------------------------------- compliance M (Sec. 2, R2)
def paper_compliance(lam, mu):
    """M as printed in Sec. 2 (M_22 read as (l+m)/(3l+2m), the isotropic value)."""
    d = 3 * lam + 2 * mu
    a, b = (lam + mu) / d, -lam / (2 * d)
    M = np.array([[a, b, b, 0, 0, 0], [b, a, b, 0, 0, 0], [b, b, a, 0, 0, 0],
                  [0, 0, 0, 1, 0, 0], [0, 0, 0, 0, 1, 0], [0, 0, 0, 0, 0, 1]], dtype=float)
    return M / mu


def probe_stiffness(lam, mu):
    """Column of the oracle's stress update for unit strain rates, read from
    one stress update of a homogeneous solid with linear velocity fields."""
    g = W.Grid(nr=12, nth=8, nz=12, pml_r=0, pml_z=0, dr=0.01, dz=0.01)
    rho = 1000.0
    vs = math.sqrt(mu / rho)
    vp = math.sqrt((lam + 2 * mu) / rho)
    # ring 0 must be a liquid: make it one, probe far from it
    med = W.layered_radial(g, [g.dr], [W.FLUID, (rho, vp, vs)])
    sc = W.Scenario("probe", med, W.Source(z=0.05), W.on_axis_receivers([0.05]), steps=1, pml_on=False)
    cols = []
    i, k = 6, 5
    rh = (np.arange(g.NR) + 0.5) * g.dr
    ri = np.arange(g.NR) * g.dr
    zc = np.arange(g.NZ) * g.dz
    zh = (np.arange(g.NZ) + 0.5) * g.dz
    dt = 1e-7
    # e_zz = 1: v_z = z ; (e_rr, e_pp) = (1, 1): v_r = r
    for which in ("vz", "vr", "vr_z", "vz_r"):
        o = oracle.Oracle(sc, dt=dt, pml_on=False)
        if which == "vz":
            o.field("vz")[:] = zh[None, None, :]
        elif which == "vr":
            o.field("vr")[:] = ri[None, :, None]
        elif which == "vr_z":
            o.field("vr")[:] = zc[None, None, :]
        else:
            o.field("vz")[:] = rh[None, :, None]
        o.stress_update()
        cols.append([o.field(n)[0, i, k] / dt for n in ("srr", "spp", "szz", "srp", "spz", "srz")])
    return np.array(cols)


@pytest.mark.parametrize("lam,mu", [(2.0e10, 8.0e10), (5.4e9, 5.5e9), (1.0e9, 3.0e9)])
def test_stiffness_inverts_paper_compliance(lam, mu):
    C_ez, C_err_epp, C_grz1, C_grz2 = probe_stiffness(lam, mu)
    M = paper_compliance(lam, mu)
    # M . (ds/dt) must return the imposed strain rates
    assert np.allclose(M @ C_ez, [0, 0, 1, 0, 0, 0], atol=1e-12)
    assert np.allclose(M @ C_err_epp, [1, 1, 0, 0, 0, 0], atol=1e-12)
    # v_r = z also gives e_phiphi = u_r / r = z / r at the probed cell
    g_i, g_k, h = 6, 5, 0.01
    assert np.allclose(M @ C_grz1, [0, g_k * h / ((g_i + 0.5) * h), 0, 0, 0, 1], atol=1e-12)
    assert np.allclose(M @ C_grz2, [0, 0, 0, 0, 0, 1], atol=1e-12)
    # the identity M (1,1,1,0,0,0) = (1,1,1,0,0,0)/(3 lam + 2 mu) of the printed M
    assert np.allclose(M @ [1, 1, 1, 0, 0, 0], np.array([1, 1, 1, 0, 0, 0]) / (3 * lam + 2 * mu), rtol=1e-14)


# ------------------------------------- analytic operators of Eq. 1 (R1, R3)
def _smooth_case(h):
    nr, nz = int(round(0.2 / h)), int(round(0.2 / h))
    g = W.Grid(nr=nr, nth=int(round(0.064 / h)), nz=nz, pml_r=0, pml_z=0, dr=h, dz=h)
    rho, vp, vs = 1000.0, 3000.0, 1500.0
    med = W.layered_radial(g, [g.dr], [W.FLUID, (rho, vp, vs)])
    return g, W.Scenario("ops", med, W.Source(z=0.1), W.on_axis_receivers([0.1]), steps=1, pml_on=False), rho, vp, vs


A_R, A_T, A_Z = 9.0, 1, 11.0


def _fld(r, t, z, pr, pt, pz):
    """sin/cos products: pr,pz in {0: sin, 1: cos}; pt = azimuthal phase."""
    R = np.sin(A_R * r) if pr == 0 else np.cos(A_R * r)
    T = np.cos(A_T * t + pt)
    Z = np.sin(A_Z * z) if pz == 0 else np.cos(A_Z * z)
    return R * T * Z


def _d(r, t, z, pr, pt, pz, var):
    if var == "r":
        R = A_R * (np.cos(A_R * r) if pr == 0 else -np.sin(A_R * r))
        return R * np.cos(A_T * t + pt) * (np.sin(A_Z * z) if pz == 0 else np.cos(A_Z * z))
    if var == "t":
        return (np.sin(A_R * r) if pr == 0 else np.cos(A_R * r)) * (-A_T * np.sin(A_T * t + pt)) * \
            (np.sin(A_Z * z) if pz == 0 else np.cos(A_Z * z))
    Z = A_Z * (np.cos(A_Z * z) if pz == 0 else -np.sin(A_Z * z))
    return (np.sin(A_R * r) if pr == 0 else np.cos(A_R * r)) * np.cos(A_T * t + pt) * Z


SPEC = {"srr": (0, 0.1, 0), "spp": (1, 0.7, 0), "szz": (0, 1.3, 1), "srp": (1, 0.4, 1),
        "spz": (0, 2.1, 1), "srz": (1, 0.9, 0),
        "vr": (0, 0.3, 1), "vp": (1, 1.7, 0), "vz": (0, 2.5, 0)}


def _node(g, name):
    """coordinates (r, theta, z) of the stored nodes of a field (R3)."""
    i = np.arange(g.NR)[None, :, None] * 1.0
    j = np.arange(g.nth)[:, None, None] * 1.0
    k = np.arange(g.NZ)[None, None, :] * 1.0
    half_r = name in ("srr", "spp", "szz", "vp", "vz", "spz")
    half_t = name in ("vp", "srp", "spz")
    half_z = name in ("vz", "srz", "spz")
    dth = 2 * np.pi / g.nth
    return ((i + 0.5 * half_r) * g.dr + 0 * j + 0 * k, (j + 0.5 * half_t) * dth + 0 * i + 0 * k,
            (k + 0.5 * half_z) * g.dz + 0 * i + 0 * j)


def _operator_errors(h):
    g, sc, rho, vp_, vs_ = _smooth_case(h)
    mu = rho * vs_ ** 2
    lam = rho * vp_ ** 2 - 2 * mu
    dt = 1e-9
    # --- velocity side: v = dt/rho * (A s_r + (1/r)B s_phi + C s_z + (1/r)(A-D) s)
    o = oracle.Oracle(sc, dt=dt, pml_on=False)
    for n in ("srr", "spp", "szz", "srp", "spz", "srz"):
        o.field(n)[:] = _fld(*_node(g, n), *SPEC[n])
    o.velocity_update()

    def S(n, pos, var=None):
        return _fld(*pos, *SPEC[n]) if var is None else _d(*pos, *SPEC[n], var)

    errs = {}
    ii = np.arange(g.NR)
    mask_r = ((ii * g.dr >= 0.05) & (ii < g.NR - 2))[None, :, None]
    inner_z = np.zeros(g.NZ, bool)
    inner_z[3:-3] = True
    m = np.broadcast_to(mask_r & inner_z[None, None, :], g.shape)
    p = _node(g, "vr")
    r = p[0]
    ex = (S("srr", p, "r") + S("srp", p, "t") / r + S("srz", p, "z") + (S("srr", p) - S("spp", p)) / r) / rho
    errs["vr"] = np.abs(o.field("vr") / dt - ex)[m].max() / np.abs(ex[m]).max()
    p = _node(g, "vp")
    r = p[0]
    ex = (S("srp", p, "r") + S("spp", p, "t") / r + S("spz", p, "z") + 2 * S("srp", p) / r) / rho
    errs["vp"] = np.abs(o.field("vp") / dt - ex)[m].max() / np.abs(ex[m]).max()
    p = _node(g, "vz")
    r = p[0]
    ex = (S("srz", p, "r") + S("spz", p, "t") / r + S("szz", p, "z") + S("srz", p) / r) / rho
    errs["vz"] = np.abs(o.field("vz") / dt - ex)[m].max() / np.abs(ex[m]).max()
    # --- stress side: s = dt * C(lam, mu) e(v)
    o = oracle.Oracle(sc, dt=dt, pml_on=False)
    for n in ("vr", "vp", "vz"):
        o.field(n)[:] = _fld(*_node(g, n), *SPEC[n])
    o.field("vr")[:, 0, :] = 0
    o.stress_update()

    def V(n, pos, var=None):
        return _fld(*pos, *SPEC[n]) if var is None else _d(*pos, *SPEC[n], var)

    p = _node(g, "srr")
    r = p[0]
    err_ = V("vr", p, "r")
    epp = V("vp", p, "t") / r + V("vr", p) / r
    ezz = V("vz", p, "z")
    for n, ex in (("srr", (lam + 2 * mu) * err_ + lam * (epp + ezz)),
                  ("spp", (lam + 2 * mu) * epp + lam * (err_ + ezz)),
                  ("szz", (lam + 2 * mu) * ezz + lam * (err_ + epp))):
        errs[n] = np.abs(o.field(n) / dt - ex)[m].max() / np.abs(ex[m]).max()
    p = _node(g, "srp")
    r = p[0]
    ex = mu * (V("vp", p, "r") + V("vr", p, "t") / r - V("vp", p) / r)
    errs["srp"] = np.abs(o.field("srp") / dt - ex)[m].max() / np.abs(ex[m]).max()
    p = _node(g, "spz")
    r = p[0]
    ex = mu * (V("vz", p, "t") / r + V("vp", p, "z"))
    errs["spz"] = np.abs(o.field("spz") / dt - ex)[m].max() / np.abs(ex[m]).max()
    p = _node(g, "srz")
    ex = mu * (V("vz", p, "r") + V("vr", p, "z"))
    errs["srz"] = np.abs(o.field("srz") / dt - ex)[m].max() / np.abs(ex[m]).max()
    return errs


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_operators_match_cylindrical_equations_second_order():
    """Every discrete operator reproduces the textbook cylindrical velocity-
    stress system (Eq. 1 read through R1) on smooth fields, with error
    falling ~4x per halving of h away from the axis."""
    e1 = _operator_errors(0.004)
    e2 = _operator_errors(0.002)
    for n in e1:
        assert e1[n] < 2e-2, (n, e1[n])
        ratio = e1[n] / e2[n]
        assert 3.0 < ratio < 5.5, (n, e1[n], e2[n], ratio)


# ----------------------------------------- discrete energy invariant (R3-R5, R9)
def _energy_medium():
    g = W.Grid(nr=40, nth=8, nz=60, pml_r=0, pml_z=0, dr=0.005, dz=0.005)
    return W.cased_well(g, z_top=0.15)


def test_energy_conserved_pml_off():
    med = _energy_medium()
    f, coef = random_admissible_state(med, seed=7)
    sc = W.Scenario("energy", med, W.Source(z=0.1), W.on_axis_receivers([0.1]), steps=0, pml_on=False)
    o = oracle.Oracle(sc, max_steps=0, pml_on=False)
    o.dt  # CFL 0.5
    for n, a in f.items():
        o.field(n)[:] = a
    g = med.grid
    E = []
    v_old = {n: o.field(n).copy() for n in ("vr", "vp", "vz")}
    for it in range(1500):
        s_now = {n: o.field(n).copy() for n in ("srr", "spp", "szz", "srp", "spz", "srz")}
        o.velocity_update()
        v_new = {n: o.field(n).copy() for n in ("vr", "vp", "vz")}
        if it % 50 == 0 or it == 1499:
            E.append(energy(coef, g, v_old, v_new, s_now))
        o.stress_update()
        v_old = v_new
    E = np.array(E)
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12, np.max(np.abs(E - E[0])) / E[0]


def test_energy_not_conserved_with_pml():
    """Sanity of the invariant: with the PML on, energy leaves the domain."""
    med = _energy_medium()
    f, coef = random_admissible_state(med, seed=3)
    g = med.grid
    g2 = W.Grid(nr=30, nth=8, nz=40, pml_r=10, pml_z=10, dr=g.dr, dz=g.dz)
    med2 = W.Medium(g2, med.cell_id, med.rho, med.vp, med.vs)
    sc = W.Scenario("energy", med2, W.Source(z=0.1), W.on_axis_receivers([0.1]), steps=0)
    o = oracle.Oracle(sc, max_steps=0)
    for n, a in f.items():
        o.field(n)[:] = a
    v_old = {n: o.field(n).copy() for n in ("vr", "vp", "vz")}
    s_now = {n: o.field(n).copy() for n in ("srr", "spp", "szz", "srp", "spz", "srz")}
    o.velocity_update()
    E0 = energy(coef, g, v_old, {n: o.field(n).copy() for n in ("vr", "vp", "vz")}, s_now)
    o.stress_update()
    o.step(600)
    v_old = {n: o.field(n).copy() for n in ("vr", "vp", "vz")}
    s_now = {n: o.field(n).copy() for n in ("srr", "spp", "szz", "srp", "spz", "srz")}
    o.velocity_update()
    E1 = energy(coef, g, v_old, {n: o.field(n).copy() for n in ("vr", "vp", "vz")}, s_now)
    assert 0 < E1 < 0.5 * E0


def test_source_energy_then_conservation():
    """A Ricker-driven run with the PML off: once the pulse is over
    (t > 4/f0) the energy stays constant."""
    g = W.Grid(nr=40, nth=8, nz=80, pml_r=0, pml_z=0, dr=0.005, dz=0.005)
    med = W.cased_well(g, z_top=0.2)
    sc = W.Scenario("e", med, W.Source(z=0.15, f0=20e3), W.on_axis_receivers([0.2]), steps=2000, pml_on=False)
    o = oracle.Oracle(sc, pml_on=False)
    coef = node_coefficients(med)
    n0 = int(math.ceil((4.0 / 20e3) / o.dt)) + 1
    o.step(n0)
    E = []
    for it in range(400):
        v_old = {n: o.field(n).copy() for n in ("vr", "vp", "vz")}
        s_now = {n: o.field(n).copy() for n in ("srr", "spp", "szz", "srp", "spz", "srz")}
        o.step(1)
        if it % 40 == 0:
            # velocity after this step is v^{n+1/2}
            E.append(energy(coef, g, v_old, {n: o.field(n).copy() for n in ("vr", "vp", "vz")}, s_now))
    E = np.array(E)
    assert E[0] > 0
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-11


# ------------------------------------------------------ azimuthal symmetry
def test_axisymmetric_problem_is_theta_independent():
    sc = W.config1(steps=300)
    o = oracle.Oracle(sc)
    o.step(300)
    for n in ("vp", "srp", "spz"):
        assert np.all(o.field(n) == 0.0), n
    for n in ("vr", "vz", "srr", "spp", "szz", "srz"):
        a = o.field(n)
        scale = np.abs(a).max()
        assert scale > 0
        assert np.abs(a - a[:1]).max() <= 1e-14 * scale, n


def test_liquid_has_isotropic_stress_and_no_shear():
    """mu = 0 in the liquid (Sec. 2): shear stresses vanish and the normal
    stresses stay equal in every liquid cell."""
    sc = W.config1(steps=300)
    o = oracle.Oracle(sc)
    o.step(300)
    _, _, mu = lame(sc.medium)
    fluid = mu[sc.medium.cell_id] == 0
    srr, spp, szz = o.field("srr"), o.field("spp"), o.field("szz")
    assert np.abs(srr[fluid]).max() > 0
    # equal up to the rounding of the three (differently ordered) Lame sums
    sc_ = np.abs(srr[fluid]).max()
    assert np.abs(srr[fluid] - spp[fluid]).max() <= 1e-13 * sc_
    assert np.abs(srr[fluid] - szz[fluid]).max() <= 1e-13 * sc_
    # shear nodes touching a liquid cell
    f = fluid
    touch_rz = np.zeros_like(f)
    touch_rz[:, 1:, :-1] = f[:, :-1, :-1] | f[:, 1:, :-1] | f[:, :-1, 1:] | f[:, 1:, 1:]
    assert np.all(o.field("srz")[touch_rz] == 0)


# ------------------------------- point source in a homogeneous liquid (R6)
def _point_source_error(h, f0=10e3, c=1500.0, rho=1000.0):
    pml = 10
    nr = int(round(0.3 / h))
    zs = 0.1
    nz = int(round(0.65 / h))
    g = W.Grid(nr=nr, nth=4, nz=nz, pml_r=pml, pml_z=pml, dr=h, dz=h)
    med = W.homogeneous(g, (rho, c, 0.0))
    R = np.array([0.2, 0.3, 0.4])
    sc = W.Scenario("pt", med, W.Source(z=zs, f0=f0, amplitude=1.0), W.on_axis_receivers(zs + R), cfl=0.5,
                    steps=0)
    o = oracle.Oracle(sc, max_steps=1)
    dt = o.dt
    T = 2.0 / f0 + R.max() / c + 1.6 / f0
    n = int(math.ceil(T / dt))
    o = oracle.Oracle(sc, max_steps=n)
    o.step(n)
    p = o.traces()
    t = (np.arange(n) + 1) * dt
    errs = []
    for q, Rq in enumerate(R):
        tau = t - Rq / c - 2.0 / f0
        a = (math.pi * f0 * tau) ** 2
        fprime = 2 * math.pi ** 2 * f0 ** 2 * tau * (2 * a - 3) * np.exp(-a)
        exact = -fprime / (4 * math.pi * c ** 2 * Rq)
        win = np.abs(tau) < 1.5 / f0
        errs.append(rel_l2(p[q, win], exact[win]))
    return np.array(errs)


def test_point_source_closed_form_and_order():
    """p(R, t) = -A f'(t - R/c) / (4 pi c^2 R) on the axis of a homogeneous
    liquid; the error falls ~4x when h halves (second order)."""
    e_coarse = _point_source_error(0.004)
    e_fine = _point_source_error(0.002)
    # The error is the scheme's second-order phase error, which grows with R:
    # (kh)^2/24 * omega * R / c at the rms frequency of -f' (about 1.4 f0,
    # k = 58.6 rad/m) gives 1.3 % at h = 2 mm, R = 0.4 m.
    assert np.all(e_fine < 0.025), e_fine
    ratio = e_coarse / e_fine
    assert np.all((ratio > 3.0) & (ratio < 5.5)), (e_coarse, e_fine)


# ----------------------------------------- open-hole tube wave (Biot 1952)
def test_open_hole_tube_wave_speed():
    f0 = 1e3
    g = W.Grid(nr=40, nth=4, nz=400, pml_r=8, pml_z=10, dr=0.01, dz=0.02)
    med = W.layered_radial(g, [0.1], [W.FLUID, W.ROCK])
    zs = 0.5
    zr = zs + np.arange(2.0, 6.01, 1.0)
    sc = W.Scenario("tube", med, W.Source(z=zs, f0=f0), W.on_axis_receivers(zr), cfl=0.5, steps=0)
    dt = oracle.Oracle(sc, max_steps=1).dt
    rf, vf = W.FLUID[0], W.FLUID[1]
    mu = W.ROCK[0] * W.ROCK[2] ** 2
    vt = vf / math.sqrt(1 + rf * vf ** 2 / mu)
    assert vt == pytest.approx(1382.5, abs=0.1)
    n = int(math.ceil((2.0 / f0 + (zr[-1] - zs) / vt + 1.5 / f0) / dt))
    o = oracle.Oracle(sc, max_steps=n)
    o.step(n)
    p = o.traces()
    # arrival time of the tube wave: envelope-weighted cross-correlation peak
    lag = []
    for q in range(1, len(zr)):
        a, b = p[0], p[q]
        cc = np.correlate(b, a, mode="full")
        m = int(np.argmax(cc))
        y0, y1, y2 = cc[m - 1], cc[m], cc[m + 1]
        frac = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
        lag.append((m - (len(a) - 1) + frac) * dt)
    lag = np.array(lag)
    speed = np.polyfit(lag, zr[1:] - zr[0], 1)[0]
    assert speed == pytest.approx(vt, rel=0.02), speed


# ------------------------------------------------------- PML bound (R8)
def _pml_case(nr, nz, pml, big):
    h = 0.01
    g = W.Grid(nr=nr, nth=4, nz=nz, pml_r=pml, pml_z=pml, dr=h, dz=h)
    off = (nz - 100) // 2 * h
    med = W.cased_well(g, z_top=0.6 + off)
    rec = W.Receivers(r=np.array([0.0, 0.0, 0.0, 0.25, 0.25]), theta=np.zeros(5),
                      z=np.array([0.3, 0.6, 0.8, 0.3, 0.7]) + off)
    return W.Scenario("pml", med, W.Source(z=0.5 + off, f0=5e3), rec, cfl=0.5, steps=0)


def test_pml_reflection_bound():
    """Traces with a 10-cell PML against a domain large enough that no wall
    reflection reaches the receivers.  The layer is designed for an amplitude
    reflection R0 = 1e-3 at normal incidence (1e-6 in energy); allowing 10x
    for oblique incidence and the discrete layer, every receiver (two of them
    5 cm from the radial layer) must see reflected energy <= 1e-5 (-50 dB)."""
    small = _pml_case(30, 100, 10, False)
    big = _pml_case(150, 400, 0, True)
    # identical dt for both runs: the smaller of the two CFL steps
    dt = min(oracle.Oracle(small, max_steps=1).dt, oracle.Oracle(big, max_steps=1).dt)
    T = 2.0 / 5e3 + 0.25e-3
    n = int(math.ceil(T / dt))
    a = oracle.Oracle(small, max_steps=n, dt=dt)
    a.step(n)
    b = oracle.Oracle(big, max_steps=n, dt=dt, pml_on=False)
    b.step(n)
    pa, pb = a.traces(), b.traces()
    refl = np.sum((pa - pb) ** 2, axis=1) / np.sum(pb ** 2, axis=1)
    assert np.all(refl < 1e-5), refl
    # and the PML is doing something: rigid walls at the same place reflect strongly
    c = oracle.Oracle(small, max_steps=n, dt=dt, pml_on=False)
    c.step(n)
    rigid = np.sum((c.traces() - pb) ** 2, axis=1) / np.sum(pb ** 2, axis=1)
    assert np.all(rigid > 100 * refl), (rigid, refl)


def test_pml_long_run_is_stable():
    """No late-time growth over 20000 steps.  An open hole empties through
    the PML (decay by orders of magnitude); a cased well keeps a slowly
    leaking radial resonance of the liquid column inside the steel pipe, so
    there the check is only that nothing grows."""
    g = W.Grid(nr=24, nth=4, nz=48, pml_r=10, pml_z=10, dr=0.005, dz=0.005)
    for name, med in (("open", W.layered_radial(g, [0.05], [W.FLUID, W.ROCK])),
                      ("cased", W.cased_well(g, z_top=0.12))):
        sc = W.Scenario("long", med, W.Source(z=0.1, f0=20e3), W.on_axis_receivers([0.15]), steps=20000)
        o = oracle.Oracle(sc)
        peaks = []
        for blk in range(20):
            o.step(1000)
            peaks.append(max(np.abs(o.field(n)).max() for n in oracle.FIELDS))
        peaks = np.array(peaks)
        assert np.all(np.isfinite(peaks)), name
        if name == "open":
            assert peaks[-1] < 1e-4 * peaks[0], peaks
        else:
            assert peaks[10:].max() <= peaks[:10].max(), peaks


# ---------------------------------------------------------------- convergence in a solid (Eq. 1, Sec. 3)
def _ring_pulse_run(f, h0=0.01, n0=16, dt0=None):
    """Axisymmetric smooth pulse in a homogeneous solid (liquid ring 0, never
    reached in the window), rigid walls, no source; grid h0 / f, dt0 / f, n0 f
    steps.  Returns the stresses at the final (integer) time and dt0."""
    h = h0 / f
    g = W.Grid(nr=30 * f, nth=4, nz=36 * f, pml_r=0, pml_z=0, dr=h, dz=h)
    cid = np.ones(g.shape, dtype=np.uint16)
    cid[:, 0, :] = 0
    med = W.Medium(g, cid, np.array([1000.0, 2400.0]), np.array([1500.0, 4000.0]), np.array([0.0, 2300.0]))
    sc = W.Scenario("conv", med, W.Source(z=0.05, amplitude=0.0), W.on_axis_receivers([0.05]), steps=0,
                    pml_on=False)
    if dt0 is None:
        dt0 = oracle.cfl_dt(W.Medium(W.Grid(nr=30, nth=4, nz=36, pml_r=0, pml_z=0, dr=h0, dz=h0),
                                     np.ones((4, 30, 36), np.uint16), med.rho, med.vp, med.vs), 0.5)
    o = oracle.Oracle(sc, max_steps=0, dt=dt0 / f, pml_on=False)
    r0, z0, s = 0.15, 0.18, 0.025
    rh = (np.arange(g.NR) + 0.5) * h   # cell-centre radius
    ri = np.arange(g.NR) * h           # integer-node radius
    zc = np.arange(g.NZ) * h           # cell-centre depth
    zh = (np.arange(g.NZ) + 0.5) * h   # half-node depth
    G = lambda r, z: np.exp(-((r[:, None] - r0) ** 2 + (z[None, :] - z0) ** 2) / (2 * s * s))
    # a velocity field at rest stresses (so dv/dt = 0 at t = 0 and v(-dt/2) = v(0) + O(dt^2)),
    # mixing radial and vertical motion so that both P and S terms act
    vr = G(ri, zc) * (zc[None, :] - z0) / s
    vz = G(rh, zh) * (rh[:, None] - r0) / s
    vr[0, :] = 0.0
    vz[:, -1] = 0.0
    o.field("vr")[:] = vr[None]
    o.field("vz")[:] = vz[None]
    o.step(n0 * f)
    return {n: o.field(n)[0].copy() for n in ("srr", "spp", "szz", "srz")}, dt0


def test_solid_refinement_by_three_is_second_order():
    """Refinement ratio 3 (the staggered nodes of h/3 contain those of h):
    log3(|u_h - u_h/3| / |u_h/3 - u_h/9|) = 2 +- 0.3 on the stresses at the
    nodes the three grids share, at the same time (fixed dt / h)."""
    u1, dt0 = _ring_pulse_run(1)
    u3, _ = _ring_pulse_run(3, dt0=dt0)
    u9, _ = _ring_pulse_run(9, dt0=dt0)

    def restrict(u, f, name):
        # coarse node (i, k) of a cell-centre radius / integer depth field sits at (f i + (f-1)/2, f k)
        oi = (f - 1) // 2 if name in ("srr", "spp", "szz") else 0
        ok = (f - 1) // 2 if name == "srz" else 0
        return u[oi::f, ok::f][:30, :36]

    e1 = e2 = 0.0
    for n in ("srr", "spp", "szz", "srz"):
        a, b, c = u1[n], restrict(u3[n], 3, n), restrict(u9[n], 9, n)
        e1 += np.sum((a - b) ** 2)
        e2 += np.sum((b - c) ** 2)
    order = math.log(math.sqrt(e1 / e2), 3)
    assert abs(order - 2.0) <= 0.3, order


# ---------------------------------------------------------------- stability limit (power iteration)
def test_cfl_formula_is_inside_the_discrete_stability_limit():
    """The leapfrog step is stable iff dt <= 2 / sqrt(lambda_max) of the
    operator v -> -(velocity update of the stress update of v) per unit dt^2.
    Power iteration on the oracle's own half-steps (dt = 1, PML off, stresses
    reset to zero) estimates lambda_max on the 70 x 16 x 320 cased well; the
    CFL 0.5 formula's dt must sit below 0.6 of that limit."""
    sc = W.config1(steps=0)
    o = oracle.Oracle(sc, max_steps=0, dt=1.0, pml_on=False)
    dt_formula = oracle.cfl_dt(sc.medium, 0.5)
    rng = np.random.default_rng(1)
    x = {n: rng.standard_normal(sc.grid.shape) for n in ("vr", "vp", "vz")}
    x["vr"][:, 0, :] = 0.0
    x["vz"][:, :, -1] = 0.0
    lam = 0.0
    for it in range(150):
        nrm = math.sqrt(sum(np.sum(a * a) for a in x.values()))
        for n in x:
            x[n] /= nrm
        for n in ("srr", "spp", "szz", "srp", "spz", "srz"):
            o.field(n)[:] = 0.0
        for n in x:
            o.field(n)[:] = 0.0
        # stress from v = x, then the velocity that stress drives from v = 0
        for n in x:
            o.field(n)[:] = x[n]
        o.stress_update()
        for n in x:
            o.field(n)[:] = 0.0
        o.velocity_update()
        y = {n: -o.field(n).copy() for n in x}
        lam = sum(np.sum(y[n] * x[n]) for n in x)  # Rayleigh quotient (x normalised)
        x = y
    dt_crit = 2.0 / math.sqrt(lam)
    assert lam > 0
    assert dt_formula <= 0.6 * dt_crit, (dt_formula, dt_crit)


# ------------------------------------------- point forces and torsion (R12, R13)
def _force_field(c, rho, A, f0, cos_t, R, t):
    """Pressure of a point force A f(t) in a homogeneous liquid at distance R,
    cos_t = cosine between the force and the direction to the receiver:
    p = cos_t / (4 pi) [A f'(t - R/c) / (c R) + A f(t - R/c) / R^2]."""
    tau = t - R / c - 2.0 / f0
    a = (math.pi * f0 * tau) ** 2
    f = (1 - 2 * a) * np.exp(-a)
    fp = 2 * math.pi ** 2 * f0 ** 2 * tau * (2 * a - 3) * np.exp(-a)
    return cos_t / (4 * math.pi) * A * (fp / (c * R) + f / R ** 2), tau


def test_longitudinal_force_closed_form_and_antisymmetry():
    """Point force along z on the axis of a homogeneous liquid (R12): the
    axis pressure above and below the force follows the dipole closed form
    (opposite signs) within the scheme's second-order phase error."""
    h, f0, c, rho = 0.002, 10e3, 1500.0, 1000.0
    g = W.Grid(nr=150, nth=4, nz=350, pml_r=10, pml_z=10, dr=h, dz=h)
    med = W.homogeneous(g, (rho, c, 0.0))
    zs = 0.3
    ks = int(round(zs / h))
    z_force = (ks + 0.5) * h  # the v_z node the force acts on
    zr = np.array([zs + 0.2, zs + 0.3, zs - 0.2])
    sc = W.Scenario("fz", med, W.Source(kind=W.SOURCE_LONGITUDINAL, z=zs, f0=f0), W.on_axis_receivers(zr),
                    cfl=0.5, steps=0)
    dt = oracle.Oracle(sc, max_steps=1).dt
    n = int(math.ceil((2.0 / f0 + 0.32 / c + 1.6 / f0) / dt))
    o = oracle.Oracle(sc, max_steps=n)
    o.step(n)
    p = o.traces()
    t = (np.arange(n) + 1) * dt
    for q, z in enumerate(zr):
        zc = round(z / h) * h
        R = abs(zc - z_force)
        exact, tau = _force_field(c, rho, 1.0, f0, np.sign(zc - z_force), R, t)
        win = np.abs(tau) < 1.5 / f0
        assert rel_l2(p[q, win], exact[win]) < 0.03, (z, rel_l2(p[q, win], exact[win]))


def test_transverse_force_is_a_dipole():
    """Horizontal point force on the axis (R12): the ring-mean (axis)
    pressure vanishes, the field at theta and theta + pi is exactly opposite,
    and off-axis pressure in the source plane follows the dipole closed form
    with cos(theta - phi0)."""
    h, f0, c, rho = 0.004, 5e3, 1500.0, 1000.0
    nth = 16
    g = W.Grid(nr=60, nth=nth, nz=120, pml_r=10, pml_z=10, dr=h, dz=h)
    med = W.homogeneous(g, (rho, c, 0.0))
    zs, phi0 = 0.24, 2 * math.pi * 3 / nth
    r_rec = (30 + 0.5) * h
    th = np.array([phi0, phi0 + math.pi, phi0 + math.pi / 2, 0.0])
    rec = W.Receivers(r=np.array([r_rec] * 4 + [0.0]), theta=np.append(th, 0.0), z=np.array([zs] * 5))
    sc = W.Scenario("fx", med, W.Source(kind=W.SOURCE_TRANSVERSE, theta=phi0, z=zs, f0=f0), rec, cfl=0.5, steps=0)
    dt = oracle.Oracle(sc, max_steps=1).dt
    n = int(math.ceil((2.0 / f0 + r_rec / c + 1.6 / f0) / dt))
    o = oracle.Oracle(sc, max_steps=n)
    o.step(n)
    p = o.traces()
    peak = np.abs(p[0]).max()
    assert peak > 0
    assert np.abs(p[0] + p[1]).max() <= 1e-12 * peak      # theta + pi: opposite
    assert np.abs(p[2]).max() <= 1e-12 * peak              # perpendicular: zero
    assert np.abs(p[4]).max() <= 1e-12 * peak              # axis (ring mean): zero
    t = (np.arange(n) + 1) * dt
    exact, tau = _force_field(c, rho, 1.0, f0, math.cos(0.0 - phi0), r_rec, t)
    win = np.abs(tau) < 1.5 / f0
    assert rel_l2(p[3, win], exact[win]) < 0.05, rel_l2(p[3, win], exact[win])


def test_torsion_ring_in_a_free_pipe():
    """Torsion ring in the wall of a free steel pipe (liquid inside and
    outside, R13): the motion is pure SH (v_phi, s_rphi, s_phiz only, theta
    independent), the liquid stays exactly at rest, and the torsional pulse
    runs along the pipe at the steel's shear speed (the T(0,1) mode of a
    free tube is non-dispersive)."""
    dr, dz, f0 = 0.0025, 0.005, 10e3
    g = W.Grid(nr=60, nth=4, nz=360, pml_r=8, pml_z=12, dr=dr, dz=dz)
    med = W.layered_radial(g, [0.10, 0.11], [W.FLUID, W.STEEL, W.FLUID])
    zs = 0.3
    sc = W.Scenario("tor", med, W.Source(kind=W.SOURCE_TORSION, r=0.105, z=zs, f0=f0), W.on_axis_receivers([zs]),
                    cfl=0.5, steps=0)
    o = oracle.Oracle(sc, max_steps=0)
    dt = o.dt
    z1, z2 = zs + 0.4, zs + 1.2
    k1, k2 = int(round(z1 / dz)) + 12, int(round(z2 / dz)) + 12
    i_w = int(0.105 / dr)  # cell inside the wall
    vs = W.STEEL[2]
    n = int(math.ceil((2.0 / f0 + (z2 - zs) / vs + 1.5 / f0) / dt))
    s1, s2 = np.zeros(n), np.zeros(n)
    for m in range(n):
        o.step(1)
        vp = o.field("vp")
        s1[m], s2[m] = vp[0, i_w, k1], vp[0, i_w, k2]
    fl = np.zeros(g.shape, dtype=bool)
    rc = g.r_centre()
    fl[:, (rc < 0.10) | (rc >= 0.11), :] = True
    for name in ("vr", "vz", "srr", "spp", "szz", "srz"):
        assert np.all(o.field(name) == 0.0), name
    vpf = o.field("vp")
    assert np.abs(vpf).max() > 0
    assert np.all(vpf[:, :i_w - 3, :] == 0.0) and np.all(vpf[:, i_w + 4:, :] == 0.0)  # liquid at rest
    assert np.all(vpf == vpf[:1])  # theta independent
    # moveout between the two stations (peak of the envelope by cross-correlation)
    cc = np.correlate(s2, s1, mode="full")
    lag = (np.argmax(cc) - (n - 1)) * dt
    v = (z2 - z1) / lag
    assert v == pytest.approx(vs, rel=0.02), v
