"""Pins of two oracle parts that the earlier pins bound only loosely.

* The time step (reading R7 of Sec. 3's scheme, dt = CFL * min over cells of
  1 / (Vp sqrt(1/dr^2 + 1/(r dth)^2 + 1/dz^2)), r the cell centre): the
  oracle's dt on three workloads against values worked out by hand from the
  workload geometry, one limited by the steel ring and two by the axis ring.
  The axis cases catch a radius taken at the wrong stagger (r_i = 0 on the
  axis instead of r_{i+1/2}), a dropped term or a wrong azimuthal step.
* The storage rounding of the precision variant (16-bit storage, FP32
  arithmetic): the oracle's rounding against the IEEE 754 conversions of
  NumPy (binary16) and PyTorch (bfloat16), both round to nearest even, and the
  invariant that every field of a rounded run stays representable.
"""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W


# ---------------------------------------------------------------- time step (R7)
# Hand values of the time step, worked out from each geometry (reading R7):
#  * 70x16x320 cased well, dr = dz = 5 mm, 16 azimuthal nodes: the innermost
#    steel cell (centre 0.1025 m, Vp 5900 m/s) limits: 2.985e-7 s.
#  * the 20 m well, dr = dz = 2.5 mm, 64 nodes: the axis liquid ring
#    (centre 1.25 mm, r dth = 0.123 mm, Vp 1500 m/s) limits: 4.08e-8 s.
#  * a 64-case batch member, dr = dz = 2.5 mm, 32 nodes: the axis ring
#    (r dth = 0.245 mm) limits: 8.10e-8 s.
@pytest.mark.parametrize("which,hand,rel", [
    ("config1", 2.985e-7, 3e-4),
    ("config2", 4.08e-8, 1.5e-3),
    ("case", 8.10e-8, 1e-3),
])
def test_time_step_matches_hand_values(which, hand, rel):
    sc = {"config1": W.config1, "config2": W.config2, "case": lambda: W.scenario_case(1)}[which]()
    dt = oracle.cfl_dt(sc.medium, 0.5)
    assert abs(dt / hand - 1.0) <= rel, (which, dt, hand)


def test_time_step_rounding_of_the_printed_values_is_consistent():
    """The three hand values to more digits agree with the oracle to 1e-6:
    2.98472e-7 (steel), 4.08079e-8 and 8.10350e-8 (axis)."""
    got = [oracle.cfl_dt(W.config1().medium, 0.5), oracle.cfl_dt(W.scenario_case(1).medium, 0.5)]
    assert got[0] == pytest.approx(2.98472e-7, rel=2e-6)
    assert got[1] == pytest.approx(8.10350e-8, rel=2e-6)


# ---------------------------------------------------------------- storage rounding
def _probe_values(seed=1):
    rng = np.random.default_rng(seed)
    mags = np.concatenate([rng.uniform(-30, 17, 20000), rng.uniform(-30, -13, 2000)])  # log2 |x|
    x = rng.choice([-1.0, 1.0], mags.size) * 2.0 ** mags
    # ties: values exactly half way between two FP16 (BF16) neighbours, and near the overflow
    k = rng.integers(1024, 2048, 500).astype(np.float64)
    ties16 = (k + 0.5) * 2.0 ** rng.integers(-24, 5, 500)
    kb = rng.integers(128, 256, 500).astype(np.float64)
    tiesb = (kb + 0.5) * 2.0 ** rng.integers(-20, 20, 500)
    edge = np.array([65504.0, 65519.99, 65520.0, 70000.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 0.0, -0.0])
    return np.concatenate([x, ties16, -ties16, tiesb, -tiesb, edge])


def test_fp16_rounding_matches_ieee_binary16():
    x = _probe_values()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float16).astype(np.float64)
    got = oracle.round_storage(x, "f16")
    assert np.array_equal(got, ref, equal_nan=True)


def test_bf16_rounding_matches_torch_bfloat16():
    torch = pytest.importorskip("torch")
    x = _probe_values(2)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = oracle.round_storage(x, "bf16")
    assert np.array_equal(got, ref)


def fp16_scales(sc):
    """Scales of the FP16 storage: stresses by 1/|A|, velocities by 1/|A|
    times the impedance rho Vp of the source cell (keeps both in FP16's
    normal range)."""
    m = sc.medium
    g = m.grid
    ks = int(round(sc.source.z / g.dz)) + g.pml_z
    is_ = 0 if sc.source.r < g.dr else int(np.floor(sc.source.r / g.dr))
    m0 = int(m.cell_id[0, is_, ks])
    ss = 1.0 / abs(sc.source.amplitude)
    return ss * m.rho[m0] * m.vp[m0], ss


def _small_case(r=0.0):
    g = W.Grid(nr=20, nth=8, nz=60, pml_r=6, pml_z=6, dr=0.005, dz=0.005)
    med = W.cased_well(g, z_top=0.2, casing_in=0.05, casing_t=0.01, cement_out=0.08)
    return W.Scenario("small", med, W.Source(r=r, theta=0.3, z=0.1, f0=25e3), W.on_axis_receivers([0.15, 0.25]),
                      steps=150)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_rounded_run_keeps_every_field_representable(storage):
    """After each step every stored value round(value * scale) is a value of
    the format: rounding it again changes nothing (all nine fields, so a
    field left out of the rounding fails; an off-axis source excites them all
    once the pulse, delayed by 2/f0 = 80 us = 266 steps, has gone out)."""
    sc = _small_case(r=0.02)
    scales = fp16_scales(sc) if storage == "f16" else (1.0, 1.0)
    o = oracle.Oracle(sc, storage=storage, scales=scales, max_steps=400)
    o.step(400)
    zero = []
    for q, name in enumerate(oracle.FIELDS):
        s = scales[0] if q < 3 else scales[1]
        stored = o.field(name) * s
        if np.abs(stored).max() == 0:
            zero.append(name)
        again = oracle.round_storage(stored, storage)
        assert np.allclose(again, stored, rtol=1e-14, atol=0), name
    assert zero == [], zero


def test_rounded_run_differs_from_fp64_by_the_storage_resolution():
    """BF16 storage moves the traces away from the FP64 run by far more than
    FP16 storage does (resolution 2^-8 vs 2^-11), and neither is exact; the
    rounding mode "f64" is the plain oracle bit for bit."""
    sc = _small_case()
    n = 400
    ref = oracle.Oracle(sc, max_steps=n).step(n).traces()
    same = oracle.Oracle(sc, storage="f64", max_steps=n).step(n).traces()
    assert np.array_equal(ref, same)
    eb = np.linalg.norm(oracle.Oracle(sc, storage="bf16", max_steps=n).step(n).traces() - ref) / np.linalg.norm(ref)
    eh = np.linalg.norm(oracle.Oracle(sc, storage="f16", scales=fp16_scales(sc), max_steps=n).step(n).traces()
                        - ref) / np.linalg.norm(ref)
    assert 0 < eh < eb, (eh, eb)
    assert eb > 2.0 ** -12 and eh > 2.0 ** -16, (eh, eb)


# ---------------------------------------------------------------- stochastic rounding (FP16)
def test_splitmix64_published_outputs():
    """SplitMix64 from seed 0 (Steele, Lea and Flood): the first outputs of
    the reference generator, and the same as the input generators' own copy."""
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(2) == 0x06C45D188009454F
    ks = np.array([0, 1, 7, 123456789, 2 ** 40 + 3], dtype=np.uint64)
    assert [oracle.splitmix64(int(k)) for k in ks] == [int(x) for x in W.splitmix64(0, ks)]


def test_dither_takes_16_bits_per_cell_of_one_hash_per_four_cells():
    nth, NR, NZ = 8, 26, 71
    for n, q, j, i, k in [(0, 0, 0, 0, 0), (5, 3, 2, 7, 13), (999, 8, 7, 25, 70)]:
        key = (((n * 9 + q) * nth + j) * NR + i) * ((NZ + 3) // 4) + k // 4
        z = oracle.splitmix64(key)
        assert oracle.sr_dither(n, q, j, i, k, nth, NR, NZ) == (z >> (16 * (k % 4))) & 0x1FFF


def test_stochastic_rounding_is_unbiased_and_stays_between_neighbours():
    """For FP32 values in FP16's range, over all 8192 dithers the rounded
    values are the two FP16 neighbours of x and average to x: exactly in the
    normal range (an FP32 value has 13 bits below the FP16 spacing there, as
    many as the dither), within 2^-13 of the spacing 2^-24 below it; values
    of the format are kept for every dither."""
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.uniform(-2, 2, 40), rng.uniform(-1e-5, 1e-5, 20), 2.0 ** -rng.integers(15, 24, 10)])
    xs = xs.astype(np.float32).astype(np.float64)
    d = np.arange(8192)
    for x in xs:
        r = oracle.round_stochastic_f16(np.full(8192, x), d)
        lo = np.float16(x)
        nb = {float(lo), float(np.nextafter(lo, np.float16(np.inf))), float(np.nextafter(lo, np.float16(-np.inf)))}
        assert set(np.unique(r)) <= nb, x
        tol = 0.0 if abs(x) >= 2.0 ** -14 else 2.0 ** -24 / 8192
        assert abs(r.mean() - x) <= tol + 1e-15 * abs(x), (x, r.mean())
    for h in np.float16([0.5, -1.25, 6.0e-5, 3.0e-8, 1024.0]):
        assert np.all(oracle.round_stochastic_f16(np.full(64, float(h)), np.arange(0, 8192, 128)) == float(h))


def test_stochastic_rounding_run_keeps_fields_in_fp16():
    sc = _small_case(r=0.02)
    scales = fp16_scales(sc)
    o = oracle.Oracle(sc, storage="f16sr", scales=scales, max_steps=300)
    o.step(300)
    for q, name in enumerate(oracle.FIELDS):
        s = scales[0] if q < 3 else scales[1]
        stored = o.field(name) * s
        assert np.abs(stored).max() > 0, name
        assert np.allclose(oracle.round_storage(stored, "f16"), stored, rtol=1e-14, atol=0), name
