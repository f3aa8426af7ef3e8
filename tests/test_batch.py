"""Batched scenarios: host-side validation (CPU) and, on the GPU, every case
of a batch of uneven wells equals its own single run and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import rel_l2


def small_cases(n=5, seed=0):
    """Cased wells of uneven length, different grading, casing, source and
    receiver layouts (one with an off-axis source) on a reduced grid."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        nz = int(rng.choice([37, 64, 96, 150, 211]))
        g = W.Grid(nr=30, nth=8, nz=nz, pml_r=6, pml_z=6, dr=0.004, dz=0.004)
        L = nz * g.dz
        med = W.cased_well(g, z_top=float(rng.uniform(0.3, 0.7)) * L, ramp=float(rng.uniform(0, 0.1)),
                           top_frac=float(rng.uniform(0, 1)), casing_in=0.05, casing_t=float(rng.uniform(0.006, 0.01)),
                           cement_out=0.08)
        src = W.Source(r=0.0 if c % 3 else 0.021, theta=0.4, z=0.4 * L, f0=25e3)
        rec = W.Receivers(r=np.array([0.0, 0.03]), theta=np.array([0.0, 1.3]), z=np.array([0.2 * L, 0.8 * L]))
        out.append(W.Scenario(f"small{c}", med, src, rec, steps=160))
    return out


def test_batch_rejects_bad_case_before_device_work():
    from paper_2302_13907_gb300.binding import BatchSimulation, SimError, SIM_EINVAL
    cases = small_cases(3)
    cases[1].source.z = 99.0
    with pytest.raises(SimError) as ei:
        BatchSimulation(cases)
    assert ei.value.code == SIM_EINVAL and "case 1" in str(ei.value)
    with pytest.raises(SimError):
        BatchSimulation([])


@pytest.mark.gpu
def test_batch_equals_single_runs_and_oracle():
    from paper_2302_13907_gb300.binding import BatchSimulation, Simulation
    cases = small_cases(5)
    with BatchSimulation(cases, graph_chunk=32) as b:
        n, items, grid = b.config()
        assert n == 5 and items > 0 and grid > 0
        b.run(100)
        b.run(60)
        b.sync()
        got = [b.traces(c) for c in range(5)]
        got_f = [b.field(c, "srr") for c in range(5)]
        got_vz = b.field(0, "vz")
    for c, sc in enumerate(cases):
        with Simulation(sc, kernel="split", tile=2004) as s:
            s.step(160)
            ref = s.traces()
            assert got[c].shape == ref.shape
            assert rel_l2(got[c], ref) <= 1e-6, c
            assert rel_l2(got_f[c], s.field("srr")) <= 1e-6, c
    # against the oracle element by element (the receivers of this small case
    # may still see only the exponentially small tail ahead of the wavefront)
    o = oracle.Oracle(cases[0])
    o.step(160)
    for a, ref in ((got_f[0], o.field("srr")), (got_vz, o.field("vz"))):
        assert np.abs(a - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.gpu
def test_batch_of_cement_cases():
    """Three cement-hardening cases (136 x 32 x Nz, uneven Nz) in one batch
    against their single runs."""
    from paper_2302_13907_gb300.binding import BatchSimulation, Simulation
    cases = [W.scenario_case(s) for s in (3, 6, 7)]
    assert len({c.grid.nz for c in cases}) > 1
    with BatchSimulation(cases, max_steps=64) as b:
        b.run(64)
        got = [b.traces(c) for c in range(3)]
    for c, sc in enumerate(cases):
        with Simulation(sc, kernel="split", tile=2004, max_steps=64) as s:
            s.step(64)
            assert rel_l2(got[c], s.traces()) <= 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [0, 1, -2])
def test_batch_mixing_small_and_cement_cases(tile):
    """Two small wells (shared persistent launches) and three cement cases
    (own launches, on parallel graph branches) in one batch; with tile = 1
    every case runs in the shared launches, with tile = -2 on two branches.
    Each case against its single run."""
    from paper_2302_13907_gb300.binding import BatchSimulation, Simulation
    cases = small_cases(2, seed=3) + [W.scenario_case(s) for s in (3, 6, 7)]
    steps = 160
    with BatchSimulation(cases, max_steps=steps, graph_chunk=32, tile=tile) as b:
        own, branches = b.layout()
        assert own == (0 if tile == 1 else 3)
        if tile == -2:
            assert branches == 2
        b.run(steps)
        b.sync()
        got = [b.traces(c) for c in range(len(cases))]
        got_f = [b.field(c, "srr") for c in range(len(cases))]
    for c, sc in enumerate(cases):
        with Simulation(sc, kernel="split", tile=2004, max_steps=steps) as s:
            s.step(steps)
            ref, ref_f = s.traces(), s.field("srr")  # the well's liquid has no shear stress
            assert np.abs(ref_f).max() > 0, c
            assert rel_l2(got_f[c], ref_f) <= 1e-6, c
            if np.abs(ref).max() > 0:  # the pulse may not have reached a receiver yet
                assert rel_l2(got[c], ref) <= 1e-6, c
