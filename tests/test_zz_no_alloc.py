"""sim_read_field_noalloc: the field read-back for callers that cannot
allocate device memory (a process whose device memory is held by a caching
allocator, a monitoring thread that must not synchronise the device through
cudaFree).  It must return exactly what sim_read_field returns; checked on two
calls in a row (the fixed scratch keeps the previous call's contents) and for
two different fields and storage types.  This file is collected last."""
import numpy as np
import pytest

from paper_2302_13907_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_noalloc_read_matches_allocating_read(storage):
    from paper_2302_13907_gb300.binding import Simulation
    sc = W.config1(steps=120)
    with Simulation(sc, storage=storage) as s:
        s.step(60)
        a1 = s.field_noalloc("srr")
        b1 = s.field("srr")
        s.step(60)
        a2 = s.field_noalloc("vz")   # second call in a row, another field
        b2 = s.field("vz")
        a3 = s.field_noalloc("srr")
        b3 = s.field("srr")
    assert np.abs(b1).max() > 0 and np.abs(b2).max() > 0
    for a, b in ((a1, b1), (a2, b2), (a3, b3)):
        assert np.array_equal(a, b)


def test_noalloc_rejects_fields_beyond_the_scratch():
    from paper_2302_13907_gb300.binding import SimError, SIM_EINVAL, Simulation
    g = W.Grid(nr=120, nth=64, nz=600, pml_r=8, pml_z=8, dr=0.005, dz=0.005)  # 64*128*640 > 4 Mi cells
    sc = W.Scenario("big", W.cased_well(g, z_top=1.5), W.Source(z=0.5), W.on_axis_receivers([1.0]), steps=4)
    with Simulation(sc, kernel="split") as s:
        with pytest.raises(SimError) as ei:
            s.field_noalloc("srr")
        assert ei.value.code == SIM_EINVAL
        s.step(2)
        assert s.field("srr").shape == g.shape
