"""Z slabs of one well on the GPU (sim_create_slab, sim_half_step,
sim_get_planes / sim_put_planes): two and three slabs of one well in one
process on one GPU, sharing a stream, swapping their boundary planes after
each half-step (slabs.run_local), against the undivided well on the same
kernels: every field of every owned cell (within 1e-5 of the field's
maximum: the cells next to an inner boundary run the general cell body, the
undivided well the lean one, and the two fuse multiply-adds differently) and
every receiver trace.  The decomposition itself is exact: the oracle's slabs
reproduce the undivided oracle bit for bit (test_slabs_gloo)."""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import slabs
from paper_2302_13907_gb300 import workloads as W
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _scenario(kind=0, ks=None):
    """ks: the stored z index of the source (None: z = 0.36 m)."""
    g = W.Grid(nr=40, nth=16, nz=300, pml_r=8, pml_z=8, dr=0.004, dz=0.003)
    med = W.cased_well(g, z_top=0.5, casing_in=0.08, casing_t=0.01, cement_out=0.12)
    rec = W.Receivers(r=np.array([0.0, 0.013, 0.0, 0.03]), theta=np.array([0.0, 1.1, 0.0, 2.0]),
                      z=np.array([0.1, 0.35, 0.5, 0.8]))
    z = 0.36 if ks is None else (ks - g.pml_z) * g.dz
    src = W.Source(kind=kind, r=0.006 if kind != 3 else 0.085, theta=0.4, z=z, f0=40e3)
    return W.Scenario("slabs", med, src, rec, steps=400)


@pytest.mark.parametrize("ws,kind,ks", [(2, 0, None), (3, 0, None), (2, 1, None), (3, 3, None),
                                        # on the cut of two slabs (stored k 160 is slab 1's first cell)
                                        (2, 0, 160), (2, 1, 159), (2, 2, 159)])
def test_slabs_reproduce_the_whole_well(ws, kind, ks):
    import torch
    from paper_2302_13907_gb300.binding import Simulation
    sc = _scenario(kind, ks)
    if ks is not None:
        assert slabs.plan(sc.grid.NZ, 2).owned(1)[0] == 160
    g = sc.grid
    p = slabs.plan(g.NZ, ws)
    stream = torch.cuda.current_stream().cuda_stream
    tile = 22852324
    with Simulation(sc, kernel="split", tile=tile, stream=stream) as whole:
        whole.step(sc.steps)
        ref = {f: whole.field(f) for f in oracle.FIELDS}
        ref_tr = whole.traces()
    engines = [slabs.SimSlab(sc, p, r, stream=stream, tile=tile) for r in range(ws)]
    try:
        slabs.run_local(engines, p, sc.steps)
        torch.cuda.synchronize()
        tr = np.zeros_like(ref_tr)
        rec_k = np.rint(sc.receivers.z / g.dz).astype(int) + g.pml_z
        for r, e in enumerate(engines):
            s0, s1 = p.owned(r)
            l0 = e.sim.l0
            for f in oracle.FIELDS:
                a = e.sim.field(f)[:, :, s0 - l0:s1 - l0]
                b = ref[f][:, :, s0:s1]
                scale = np.abs(ref[f]).max()
                d = np.abs(a - b).max() / max(scale, 1e-30)
                print(f"slab {r} {f}: max |diff| / max {d:.2e}")
                # the cells next to an inner boundary sit in the slab's z-end tiles and run the
                # general body (identity z stretch there), the undivided well runs the lean one:
                # the lean body lets the compiler fuse a derivative's product into the sum that
                # follows, the general body's PML select does not, so the two round differently
                assert d <= 1e-5, (r, f, d)
            mine = (rec_k >= s0) & (rec_k < s1)
            t = e.sim.traces()
            tr[mine] = t[mine]
            assert np.all(t[~mine] == 0)
        # the torsion ring makes no pressure (pure shear): its traces are zero
        assert (np.abs(ref_tr).max() > 0) == (kind != 3)
        assert np.abs(tr - ref_tr).max() <= 1e-5 * max(np.abs(ref_tr).max(), 1e-30)
    finally:
        for e in engines:
            e.sim.close()


def test_slab_rejects_misaligned_bounds():
    from paper_2302_13907_gb300.binding import SIM_EINVAL, SimError, Simulation
    sc = _scenario()
    with pytest.raises(SimError) as ei:
        Simulation(sc, slab=(0, 101))
    assert ei.value.code == SIM_EINVAL
