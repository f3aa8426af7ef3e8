"""Z-slab decomposition of one well (Sec. 4) as two and three gloo ranks on
the CPU: each rank runs the FP64 oracle on its slab only (updates, sources
and receivers restricted to its own z cells) and swaps the boundary planes
of the fields it just updated with its neighbours after each half-step
(paper_2302_13907_gb300/slabs.py).  Every field of every owned cell and
every receiver trace equals the undivided oracle run bit for bit, also with
the volumetric source and the two point forces placed on a slab boundary."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2302_13907_gb300 import slabs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scenario(kind=0, ks=None):
    """ks: the stored z index of the source (None: z = 0.1 m); on a cut the
    source's nodes fall on both sides of a slab boundary."""
    from paper_2302_13907_gb300 import workloads as W
    g = W.Grid(nr=12, nth=6, nz=70, pml_r=4, pml_z=4, dr=0.004, dz=0.003)
    med = W.cased_well(g, z_top=0.12, casing_in=0.016, casing_t=0.008, cement_out=0.032)
    rec = W.Receivers(r=np.array([0.0, 0.013, 0.0, 0.03]), theta=np.array([0.0, 1.1, 0.0, 2.0]),
                      z=np.array([0.02, 0.09, 0.16, 0.2]))
    z = 0.1 if ks is None else (ks - g.pml_z) * g.dz
    return W.Scenario("slabs", med, W.Source(kind=kind, r=0.006, theta=0.4, z=z, f0=60e3), rec, steps=160)


class OracleSlab:
    """The oracle as a slab engine: it holds the whole well but updates,
    injects and samples only its own z cells."""

    def __init__(self, sc, k_lo, k_hi):
        import oracle
        self.o = oracle.Oracle(sc)
        self.o.set_zrange(k_lo, k_hi)
        self.force = sc.source.kind in (1, 2)

    def velocity_half(self, n):
        self.o.velocity_update()
        if self.force:
            self.o.inject_source(n)

    def stress_half(self, n):
        self.o.stress_update()
        if not self.force:
            self.o.inject_source(n)

    def sample(self, n):
        self.o.sample(n)
        self.o.set_steps_done(n + 1)

    def get_planes(self, group, k0, k1):
        return np.stack([self.o.field(f)[:, :, k0:k1] for f in slabs.GROUPS[group]])

    def set_planes(self, group, k0, a):
        for q, f in enumerate(slabs.GROUPS[group]):
            self.o.field(f)[:, :, k0:k0 + a.shape[-1]] = a[q]


def _rank(rank, ws, port, out_dir, kind=0, ks=None):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        sc = _scenario(kind, ks)
        p = slabs.plan(sc.grid.NZ, ws)
        s0, s1 = p.owned(rank)
        e = OracleSlab(sc, s0, s1)
        slabs.run(e, p, rank, sc.steps, dist)
        import oracle
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), s0=s0, s1=s1,
                 **{f: e.o.field(f)[:, :, s0:s1] for f in oracle.FIELDS}, traces=e.o.traces())
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(600)
@pytest.mark.parametrize("ws,kind,ks", [(2, 0, None), (3, 0, None),
                                        # on the cut of two slabs (stored k 40 is rank 1's first cell)
                                        (2, 0, 40), (2, 1, 39), (2, 2, 39)])
def test_slab_ranks_reproduce_the_whole_well(tmp_path, ws, kind, ks):
    import oracle
    if ks is not None:
        assert slabs.plan(78, 2).owned(1)[0] == 40
    mp.spawn(_rank, args=(ws, _free_port(), str(tmp_path), kind, ks), nprocs=ws, join=True)
    sc = _scenario(kind, ks)
    ref = oracle.Oracle(sc)
    ref.step(sc.steps)
    p = slabs.plan(sc.grid.NZ, ws)
    got_tr = np.zeros_like(ref.traces())
    g = sc.grid
    rec_k = np.rint(sc.receivers.z / g.dz).astype(int) + g.pml_z
    for r in range(ws):
        d = np.load(tmp_path / f"rank{r}.npz")
        s0, s1 = int(d["s0"]), int(d["s1"])
        assert (s0, s1) == p.owned(r)
        for f in oracle.FIELDS:
            assert np.array_equal(d[f], ref.field(f)[:, :, s0:s1]), (r, f)
        mine = (rec_k >= s0) & (rec_k < s1)
        got_tr[mine] = d["traces"][mine]
    assert np.array_equal(got_tr, ref.traces())
    assert np.abs(ref.traces()).max() > 0


def test_plan_is_contiguous_and_aligned():
    p = slabs.plan(1056, 4)
    assert p.bounds[0][0] == 0 and p.bounds[-1][1] == 1056
    for (a, b), (c, d) in zip(p.bounds, p.bounds[1:]):
        assert b == c and b % 4 == 0
    assert max(b - a for a, b in p.bounds) - min(b - a for a, b in p.bounds) <= 4
    assert p.local_range(0) == (0, p.bounds[0][1] + slabs.GHOST)
    with pytest.raises(ValueError):
        slabs.plan(20, 4)
