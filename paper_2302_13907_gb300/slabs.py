"""Z-slab decomposition of one well over several processes (Sec. 4 of the
paper: each processing unit owns a contiguous range of z planes and swaps the
planes next to its boundaries with its two neighbours every step).

Each rank owns stored z cells [s0, s1) of the well and keeps GHOST cells on
each side it shares with a neighbour.  One step is

    velocity half-step of the owned cells (and the point forces of step n)
    swap the velocities: owned [s0, s0 + GHOST) -> rank - 1, [s1 - GHOST, s1) -> rank + 1
    stress half-step of the owned cells (and the volumetric / torsion source)
    swap the stresses the same way
    receivers inside [s0, s1)

The velocity update of a cell reads stresses one cell away in z and the
stress update velocities one cell away, so one exchanged plane per side would
do; GHOST = 4 keeps every owned range aligned to the four-cell vectors of
the kernels.  The swaps are nonblocking point-to-point messages of
torch.distributed (gloo for host tensors, NCCL for device tensors); nothing
else crosses ranks, and each owned cell is updated from the same values as in
the undivided well, so the decomposed run reproduces it exactly.

The per-rank work is an `engine` object:
    velocity_half(n), stress_half(n), sample(n)
    get_planes(group, k0, k1) -> array [fields][nth][NR][k1 - k0]
    set_planes(group, k0, array)
with group "v" (v_r, v_phi, v_z) or "s" (the six stresses) and k in the
well's stored z index.  SimSlab is that engine for a library handle
(sim_create_slab: its planes stay on the device, on the stream the handle
and the collectives share); exchange_local swaps the slabs of one process
(several slabs on one GPU) without collectives.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GHOST = 4
GROUPS = {"v": ("vr", "vp", "vz"), "s": ("srr", "spp", "szz", "srp", "spz", "srz")}


@dataclass(frozen=True)
class SlabPlan:
    NZ: int
    bounds: tuple  # ((s0, s1) per rank), contiguous, covering 0 .. NZ

    @property
    def ranks(self) -> int:
        return len(self.bounds)

    def owned(self, rank: int):
        return self.bounds[rank]

    def local_range(self, rank: int):
        """Stored cells a rank holds: its own and its ghost cells."""
        s0, s1 = self.bounds[rank]
        return max(0, s0 - GHOST), min(self.NZ, s1 + GHOST)


def plan(NZ: int, ranks: int) -> SlabPlan:
    """Contiguous slabs of nearly equal size whose inner boundaries fall on
    multiples of four cells; every slab at least 2 GHOST cells wide."""
    if ranks < 1:
        raise ValueError("need at least one rank")
    cuts = [0]
    for r in range(1, ranks):
        c = int(round(r * NZ / ranks / 4.0)) * 4
        cuts.append(c)
    cuts.append(NZ)
    bounds = tuple((cuts[r], cuts[r + 1]) for r in range(ranks))
    if any(b - a < 2 * GHOST for a, b in bounds):
        raise ValueError(f"{NZ} z cells are too few for {ranks} slabs of at least {2 * GHOST} cells")
    return SlabPlan(NZ, bounds)


def exchange(engine, p: SlabPlan, rank: int, group: str, comm, device=None):
    """Swap the boundary planes of `group` with both neighbours (nonblocking
    sends and receives, then wait)."""
    import torch

    s0, s1 = p.owned(rank)
    reqs, into = [], []

    def tens(a):
        t = torch.as_tensor(np.ascontiguousarray(a)) if isinstance(a, np.ndarray) else a
        return t.to(device) if device is not None else t

    if rank > 0:
        out = tens(engine.get_planes(group, s0, s0 + GHOST))
        buf = torch.empty_like(out)
        reqs += [comm.isend(out, rank - 1), comm.irecv(buf, rank - 1)]
        into.append((s0 - GHOST, buf))
    if rank < p.ranks - 1:
        out = tens(engine.get_planes(group, s1 - GHOST, s1))
        buf = torch.empty_like(out)
        reqs += [comm.isend(out, rank + 1), comm.irecv(buf, rank + 1)]
        into.append((s1, buf))
    for r in reqs:
        r.wait()
    for k0, buf in into:
        engine.set_planes(group, k0, buf.cpu().numpy() if buf.device.type == "cpu" else buf)


def run(engine, p: SlabPlan, rank: int, steps: int, comm, first_step: int = 0, device=None):
    """`steps` leapfrog steps of this rank's slab, swapping boundary planes
    after each half-step."""
    for n in range(first_step, first_step + steps):
        engine.velocity_half(n)
        exchange(engine, p, rank, "v", comm, device)
        engine.stress_half(n)
        exchange(engine, p, rank, "s", comm, device)
        engine.sample(n)


class SimSlab:
    """A slab of the well on one GPU: a sim_create_slab handle whose planes
    are exchanged as CUDA tensors on `stream` (the handle's stream)."""

    def __init__(self, scenario, p: SlabPlan, rank: int, stream=None, **kw):
        import torch
        from .binding import Simulation
        self.sim = Simulation(scenario, slab=p.owned(rank), stream=stream, kernel="split", **kw)
        self.rows = scenario.grid.nth * scenario.grid.NR
        self._torch = torch

    def velocity_half(self, n):
        self.sim.half_step(0)

    def stress_half(self, n):
        self.sim.half_step(1)

    def sample(self, n):
        pass

    def get_planes(self, group, k0, k1):
        t = self._torch
        out = t.empty((len(GROUPS[group]), self.rows, k1 - k0), dtype=t.float32, device="cuda")
        return self.sim.get_planes(0 if group == "v" else 1, k0, k1, out)

    def set_planes(self, group, k0, buf):
        self.sim.put_planes(0 if group == "v" else 1, k0, k0 + buf.shape[-1], buf.contiguous())


def exchange_local(engines, p: SlabPlan, group: str):
    """The swap of `group` between the slabs of one process (rank r's engine
    is engines[r]): each inner boundary's four own cells on each side go to
    the other slab's ghost cells."""
    for r in range(p.ranks - 1):
        a, b = engines[r], engines[r + 1]
        cut = p.owned(r)[1]
        lo = a.get_planes(group, cut - GHOST, cut)
        hi = b.get_planes(group, cut, cut + GHOST)
        b.set_planes(group, cut - GHOST, lo)
        a.set_planes(group, cut, hi)


def run_local(engines, p: SlabPlan, steps: int, first_step: int = 0):
    """`steps` leapfrog steps of all slabs of one process, swapping after
    each half-step."""
    for n in range(first_step, first_step + steps):
        for e in engines:
            e.velocity_half(n)
        exchange_local(engines, p, "v")
        for e in engines:
            e.stress_half(n)
        exchange_local(engines, p, "s")
        for e in engines:
            e.sample(n)
