"""Seeded synthetic cased-well workloads (inputs only).

This module decides, from a geometry description and a seed, which material
every grid cell holds and the (rho, Vp, Vs) of every material ID, where the
source sits and where the receivers are.  It holds none of the numerical
method's arithmetic: no Lame moduli, no time step, no wavelet, no PML, no
stencil.  Both the CUDA simulator and the FP64 oracle consume what it returns,
and nothing else is shared between them.

Grid convention (the paper's cylindrical frame, Sec. 2 and Sec. 3):
  * cell (i, j, k) has its centre at r = (i + 1/2) dr, theta = j dtheta,
    z = (k - pml_z) dz, with i in [0, NR), j in [0, Nth), k in [0, NZ),
    NR = nr + pml_r, NZ = nz + 2 pml_z;  z is depth, increasing downward;
  * arrays are laid out [theta][r][z] with z fastest;
  * the material of a cell is decided by its centre on half-open intervals
    (the paper attaches the medium parameters to the central point, Sec. 3).

Media of the well (values of the cased-well workloads): fluid, steel casing,
cement annulus (fluid above the cement top), host rock.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, Sequence

import numpy as np

# (rho [kg/m^3], Vp [m/s], Vs [m/s]); Vs = 0 marks a fluid (the paper models
# the liquid as a medium whose shear modulus vanishes, Sec. 2).
FLUID = (1000.0, 1500.0, 0.0)
STEEL = (7850.0, 5900.0, 3200.0)
CEMENT = (1900.0, 3000.0, 1700.0)
ROCK = (2400.0, 4000.0, 2300.0)

SOURCE_MONOPOLE = 0  # volumetric point source (Sec. 2, first source type)
SOURCE_TRANSVERSE = 1  # point force in the radial / horizontal direction (second type)
SOURCE_LONGITUDINAL = 2  # point force along z (third type)
SOURCE_TORSION = 3  # torsion ring about the well axis (fourth type)
QUANTITY_PRESSURE = 0


@dataclass(frozen=True)
class Grid:
    """Interior cell counts, PML widths and steps of the cylindrical grid."""

    nr: int
    nth: int
    nz: int
    pml_r: int
    pml_z: int
    dr: float
    dz: float

    @property
    def NR(self) -> int:
        return self.nr + self.pml_r

    @property
    def NZ(self) -> int:
        return self.nz + 2 * self.pml_z

    @property
    def shape(self) -> tuple:
        return (self.nth, self.NR, self.NZ)

    @property
    def cells(self) -> int:
        return self.nth * self.NR * self.NZ

    def r_centre(self) -> np.ndarray:
        return (np.arange(self.NR) + 0.5) * self.dr

    def z_centre(self) -> np.ndarray:
        return (np.arange(self.NZ) - self.pml_z) * self.dz


@dataclass
class Medium:
    grid: Grid
    cell_id: np.ndarray  # uint16 [nth][NR][NZ]
    rho: np.ndarray  # float64 [n_mat]
    vp: np.ndarray
    vs: np.ndarray

    @property
    def n_mat(self) -> int:
        return int(self.rho.shape[0])


@dataclass
class Source:
    kind: int = SOURCE_MONOPOLE
    r: float = 0.0  # r < dr places the source on the axis (all ring-0 nodes)
    theta: float = 0.0
    z: float = 0.0
    f0: float = 10e3
    amplitude: float = 1.0


@dataclass
class Receivers:
    r: np.ndarray
    theta: np.ndarray
    z: np.ndarray
    quantity: int = QUANTITY_PRESSURE

    @property
    def n(self) -> int:
        return int(self.z.shape[0])


@dataclass
class Scenario:
    name: str
    medium: Medium
    source: Source
    receivers: Receivers
    cfl: float = 0.5
    steps: int = 800
    pml_on: bool = True
    params: dict = field(default_factory=dict)

    @property
    def grid(self) -> Grid:
        return self.medium.grid


def on_axis_receivers(z: Sequence[float]) -> Receivers:
    z = np.asarray(z, dtype=np.float64)
    return Receivers(r=np.zeros_like(z), theta=np.zeros_like(z), z=z)


class _Registry:
    """Deduplicating table of (rho, Vp, Vs) -> material ID."""

    def __init__(self):
        self._ids = {}
        self.rows = []

    def id(self, mat) -> int:
        key = (float(mat[0]), float(mat[1]), float(mat[2]))
        got = self._ids.get(key)
        if got is None:
            got = len(self.rows)
            if got > 0xFFFF:
                raise ValueError("more than 65536 materials")
            self._ids[key] = got
            self.rows.append(key)
        return got

    def arrays(self):
        t = np.asarray(self.rows, dtype=np.float64).reshape(-1, 3)
        return t[:, 0].copy(), t[:, 1].copy(), t[:, 2].copy()


def _moduli(mat):
    rho, vp, vs = mat
    mu = rho * vs * vs
    return rho, rho * vp * vp - 4.0 * mu / 3.0, mu  # rho, bulk K, shear mu


def _from_moduli(rho, K, mu):
    return (rho, math.sqrt((K + 4.0 * mu / 3.0) / rho), math.sqrt(max(mu, 0.0) / rho))


def graded_cement(cement, level: float, top_frac: float):
    """Cement whose shear modulus is top_frac + (1 - top_frac) * level of full,
    bulk modulus and density held fixed (the cement-hardening profile)."""
    rho, K, mu = _moduli(cement)
    return _from_moduli(rho, K, mu * (top_frac + (1.0 - top_frac) * level))


def straddle_material(inner, outer, frac_inner: float):
    """Volume-fraction average of a cell cut by a cylindrical interface:
    density arithmetic, bulk and shear moduli harmonic (Reuss)."""
    if frac_inner >= 1.0:
        return inner
    if frac_inner <= 0.0:
        return outer
    r1, K1, m1 = _moduli(inner)
    r2, K2, m2 = _moduli(outer)
    rho = frac_inner * r1 + (1 - frac_inner) * r2
    K = 1.0 / (frac_inner / K1 + (1 - frac_inner) / K2)
    mu = 0.0 if (m1 == 0.0 or m2 == 0.0) else 1.0 / (frac_inner / m1 + (1 - frac_inner) / m2)
    return _from_moduli(rho, K, mu)


# ----------------------------------------------------------------------------
# counter-based normal deviates: SplitMix64 (Steele, Lea & Flood 2014) + Box-Muller
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """Output number `counter` of the SplitMix64 sequence started at `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def normal_deviates(seed: int, index: np.ndarray) -> np.ndarray:
    """N(0,1) deviate for each linear cell index: outputs 2L and 2L+1 of
    SplitMix64 give two uniforms, Box-Muller gives the deviate."""
    index = index.astype(np.uint64)
    a = splitmix64(seed, index * np.uint64(2))
    b = splitmix64(seed, index * np.uint64(2) + np.uint64(1))
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = (b >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _reflect_gauss_matrix(n: int, sigma: float) -> np.ndarray:
    """n x n matrix of a Gaussian smoother (std `sigma` cells) with
    half-sample-symmetric reflection at both ends."""
    rad = int(math.ceil(4 * sigma))
    x = np.arange(-rad, rad + 1)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    w /= w.sum()
    m = np.zeros((n, n))
    for i in range(n):
        for off, wt in zip(x, w):
            p = i + off
            # reflect about -1/2 and n-1/2 (repeat until inside)
            while p < 0 or p >= n:
                p = -p - 1 if p < 0 else 2 * n - p - 1
            m[i, p] += wt
    return m


def _smooth_reflect_fft(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    """Gaussian smoothing along `axis` with reflection at both ends, by FFT."""
    n = a.shape[axis]
    pad = int(math.ceil(4 * sigma))
    pad = min(pad, n - 1) if n > 1 else 0
    widths = [(0, 0)] * a.ndim
    widths[axis] = (pad, pad)
    ap = np.pad(a, widths, mode="symmetric")
    m = ap.shape[axis]
    f = np.fft.rfftfreq(m)
    h = np.exp(-2.0 * (np.pi * f * sigma) ** 2)
    shp = [1] * a.ndim
    shp[axis] = h.shape[0]
    out = np.fft.irfft(np.fft.rfft(ap, axis=axis) * h.reshape(shp), n=m, axis=axis)
    sl = [slice(None)] * a.ndim
    sl[axis] = slice(pad, pad + n)
    return out[tuple(sl)]


@dataclass(frozen=True)
class Noise:
    """Gaussian-correlated perturbation of the rock's Vp and Vs.

    White N(0,1) per cell, smoothed with a separable Gaussian whose kernel
    std is corr/2 in physical length per axis (arc length r*dtheta in theta,
    periodic), so the correlation function is exp(-d^2/corr^2); normalised by
    max|g| over the rock, scaled by `amp` and quantised to `quantum`.
    """

    seed: int = 20230227
    amp: float = 0.05
    corr: float = 0.2
    quantum: float = 1e-4


def rock_noise(grid: Grid, i0: int, noise: Noise) -> np.ndarray:
    """Quantised relative perturbation delta[j, i - i0, k] of rock cells i >= i0."""
    nth, NR, NZ = grid.shape
    nri = NR - i0
    s = 0.5 * noise.corr
    g = np.empty((nth, nri, NZ), dtype=np.float64)
    for j in range(nth):
        # linear index of the cell in the full [theta][r][z] grid
        idx = (np.uint64(j) * np.uint64(NR) + np.arange(i0, NR, dtype=np.uint64)[:, None]) * np.uint64(NZ) \
            + np.arange(NZ, dtype=np.uint64)[None, :]
        g[j] = normal_deviates(noise.seed, idx)
    # z: reflect-padded FFT smoothing
    g = _smooth_reflect_fft(g, s / grid.dz, axis=2)
    # r: reflecting smoother matrix
    W = _reflect_gauss_matrix(nri, s / grid.dr)
    g = np.einsum("ab,jbk->jak", W, g, optimize=True)
    # theta: periodic, kernel width in cells depends on the radius
    dth = 2 * np.pi / nth
    f = np.fft.fftfreq(nth)
    G = np.fft.fft(g, axis=0)
    r = (np.arange(i0, NR) + 0.5) * grid.dr
    sig = s / (r * dth)  # cells
    H = np.exp(-2.0 * (np.pi * f[:, None] * sig[None, :]) ** 2)  # [nth, nri]
    g = np.real(np.fft.ifft(G * H[:, :, None], axis=0))
    g /= np.max(np.abs(g))
    d = noise.amp * g
    return np.round(d / noise.quantum) * noise.quantum


def cased_well(grid: Grid, *, z_top: float, ramp: float = 0.0, top_frac: float = 1.0,
               casing_in: float = 0.10, casing_t: float = 0.01, cement_out: float = 0.15,
               fluid=FLUID, steel=STEEL, cement=CEMENT, rock=ROCK,
               noise: Optional[Noise] = None) -> Medium:
    """Fluid-filled well, steel casing [casing_in, casing_in + casing_t),
    cement annulus up to cement_out for depths z >= z_top (fluid above it),
    rock beyond.  The cement's shear modulus ramps linearly from top_frac of
    full at z_top to full at z_top + ramp.  A cell cut by the casing's outer
    radius gets a volume-fraction averaged material."""
    nth, NR, NZ = grid.shape
    rc = grid.r_centre()
    zc = grid.z_centre()
    eps = 1e-9 * grid.dz
    if ramp > 0:
        level = np.clip((zc - z_top) / ramp, 0.0, 1.0)
    else:
        level = np.ones(NZ)
    in_cement_zone = zc >= z_top - eps
    casing_out = casing_in + casing_t
    reg = _Registry()
    id2 = np.empty((NR, NZ), dtype=np.uint16)
    rock_i0 = None
    for i in range(NR):
        r = rc[i]
        ra, rb = i * grid.dr, (i + 1) * grid.dr
        if r < casing_in:
            id2[i, :] = reg.id(fluid)
            continue
        if r >= cement_out:
            if rock_i0 is None:
                rock_i0 = i
            id2[i, :] = reg.id(rock)
            continue
        # annulus material per depth (fluid above the top, graded cement below):
        # one ID per distinct (zone, level), assigned to all depths sharing it
        zone_key = np.where(in_cement_zone, level, -1.0)
        keys, inv = np.unique(zone_key, return_inverse=True)
        straddle = ra < casing_out < rb
        fr = (casing_out ** 2 - ra ** 2) / (rb ** 2 - ra ** 2) if straddle else 0.0
        lut = np.empty(len(keys), dtype=np.uint16)
        for q, key in enumerate(keys):
            mat_out = fluid if key < 0 else graded_cement(cement, float(key), top_frac)
            if straddle:  # cell cut by the casing's outer radius: volume fraction by int r dr
                mat = straddle_material(steel, mat_out, fr)
            elif r < casing_out:
                mat = steel
            else:
                mat = mat_out
            lut[q] = reg.id(mat)
        id2[i, :] = lut[inv]
    cell_id = np.broadcast_to(id2, (nth, NR, NZ)).copy()
    if noise is not None and rock_i0 is not None:
        d = rock_noise(grid, rock_i0, noise)
        q = np.round(d / noise.quantum).astype(np.int64)
        nq = int(round(noise.amp / noise.quantum))
        # one ID per quantised level; level 0 is the unperturbed rock already registered
        lut = np.array([reg.id((rock[0], rock[1] * (1 + m * noise.quantum), rock[2] * (1 + m * noise.quantum)))
                        for m in range(-nq, nq + 1)], dtype=np.uint16)
        cell_id[:, rock_i0:, :] = lut[np.clip(q, -nq, nq) + nq]
    rho, vp, vs = reg.arrays()
    return Medium(grid=grid, cell_id=cell_id, rho=rho, vp=vp, vs=vs)


# casing steel with the shear speed the paper quotes for its casings (Sec. 6)
PAPER_STEEL = (7850.0, 5900.0, 3220.0)


def realistic_well(grid: Grid, *, z0: float = 0.0, H_target: float = 202.0, ID_prev: float = 0.22916,
                   H_toc: float = 200.0, H_spacer: float = 200.0, L_joint: float = 12.0, L_collar: float = 0.184,
                   OD_target: float = 0.1778, OD_collar: float = 0.1945, t_target: float = 0.00919,
                   t_prev: float = 0.01105, fluid=FLUID, steel=PAPER_STEEL, cement=CEMENT,
                   rock=ROCK) -> Medium:
    """The paper's realistic cased well (Sec. 6) from its printed dimensions:
    an interior (target) casing of outer diameter OD_target down to depth
    H_target, built of joints L_joint long whose collars (L_collar long,
    outer diameter OD_collar) sit at every joint boundary, inside an exterior
    (previous) casing of inner diameter ID_prev; the annulus between them
    holds the spacer (drilling fluid) down to H_spacer and cement from H_toc
    down (the cement top).  The figure with the rest of the geometry is
    missing, so these are readings: the wall thicknesses t_target and t_prev
    (not printed), the collars centred on the joint boundaries n L_joint, the
    spacer a drilling fluid (the paper's annulus liquid has zero shear
    speed), rock outside the exterior casing, and liquid inside the interior
    casing (also below its shoe).  Depth is measured down from the top of
    the well; grid z = 0 (its first interior cell) sits at depth z0, so a
    grid can hold a section of the well.  A cell's material is decided by
    its centre."""
    nth, NR, NZ = grid.shape
    r = grid.r_centre()[:, None]
    depth = z0 + grid.z_centre()[None, :]
    r_tin, r_tout, r_col = OD_target / 2 - t_target, OD_target / 2, OD_collar / 2
    r_pin, r_pout = ID_prev / 2, ID_prev / 2 + t_prev
    in_target = depth < H_target
    n = np.round(depth / L_joint)
    collar = in_target & (n >= 1) & (np.abs(depth - n * L_joint) < L_collar / 2)
    reg = _Registry()
    F, S, C, R = reg.id(fluid), reg.id(steel), reg.id(cement), reg.id(rock)
    id2 = np.full((NR, NZ), F, dtype=np.uint16)
    annulus = (r >= r_tout) & (r < r_pin)
    id2 = np.where(annulus & (depth >= H_toc), C, id2)
    id2 = np.where(annulus & (depth < H_spacer), F, id2)
    id2 = np.where((r >= r_tin) & (r < r_tout) & in_target, S, id2)
    id2 = np.where((r >= r_tout) & (r < r_col) & collar, S, id2)
    id2 = np.where((r >= r_pin) & (r < r_pout), S, id2)
    id2 = np.where(r >= r_pout, R, id2).astype(np.uint16)
    rho, vp, vs = reg.arrays()
    return Medium(grid=grid, cell_id=np.broadcast_to(id2, (nth, NR, NZ)).copy(), rho=rho, vp=vp, vs=vs)


def realistic_well_section(z0: float = 100.0, length: float = 20.0, *, nth: int = 8, nr: int = 64, pml_r: int = 16,
                           pml_z: int = 16, dr: float = 0.0025, dz: float = 0.0025, f0: float = 8e3,
                           source_depth: Optional[float] = None, steps: int = 1000) -> Scenario:
    """A section [z0, z0 + length) of the realistic well with the paper's
    torsion source (Sec. 6): a ring one cell inside the outer wall of the
    casing that carries the collars (the target casing, liquid on both
    sides) at source_depth (default 5 m into the section), and pressure
    receivers on the axis at a quarter and three quarters of the section (a
    torsion field has no pressure: they record zeros)."""
    g = Grid(nr=nr, nth=nth, nz=int(round(length / dz)), pml_r=pml_r, pml_z=pml_z, dr=dr, dz=dz)
    med = realistic_well(g, z0=z0)
    r_src = 0.1778 / 2 - dr
    zs = (source_depth if source_depth is not None else z0 + 5.0) - z0
    return Scenario(name=f"realistic well {z0:g}-{z0 + length:g} m", medium=med,
                    source=Source(kind=SOURCE_TORSION, r=r_src, theta=0.0, z=zs, f0=f0),
                    receivers=on_axis_receivers(np.array([0.25, 0.75]) * length), cfl=0.5, steps=steps,
                    params={"z_origin": z0})


def homogeneous(grid: Grid, mat=FLUID) -> Medium:
    return Medium(grid=grid, cell_id=np.zeros(grid.shape, dtype=np.uint16),
                  rho=np.array([mat[0]]), vp=np.array([mat[1]]), vs=np.array([mat[2]]))


def layered_radial(grid: Grid, radii: Sequence[float], mats: Sequence[tuple]) -> Medium:
    """Axisymmetric z-invariant medium: mats[m] for radii[m-1] <= r < radii[m]."""
    rc = grid.r_centre()
    reg = _Registry()
    ids = np.empty(grid.NR, dtype=np.uint16)
    for i, r in enumerate(rc):
        m = int(np.searchsorted(np.asarray(radii), r, side="right"))
        ids[i] = reg.id(mats[min(m, len(mats) - 1)])
    cell_id = np.broadcast_to(ids[None, :, None], grid.shape).copy()
    rho, vp, vs = reg.arrays()
    return Medium(grid=grid, cell_id=cell_id, rho=rho, vp=vp, vs=vs)


def crop_z(medium: Medium, k0: int, nz: int) -> Medium:
    """Sub-well of nz interior cells whose first interior cell is stored cell
    k0 + pml_z of `medium`; PML cells are the neighbouring stored cells."""
    g = medium.grid
    lo = k0
    hi = k0 + nz + 2 * g.pml_z
    if lo < 0 or hi > g.NZ:
        raise ValueError("crop outside the stored grid")
    g2 = replace(g, nz=nz)
    return Medium(grid=g2, cell_id=np.ascontiguousarray(medium.cell_id[:, :, lo:hi]),
                  rho=medium.rho.copy(), vp=medium.vp.copy(), vs=medium.vs.copy())


# ----------------------------------------------------------------------------
# the cased-well workloads

def config1(steps: int = 800) -> Scenario:
    """Small FP64-checkable well: Nr=60 (dr 5 mm) + 10 PML, Nth=16, Nz=300
    (dz 5 mm) + 10 PML per end; cement top at 0.75 m; 10 kHz monopole at
    0.3 m on the axis; 4 axis receivers from 0.4 to 1.2 m; CFL 0.5."""
    g = Grid(nr=60, nth=16, nz=300, pml_r=10, pml_z=10, dr=0.005, dz=0.005)
    med = cased_well(g, z_top=0.75)
    return Scenario(name="cased-well 70x16x320" if steps == 800 else f"cased-well 70x16x320 {steps} steps",
                    medium=med, source=Source(z=0.3, f0=10e3),
                    receivers=on_axis_receivers(np.linspace(0.4, 1.2, 4)), cfl=0.5, steps=steps)


def config1_long() -> Scenario:
    return config1(steps=4000)


def config2(noise_seed: int = 20230227, nz: int = 8192, nr: int = 180) -> Scenario:
    """Full-scale 20 m well, FP32: Nr=180 (dr 2.5 mm) + 16 PML, Nth=64,
    Nz=8192 (dz 2.5 mm) + 16 PML per end, 20000 steps; cement top at 10 m with
    a linear shear ramp 0 -> full over 0.3 m; 8 kHz monopole at 9.75 m; 16 axis
    receivers at 2.0, 2.5, ..., 9.5 m; rock Vp/Vs +-5 % correlated noise.
    `nz` and `nr` shorten the well or its radius (profiling variants)."""
    g = Grid(nr=nr, nth=64, nz=nz, pml_r=16, pml_z=16, dr=0.0025, dz=0.0025)
    L = nz * g.dz
    z_top = 10.0 * L / 20.48
    med = cased_well(g, z_top=z_top, ramp=0.3, top_frac=0.0, noise=Noise(seed=noise_seed))
    zs = z_top - 0.25
    zr = zs - 7.75 + 0.5 * np.arange(16)
    if nz != 8192:  # shortened variants keep the receivers that fit
        zr = zr[zr >= 0.0]
    return Scenario(name=f"cased-well 196x64x{g.NZ}", medium=med, source=Source(z=zs, f0=8e3),
                    receivers=on_axis_receivers(zr), cfl=0.5, steps=20000)


def refinement_rows(grid: Grid, min_nth: int = 4) -> list:
    """Interface rows of the azimuthal refinement of the paper (Sec. 3): the
    azimuthal step halves each time the radius doubles, so going inward from
    the outer radius the node count halves each time the radius halves, from
    grid.nth down to min_nth: zone boundaries at rows NR / 2^k.  A boundary
    that would leave a zone under two rows, or fall inside the radial PML,
    is dropped (the zones keep their node counts from the outside in)."""
    K = 0
    while (grid.nth >> (K + 1)) >= min_nth and (grid.nth >> (K + 1)) % 2 == 0:
        K += 1
    rows = []
    for k in range(K, 0, -1):
        r = int(round(grid.NR / 2 ** k))
        if r >= (rows[-1] if rows else 0) + 2 and r <= grid.nr - 2:
            rows.append(r)
    return rows


def config3_crop(full: Optional[Scenario] = None) -> Scenario:
    """Nz=1024 crop z in [8.0, 10.56) m of the full 20 m well (same noise)."""
    full = full or config2()
    g = full.grid
    k0 = int(round(8.0 / g.dz))
    med = crop_z(full.medium, k0, 1024)
    z0 = k0 * g.dz
    return Scenario(name="cased-well crop 196x64x1056", medium=med,
                    source=Source(z=9.75 - z0, f0=8e3),
                    receivers=on_axis_receivers(np.array([8.0, 8.5, 9.0, 9.5]) - z0),
                    cfl=0.5, steps=20000, params={"z_origin": z0})


def _case_draws(seed: int):
    rng = np.random.default_rng(np.random.SeedSequence([20230227, int(seed)]))
    nz = int(rng.choice([2048, 3072, 4096, 6144]))
    u = rng.random(7)
    return nz, u


def case_features(seed: int) -> np.ndarray:
    """The six surrogate inputs of scenario_case(seed, surrogate_inputs=True)
    from its draws alone (no medium is built): cement-top depth, ramp
    length, top shear fraction, casing thickness, cement Vs, rock Vs."""
    nz, u = _case_draws(seed)
    length = nz * 0.0025
    return np.array([(0.3 + 0.4 * u[0]) * length, 0.5 * u[1], float(u[2]), 0.008 + 0.004 * u[3],
                     CEMENT[2] * (0.9 + 0.2 * u[4]), ROCK[2] * (0.9 + 0.2 * u[5])], dtype=np.float64)


def scenario_case(seed: int, surrogate_inputs: bool = False) -> Scenario:
    """One cement-hardening case: Nr=120 (dr 2.5 mm) + 16 PML, Nth=32,
    Nz in {2048, 3072, 4096, 6144} (dz 2.5 mm) + 16 PML per end; top depth
    U(0.3, 0.7) * length, ramp U(0, 0.5) m, top shear fraction U(0, 1),
    casing thickness U(8, 12) mm; with `surrogate_inputs` also cement and
    rock Vs scaled by U(0.9, 1.1) at fixed Vp/Vs and density.  8 kHz axis
    monopole 0.075 m above the top, 8 axis receivers 15 mm apart above it;
    6000 steps at CFL 0.5."""
    nz, u = _case_draws(seed)
    g = Grid(nr=120, nth=32, nz=nz, pml_r=16, pml_z=16, dr=0.0025, dz=0.0025)
    length = nz * g.dz
    z_top = (0.3 + 0.4 * u[0]) * length
    ramp = 0.5 * u[1]
    frac = float(u[2])
    t = 0.008 + 0.004 * u[3]
    cement, rock = CEMENT, ROCK
    cvs = rvs = 1.0
    if surrogate_inputs:
        cvs = 0.9 + 0.2 * u[4]
        rvs = 0.9 + 0.2 * u[5]
        cement = (CEMENT[0], CEMENT[1] * cvs, CEMENT[2] * cvs)
        rock = (ROCK[0], ROCK[1] * rvs, ROCK[2] * rvs)
    med = cased_well(g, z_top=z_top, ramp=ramp, top_frac=frac, casing_t=t, cement=cement, rock=rock)
    zs = z_top - 0.075
    zr = zs - 0.015 * np.arange(1, 9)
    params = dict(seed=int(seed), nz=nz, z_top=z_top, ramp=ramp, top_frac=frac, casing_t=t,
                  cement_vs=cement[2], rock_vs=rock[2])
    return Scenario(name=f"case{seed}", medium=med, source=Source(z=zs, f0=8e3),
                    receivers=on_axis_receivers(zr), cfl=0.5, steps=6000, params=params)


def reach_crop(sc: Scenario, reach: float = 1.6) -> Scenario:
    """The part of a well that can reach its receivers within its window:
    the interior z cells within `reach` metres of the span of the source and
    the receivers (clamped to the well; the crop's z PML are the neighbouring
    stored cells, the well's own PML where the crop meets its end).  A wave
    that leaves the span and comes back travels at most c T_end, so with
    reach > c_max T_end / 2 nothing beyond the crop can arrive inside the
    window (the cement cases: 5900 m/s x 0.486 ms / 2 = 1.43 m < 1.6 m).
    params gain k0 (first interior cell of the crop in the well) and keep
    the well's own entries."""
    g = sc.grid
    zs = np.concatenate([[sc.source.z], np.asarray(sc.receivers.z)])
    k0 = max(0, int(np.floor((zs.min() - reach) / g.dz)))
    k1 = min(g.nz, int(np.ceil((zs.max() + reach) / g.dz)) + 1)
    med = crop_z(sc.medium, k0, k1 - k0)
    z0 = k0 * g.dz
    src = replace(sc.source, z=sc.source.z - z0)
    rec = Receivers(r=np.asarray(sc.receivers.r).copy(), theta=np.asarray(sc.receivers.theta).copy(),
                    z=np.asarray(sc.receivers.z) - z0, quantity=sc.receivers.quantity)
    params = dict(sc.params)
    params["k0"] = k0
    return Scenario(name=sc.name + " crop", medium=med, source=src, receivers=rec, cfl=sc.cfl, steps=sc.steps,
                    pml_on=sc.pml_on, params=params)


def small_cement_case(seed: int, steps: int = 1200) -> Scenario:
    """Miniature of the cement-hardening family: 5 mm cells, Nr = 36 + 8 PML,
    Ntheta = 8, Nz = 240 + 8 PML per end; top depth U(0.55, 0.65) m, ramp
    U(0, 0.2) m, top shear fraction U(0, 1), casing thickness U(8, 12) mm,
    cement and rock Vs scaled by U(0.9, 1.1); 8 kHz axis monopole 0.075 m above
    the top, 4 axis receivers 15 mm apart above it.  params holds the six
    surrogate inputs."""
    rng = np.random.default_rng(np.random.SeedSequence([2302, 13907, int(seed)]))
    u = rng.random(6)
    g = Grid(nr=36, nth=8, nz=240, pml_r=8, pml_z=8, dr=0.005, dz=0.005)
    z_top = 0.55 + 0.10 * u[0]
    ramp = 0.2 * u[1]
    frac = float(u[2])
    t = 0.008 + 0.004 * u[3]
    cvs, rvs = 0.9 + 0.2 * u[4], 0.9 + 0.2 * u[5]
    cement = (CEMENT[0], CEMENT[1] * cvs, CEMENT[2] * cvs)
    rock = (ROCK[0], ROCK[1] * rvs, ROCK[2] * rvs)
    med = cased_well(g, z_top=z_top, ramp=ramp, top_frac=frac, casing_t=t, cement=cement, rock=rock)
    zs = z_top - 0.075
    params = dict(seed=int(seed), nz=g.nz, z_top=z_top, ramp=ramp, top_frac=frac, casing_t=t,
                  cement_vs=cement[2], rock_vs=rock[2])
    return Scenario(name=f"small{seed}", medium=med, source=Source(z=zs, f0=8e3),
                    receivers=on_axis_receivers(zs - 0.015 * np.arange(1, 5)), cfl=0.5, steps=steps, params=params)


def surrogate_features(sc: Scenario) -> np.ndarray:
    """The six surrogate inputs: cement-top depth, ramp length, top shear
    fraction, casing thickness, cement Vs, rock Vs."""
    p = sc.params
    return np.array([p["z_top"], p["ramp"], p["top_frac"], p["casing_t"], p["cement_vs"], p["rock_vs"]],
                    dtype=np.float64)
