"""Test-side helpers: discrete energy of the scheme and trace metrics.

The energy is written from the definition of the staggered scheme's
quadratic invariant (r-weighted kinetic energy with the two-cell density
mean, compliance energy with the cell Lame moduli and the four-cell harmonic
shear modulus), independently of the oracle's code.
"""
import numpy as np


def lame(medium):
    rho = medium.rho
    mu = rho * medium.vs ** 2
    lam = rho * medium.vp ** 2 - 2 * mu
    return rho, lam, mu


def node_coefficients(medium):
    """Per-node density means and shear-modulus harmonic means (R5)."""
    g = medium.grid
    rho_t, lam_t, mu_t = lame(medium)
    cid = medium.cell_id.astype(np.int64)
    rho = rho_t[cid]
    lam = lam_t[cid]
    mu = mu_t[cid]

    def jp(a):
        return np.roll(a, -1, axis=0)

    def hm(a, b, c, d):
        out = np.zeros_like(a)
        ok = (a > 0) & (b > 0) & (c > 0) & (d > 0)
        out[ok] = 4.0 / (1 / a[ok] + 1 / b[ok] + 1 / c[ok] + 1 / d[ok])
        return out

    nth, NR, NZ = g.shape
    rho_vr = np.full(g.shape, np.nan)
    rho_vr[:, 1:, :] = 0.5 * (rho[:, :-1, :] + rho[:, 1:, :])
    rho_vp = 0.5 * (rho + jp(rho))
    rho_vz = np.full(g.shape, np.nan)
    rho_vz[:, :, :-1] = 0.5 * (rho[:, :, :-1] + rho[:, :, 1:])
    mu_rp = np.zeros(g.shape)
    mu_rp[:, 1:, :] = hm(mu[:, :-1, :], mu[:, 1:, :], jp(mu)[:, :-1, :], jp(mu)[:, 1:, :])
    mu_rz = np.zeros(g.shape)
    mu_rz[:, 1:, :-1] = hm(mu[:, :-1, :-1], mu[:, 1:, :-1], mu[:, :-1, 1:], mu[:, 1:, 1:])
    mu_pz = np.zeros(g.shape)
    mu_pz[:, :, :-1] = hm(mu[:, :, :-1], jp(mu)[:, :, :-1], mu[:, :, 1:], jp(mu)[:, :, 1:])
    return dict(rho=rho, lam=lam, mu=mu, rho_vr=rho_vr, rho_vp=rho_vp, rho_vz=rho_vz,
                mu_rp=mu_rp, mu_rz=mu_rz, mu_pz=mu_pz)


def weights(grid):
    ri = np.arange(grid.NR) * grid.dr
    rh = (np.arange(grid.NR) + 0.5) * grid.dr
    dv = grid.dr * (2 * np.pi / grid.nth) * grid.dz
    return ri[None, :, None] * dv, rh[None, :, None] * dv


def energy(coef, grid, v_old, v_new, s):
    """E^n = 1/2 sum w rho v^{n-1/2}.v^{n+1/2} + sum w W(s^n)."""
    wi, wh = weights(grid)
    return energy_terms(coef, wi, wh, v_old, v_new, s, axis=True)


def energy_terms(coef, wi, wh, v_old, v_new, s, axis):
    """The same sum over one block of rows with node weights wi (r_i nodes)
    and wh (r_{i+1/2} nodes); `axis`: the block's first row is ring 0, whose
    v_r is not an unknown."""
    kin = 0.0
    a0 = 1 if axis else 0
    a = v_old["vr"][:, a0:, :] * v_new["vr"][:, a0:, :] * coef["rho_vr"][:, a0:, :] * wi[:, a0:, :]
    kin += a.sum()
    kin += (v_old["vp"] * v_new["vp"] * coef["rho_vp"] * wh).sum()
    kin += (v_old["vz"][:, :, :-1] * v_new["vz"][:, :, :-1] * coef["rho_vz"][:, :, :-1] * wh).sum()
    kin *= 0.5
    lam, mu = coef["lam"], coef["mu"]
    K = lam + 2 * mu / 3
    tr = s["srr"] + s["spp"] + s["szz"]
    w = tr ** 2 / (18 * K)
    solid = mu > 0
    dev = ((s["srr"] - tr / 3) ** 2 + (s["spp"] - tr / 3) ** 2 + (s["szz"] - tr / 3) ** 2)
    w = w + np.where(solid, dev / (4 * np.where(solid, mu, 1.0)), 0.0)
    pot = (w * wh).sum()

    def shear(sig, m, ww):
        ok = m > 0
        return (np.where(ok, sig ** 2 / (2 * np.where(ok, m, 1.0)), 0.0) * ww).sum()

    pot += shear(s["srp"], coef["mu_rp"], wi)
    pot += shear(s["srz"], coef["mu_rz"], wi)
    pot += shear(s["spz"], coef["mu_pz"], wh)
    return kin + pot


def random_admissible_state(medium, seed):
    """Random fields that respect the liquid constraint (isotropic stress,
    zero shear where the node's shear modulus vanishes) and the walls."""
    g = medium.grid
    coef = node_coefficients(medium)
    rng = np.random.default_rng(seed)
    f = {n: rng.standard_normal(g.shape) for n in ("vr", "vp", "vz", "srr", "spp", "szz", "srp", "spz", "srz")}
    for n in ("vr", "vp", "vz"):
        f[n] *= 1e-3
    f["vr"][:, 0, :] = 0
    f["vz"][:, :, -1] = 0
    fluid = coef["mu"] == 0
    f["spp"][fluid] = f["srr"][fluid]
    f["szz"][fluid] = f["srr"][fluid]
    f["srp"][coef["mu_rp"] == 0] = 0
    f["srz"][coef["mu_rz"] == 0] = 0
    f["spz"][coef["mu_pz"] == 0] = 0
    return f, coef


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ----------------------------------------------------------- refined grid
def zone_blocks(medium, rows):
    """The zones of the azimuthally refined grid whose zones 1 .. M-1 start at
    `rows`: (first row, rows, nth, cell IDs [nth][rows][NZ] with, below zone
    m > 0, the coarse zone's last row seen from the fine nodes (fine node j ->
    coarse cell floor(j/2)) prepended).  Zone m samples the finest grid at its
    own nodes."""
    g = medium.grid
    M = len(rows) + 1
    row0 = [0] + list(rows) + [g.NR]
    out = []
    for m in range(M):
        nth = g.nth >> (M - 1 - m)
        cid = medium.cell_id[:: g.nth // nth, row0[m]:row0[m + 1], :]
        if m > 0:
            stride_a = g.nth // (nth // 2)
            ghost = medium.cell_id[(np.arange(nth) // 2) * stride_a, row0[m] - 1, :]
            cid = np.concatenate([ghost[:, None, :], cid], axis=1)
        out.append((row0[m], row0[m + 1] - row0[m], nth, cid))
    return out


class _Block:
    def __init__(self, medium, nth, cid):
        self.rho, self.vp, self.vs = medium.rho, medium.vp, medium.vs
        self.cell_id = cid
        self.grid = type("G", (), {"shape": cid.shape})()


def refined_coefficients(medium, rows):
    """Per zone: node coefficients of its own rows (R5 with the ghost cells of R14)."""
    out = []
    for row, n, nth, cid in zone_blocks(medium, rows):
        c = node_coefficients(_Block(medium, nth, cid))
        if cid.shape[1] > n:
            c = {k: v[:, 1:, :] for k, v in c.items()}
        out.append((row, n, nth, c))
    return out


def energy_refined(grid, zcoef, v_old, v_new, s):
    """Energy of the refined grid: the sum over zones, each with its own
    azimuthal step; fields are dicts of per-zone arrays."""
    E = 0.0
    for m, (row, n, nth, c) in enumerate(zcoef):
        ri = (row + np.arange(n)) * grid.dr
        rh = (row + np.arange(n) + 0.5) * grid.dr
        dv = grid.dr * (2 * np.pi / nth) * grid.dz
        pick = lambda d: {k: v[m] for k, v in d.items()}
        E += energy_terms(c, ri[None, :, None] * dv, rh[None, :, None] * dv, pick(v_old), pick(v_new), pick(s),
                          axis=row == 0)
    return E
