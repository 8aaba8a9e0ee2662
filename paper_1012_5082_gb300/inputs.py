"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no part of the Monte Carlo method: it only builds the
inputs the method is applied to -- lattice positions, initial species,
EAM tables sampled from closed-form functions, nanocrystal geometries and
Maxwell velocities.  Both sides of every parity test receive exactly the
arrays produced here.

Units: Angstrom, eV, K, fs, amu.  Species 0 = A (solvent), 1 = B (solute).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KB_EV = 8.617333262e-5          # Boltzmann constant (eV/K)
FTM = 9.648533212331e-3         # eV/(Angstrom amu) -> Angstrom/fs^2
MASS_A = 55.845                 # amu (Fe, the paper's solvent)
MASS_B = 63.546                 # amu (Cu, the paper's solute)


# --------------------------------------------------------------- lattices
@dataclasses.dataclass
class Lattice:
    """Sites of a periodic orthorhombic cell, stored as SoA float64 arrays."""

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    box: np.ndarray                 # (3,) box lengths
    cells: tuple | None = None      # (nx, ny, nz) for a rigid BCC lattice
    a: float | None = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def bcc_lattice(nx: int, ny: int, nz: int, a: float = 2.855) -> Lattice:
    """Rigid BCC lattice; site i = ((cz*ny + cy)*nx + cx)*2 + b at
    a*(cx + b/2, cy + b/2, cz + b/2)."""
    cz, cy, cx, b = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), np.arange(2),
                                indexing="ij")
    cx = cx.ravel().astype(np.float64)
    cy = cy.ravel().astype(np.float64)
    cz = cz.ravel().astype(np.float64)
    h = 0.5 * b.ravel().astype(np.float64)
    return Lattice(x=a * (cx + h), y=a * (cy + h), z=a * (cz + h),
                   box=np.array([nx * a, ny * a, nz * a], dtype=np.float64),
                   cells=(nx, ny, nz), a=a)


def random_types(n: int, n_b: int, seed: int) -> np.ndarray:
    """n sites, exactly n_b of them species B, placed uniformly at random."""
    rng = np.random.default_rng(seed)
    t = np.zeros(n, dtype=np.uint8)
    t[rng.choice(n, size=n_b, replace=False)] = 1
    return t


# ------------------------------------------------------------- EAM tables
@dataclasses.dataclass
class EAMTables:
    """EAM functions sampled on uniform grids, with knot derivatives.

    pair[p] for p = t_i + t_j (0 AA, 1 AB, 2 BB) on r_j = j*dr;
    dens[t] on the same grid; embed[t] on rho_j = j*drho."""

    rc: float
    nr: int
    dr: float
    nrho: int
    drho: float
    pair: list
    dpair: list
    dens: list
    ddens: list
    embed: list
    dembed: list

    def arrays(self):
        return (self.pair + self.dpair + self.dens + self.ddens + self.embed + self.dembed)


@dataclasses.dataclass
class EAMParams:
    """Closed-form synthetic EAM: Morse pair D*s_ab*(e^{-2al(r-r0)} - 2e^{-al(r-r0)}),
    density f(r) = exp(-beta_f (r/re - 1)), embedding F(rho) = -A sqrt(rho) +
    c2 rho^2, pair and density multiplied by the quintic taper
    1 - 10x^3 + 15x^4 - 6x^5 on [r_in, rc]."""

    D: float = 0.4
    alpha: float = 1.4
    r0: float = 2.5
    pair_scale: tuple = (1.0, 0.85, 0.9)     # AA, AB, BB
    beta_f: float = 3.0
    re: float = 2.47
    dens_scale: tuple = (1.0, 1.0)           # f_A, f_B multipliers
    A_embed: tuple = (1.8, 1.5)              # A, B
    c2: float = 1e-3
    rc: float = 5.3
    r_in: float = 5.0
    nr: int = 5000
    nrho: int = 5000
    rho_max: float = 50.0

    # closed forms (value, derivative); used to sample the tables and by tests
    def taper(self, r):
        r = np.asarray(r, dtype=np.float64)
        w = self.rc - self.r_in
        x = np.clip((r - self.r_in) / w, 0.0, 1.0)
        psi = 1 - 10 * x**3 + 15 * x**4 - 6 * x**5
        dpsi = (-30 * x**2 + 60 * x**3 - 30 * x**4) / w
        return psi, dpsi

    def morse(self, p, r):
        r = np.asarray(r, dtype=np.float64)
        e1 = np.exp(-self.alpha * (r - self.r0))
        v = self.D * self.pair_scale[p] * (e1 * e1 - 2 * e1)
        dv = self.D * self.pair_scale[p] * (-2 * self.alpha * e1 * e1 + 2 * self.alpha * e1)
        return v, dv

    def pair(self, p, r):
        v, dv = self.morse(p, r)
        psi, dpsi = self.taper(r)
        return v * psi, dv * psi + v * dpsi

    def dens(self, t, r):
        r = np.asarray(r, dtype=np.float64)
        f = self.dens_scale[t] * np.exp(-self.beta_f * (r / self.re - 1.0))
        df = -self.beta_f / self.re * f
        psi, dpsi = self.taper(r)
        return f * psi, df * psi + f * dpsi

    def embed(self, t, rho):
        rho = np.asarray(rho, dtype=np.float64)
        v = -self.A_embed[t] * np.sqrt(rho) + self.c2 * rho * rho
        with np.errstate(divide="ignore"):
            dv = -0.5 * self.A_embed[t] / np.sqrt(rho) + 2 * self.c2 * rho
        return v, dv


def eam_tables(p: EAMParams | None = None) -> EAMTables:
    """Sample the closed-form EAM on uniform grids (values and derivatives).

    The embedding derivative is infinite at rho = 0; knot 0 takes the secant
    slope of the first interval instead."""
    p = p or EAMParams()
    dr = p.rc / (p.nr - 1)
    r = np.arange(p.nr, dtype=np.float64) * dr
    drho = p.rho_max / (p.nrho - 1)
    rho = np.arange(p.nrho, dtype=np.float64) * drho
    pair, dpair, dens, ddens, emb, demb = [], [], [], [], [], []
    K = len(p.A_embed)
    assert len(p.pair_scale) == K * (K + 1) // 2 and len(p.dens_scale) == K
    for q in range(len(p.pair_scale)):
        v, dv = p.pair(q, r)
        pair.append(np.ascontiguousarray(v))
        dpair.append(np.ascontiguousarray(dv))
    for t in range(K):
        v, dv = p.dens(t, r)
        dens.append(np.ascontiguousarray(v))
        ddens.append(np.ascontiguousarray(dv))
        v, dv = p.embed(t, rho)
        dv = dv.copy()
        dv[0] = (v[1] - v[0]) / drho
        emb.append(np.ascontiguousarray(v))
        demb.append(np.ascontiguousarray(dv))
    return EAMTables(rc=p.rc, nr=p.nr, dr=dr, nrho=p.nrho, drho=drho, pair=pair, dpair=dpair,
                     dens=dens, ddens=ddens, embed=emb, dembed=demb)


def npt_eam_params(**kw) -> EAMParams:
    """The synthetic EAM with the embedding's rho^2 coefficient raised from
    1e-3 to 0.0119446 so that the perfect BCC crystal at a = 2.855 A is at
    zero pressure and mechanically stable (the workloads' coefficient leaves
    it at about -880 kbar, with the energy falling under compression): for
    constant-pressure MD."""
    return EAMParams(c2=0.0119446, **kw)


def multi_eam_params(K: int, dens_scale=None, **kw) -> EAMParams:
    """K-species form of the synthetic EAM (K = 2..4): the binary's A and B
    plus C and D.  Pair scales in the order (0,0), (0,1), ..., (K-1,K-1);
    for K = 2 the binary parameters exactly."""
    scale = {(0, 0): 1.0, (0, 1): 0.85, (1, 1): 0.9, (0, 2): 0.8, (1, 2): 0.75, (2, 2): 0.95,
             (0, 3): 0.9, (1, 3): 0.8, (2, 3): 0.85, (3, 3): 1.05}
    A = (1.8, 1.5, 1.65, 1.95)
    pairs = tuple(scale[(a, b)] for a in range(K) for b in range(a, K))
    ds = tuple(dens_scale) if dens_scale is not None else (1.0,) * K
    return EAMParams(pair_scale=pairs, A_embed=A[:K], dens_scale=ds, **kw)


def multi_random_types(n: int, counts, seed: int) -> np.ndarray:
    """Species 0 everywhere except counts[q] sites of species q + 1, placed
    uniformly at random (a seeded permutation)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    t = np.zeros(n, dtype=np.uint8)
    k = 0
    for q, c in enumerate(counts):
        t[perm[k:k + c]] = q + 1
        k += c
    return t


# ------------------------------------------------- Ising lattice gas
@dataclasses.dataclass
class IsingParams:
    """Pair-only lattice gas on BCC up to the second neighbour shell (the
    paper's Ising-type model, Sec. II B): eps_ab(1), eps_ab(2) in units of U
    for ab = AA, AB, BB; no density, no embedding.  The pair tables are flat
    at eps(1) around the first shell (a sqrt(3)/2) and at eps(2) around the
    second (a), joined by quintic smoothsteps, and fall to zero before r_c,
    so the splines return the exact shell values."""

    U: float = 0.1                          # eV (k_B T = 0.8617 U at T = 1000 K)
    eps1: tuple = (-10.0, -9.7, -10.0)
    eps2: tuple = (-2.0, -2.0, -2.0)
    a: float = 2.855
    rc: float = 3.5
    nr: int = 2000
    steps: tuple = (2.60, 2.75, 3.05, 3.35)  # eps1 -> eps2 on [s0, s1], eps2 -> 0 on [s2, s3]

    def pair(self, p, r):
        r = np.asarray(r, dtype=np.float64)

        def step(lo, hi):
            x = np.clip((r - lo) / (hi - lo), 0.0, 1.0)
            return 10 * x**3 - 15 * x**4 + 6 * x**5, (30 * x**2 - 60 * x**3 + 30 * x**4) / (hi - lo)

        s0, s1, s2, s3 = self.steps
        e1, e2 = self.eps1[p] * self.U, self.eps2[p] * self.U
        a1, da1 = step(s0, s1)
        a2, da2 = step(s2, s3)
        v = (e1 + (e2 - e1) * a1) * (1.0 - a2)
        dv = (e2 - e1) * da1 * (1.0 - a2) - (e1 + (e2 - e1) * a1) * da2
        return v, dv


def ising_tables(p: IsingParams | None = None) -> EAMTables:
    """EAMTables of the lattice gas (zero density and embedding)."""
    p = p or IsingParams()
    dr = p.rc / (p.nr - 1)
    r = np.arange(p.nr, dtype=np.float64) * dr
    pair, dpair = [], []
    for q in range(3):
        v, dv = p.pair(q, r)
        pair.append(np.ascontiguousarray(v))
        dpair.append(np.ascontiguousarray(dv))
    nrho, rho_max = 64, 1.0
    zr, zrho = np.zeros(p.nr), np.zeros(nrho)
    return EAMTables(rc=p.rc, nr=p.nr, dr=dr, nrho=nrho, drho=rho_max / (nrho - 1), pair=pair, dpair=dpair,
                     dens=[zr.copy(), zr.copy()], ddens=[zr.copy(), zr.copy()],
                     embed=[zrho.copy(), zrho.copy()], dembed=[zrho.copy(), zrho.copy()])


# ------------------------------------------------------------ nanocrystal
def _haar_rotations(rng, k):
    """k rotation matrices uniformly distributed on SO(3) (unit quaternions
    drawn from a 4-d Gaussian)."""
    q = rng.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def nanocrystal(L: float, n_grains: int, a: float = 2.855, seed: int = 1002,
                dmin: float = 2.0) -> Lattice:
    """Periodic cube of side L filled with n_grains BCC Voronoi grains.

    Grain centres are uniform in the cube, orientations uniform on SO(3).
    Each grain's lattice (through its centre) is kept where the grain centre
    is the nearest centre under the minimum image.  Of any two atoms closer
    than dmin the later-indexed one is removed."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, L, size=(n_grains, 3))
    rots = _haar_rotations(rng, n_grains)
    # lattice points of a cube of half-width R around each centre
    R = L * math.sqrt(3.0) / 2.0 + a
    m = int(math.ceil(R / a))
    g = np.arange(-m, m + 1, dtype=np.float64)
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    base = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1) * a
    motif = np.concatenate([base, base + 0.5 * a], axis=0)
    keep_pts = []
    for k in range(n_grains):
        pts = motif @ rots[k].T + centres[k]
        pts = pts[np.all((pts >= centres[k] - L / 2) & (pts < centres[k] + L / 2), axis=1)]
        # nearest centre under the minimum image
        best = None
        for q in range(n_grains):
            d = pts - centres[q]
            d -= L * np.round(d / L)
            r2 = np.einsum("ij,ij->i", d, d)
            best = r2 if best is None else np.minimum(best, r2)
            if q == k:
                own = r2
        sel = own <= best
        pts = np.mod(pts[sel], L)
        keep_pts.append(pts)
    pos = np.concatenate(keep_pts, axis=0)
    pos = _remove_close(pos, L, dmin)
    return Lattice(x=np.ascontiguousarray(pos[:, 0]), y=np.ascontiguousarray(pos[:, 1]),
                   z=np.ascontiguousarray(pos[:, 2]), box=np.array([L, L, L]), a=a)


def _remove_close(pos: np.ndarray, L: float, dmin: float) -> np.ndarray:
    """Drop the later-indexed atom of every pair closer than dmin (periodic)."""
    from scipy.spatial import cKDTree

    pos = np.mod(pos, L)
    pos[pos >= L] = 0.0
    pairs = cKDTree(pos, boxsize=L).query_pairs(dmin, output_type="ndarray")
    alive = np.ones(len(pos), dtype=bool)
    if len(pairs):
        alive[pairs.max(axis=1)] = False
    return pos[alive]


def maxwell_velocities(types: np.ndarray, T: float, seed: int,
                       masses=(MASS_A, MASS_B)) -> tuple:
    """Velocities (Angstrom/fs) from the Maxwell distribution at T, with the
    centre-of-mass momentum removed."""
    rng = np.random.default_rng(seed)
    m = np.where(types == 1, masses[1], masses[0]).astype(np.float64)
    sig = np.sqrt(KB_EV * T * FTM / m)
    v = rng.normal(size=(types.shape[0], 3)) * sig[:, None]
    p = (v * m[:, None]).sum(axis=0) / m.sum()
    v -= p[None, :]
    return (np.ascontiguousarray(v[:, 0]), np.ascontiguousarray(v[:, 1]),
            np.ascontiguousarray(v[:, 2]))


MLP_IN, MLP_H = 10, 64
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1


def mlp_init(seed: int, out_bias: float = 0.0) -> np.ndarray:
    """Initial parameters of the 10 -> 64 -> 64 -> 1 surrogate network in the
    packed order W1[64][10], b1, W2[64][64], b2, w3[64], b3: Glorot-uniform
    weights, zero biases, b3 = out_bias (float32)."""
    rng = np.random.default_rng(seed)

    def glorot(fan_out, fan_in):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size=fan_out * fan_in)

    parts = [glorot(MLP_H, MLP_IN), np.zeros(MLP_H), glorot(MLP_H, MLP_H), np.zeros(MLP_H),
             glorot(1, MLP_H), [out_bias]]
    return np.concatenate(parts).astype(np.float32)
