"""Seeded synthetic inputs: Si/C structures, Maxwell-Boltzmann velocities and
parameter-file loading.

This module only generates inputs. It holds lattice geometry, random
displacements and placements, and Gaussian velocity draws, and none of the
potential's arithmetic (no cutoff, bond order, charge or force code). Both the
CUDA path and the CPU checker read the arrays it returns.

The structures stand in for the shapes of the paper's MD cells (Sec. 3.3: a
stepped 4H-SiC(0001) substrate of about 12,000 atoms with a fixed bottom; the
fitting-set shapes of Sec. 2: SiC crystals, amorphous C, graphene, clusters).
The paper ships no structure files, so every structure here is generated from
ideal tetrahedral geometry at a = 4.36 A.

Units: A, fs, u, eV, e. Types: 0 = Si, 1 = C.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

SI, C = 0, 1
TYPE_NAMES = ("Si", "C")
# IUPAC standard atomic weights (u)
MASS = np.array([28.0855, 12.011])
KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
EV_PER_U_TO_A2_FS2 = 9.648533212e-3  # 1 eV/u expressed in A^2/fs^2

_PARAM_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "params")


@dataclass
class Structure:
    """One periodic or open atomic configuration.

    x: (N,3) float64 positions (A); types: (N,) int32; box: (3,) float64
    orthorhombic edge lengths (ignored along non-periodic axes);
    pbc: (3,) bool; frozen: (N,) bool atoms held fixed by the integrator.
    """
    name: str
    x: np.ndarray
    types: np.ndarray
    box: np.ndarray
    pbc: np.ndarray
    frozen: np.ndarray = None
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.x = np.ascontiguousarray(self.x, dtype=np.float64)
        self.types = np.ascontiguousarray(self.types, dtype=np.int32)
        self.box = np.asarray(self.box, dtype=np.float64)
        self.pbc = np.asarray(self.pbc, dtype=bool)
        if self.frozen is None:
            self.frozen = np.zeros(len(self.types), dtype=bool)
        self.frozen = np.ascontiguousarray(self.frozen, dtype=bool)

    @property
    def n(self) -> int:
        return int(self.types.shape[0])


def load_params(name: str = "p1") -> dict:
    """Load a parameter set (JSON) shipped with the package."""
    path = name if os.path.isfile(name) else os.path.join(_PARAM_DIR, f"{name}.json")
    with open(path) as fh:
        return json.load(fh)


# --------------------------------------------------------------------------
# 3C-SiC bulk
# --------------------------------------------------------------------------
def sic_3c(ncell: int = 4, a: float = 4.36, disp: float = 0.05, seed: int = 1,
           strain=None) -> Structure:
    """Zincblende SiC, ncell^3 conventional cubic cells (or n1 x n2 x n3 for
    a 3-tuple ncell), periodic.

    Si on the fcc sites, C on the fcc sites shifted by a(1/4,1/4,1/4). Every
    coordinate is displaced by U(-disp, +disp) from a seeded generator.
    strain: optional (3,3) symmetric strain applied as x -> (I + eps) x
    (the box must stay orthorhombic, so only the diagonal is accepted).
    """
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    basis = np.concatenate([fcc, fcc + 0.25])
    btype = np.array([SI] * 4 + [C] * 4, dtype=np.int32)
    nc = np.broadcast_to(np.asarray(ncell, dtype=int), (3,))
    cells = np.stack(np.meshgrid(*(np.arange(k) for k in nc), indexing="ij"), -1).reshape(-1, 3)
    frac = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    x = frac * a
    types = np.tile(btype, len(cells))
    rng = np.random.default_rng(seed)
    x = x + rng.uniform(-disp, disp, size=x.shape)
    box = nc * a
    if strain is not None:
        eps = np.asarray(strain, dtype=np.float64)
        if np.any(np.abs(eps - np.diag(np.diag(eps))) > 0):
            raise ValueError("only diagonal strain keeps the box orthorhombic")
        f = 1.0 + np.diag(eps)
        x = x * f
        box = box * f
    x = np.mod(x, box)
    return Structure(f"3C-SiC {nc[0]}x{nc[1]}x{nc[2]}", x, types, box,
                     np.array([True, True, True]))


def sic_3c_110(rep=(1, 1, 1), a: float = 4.36, stretch_x: float = 0.0) -> Structure:
    """Zincblende SiC in the frame x = [110]/sqrt2, y = [-110]/sqrt2, z = [001]:
    a periodic tetragonal cell a/sqrt2 x a/sqrt2 x a holding 2 Si and 2 C,
    replicated rep times. A strain along this x is a shear of the cubic
    axes, so the cell carries the elastic constant C44. stretch_x scales
    x (positions and box) by 1 + stretch_x."""
    ah = a / math.sqrt(2.0)
    # cubic-frame fractional sites of the 4 atoms, mapped to the rotated cell:
    # Si at (0,0,0) and (1/2,1/2,0)a; C at (1/4,1/4,1/4) and (3/4,3/4,3/4)a
    # minus a lattice vector, so that every atom lies inside the cell
    cub = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.5], [0.25, 0.25, 0.25], [0.75, 0.25, 0.75]]) * a
    rot = np.array([[1.0, 1.0, 0.0], [-1.0, 1.0, 0.0], [0.0, 0.0, math.sqrt(2.0)]]) / math.sqrt(2.0)
    box1 = np.array([ah, ah, a])
    x1 = np.mod(cub @ rot.T, box1)
    t1 = np.array([SI, SI, C, C], dtype=np.int32)
    rep = np.broadcast_to(np.asarray(rep, dtype=int), (3,))
    cells = np.stack(np.meshgrid(*(np.arange(k) for k in rep), indexing="ij"), -1).reshape(-1, 3)
    x = (cells[:, None, :] * box1 + x1[None, :, :]).reshape(-1, 3)
    types = np.tile(t1, len(cells))
    box = box1 * rep
    f = np.array([1.0 + stretch_x, 1.0, 1.0])
    return Structure(f"3C-SiC [110] cell {rep[0]}x{rep[1]}x{rep[2]}", x * f, types, box * f,
                     np.array([True, True, True]))


def sic_4h_bulk(nx: int = 1, ny: int = 1, n_periods: int = 1, a: float = 4.36) -> Structure:
    """Periodic 4H-SiC: the slab geometry of sic_4h_slab (orthorhombic
    a_h x sqrt(3) a_h in-plane cell, ABCB stacking, bilayer period a/sqrt(3))
    with 4 n_periods bilayers and the z axis periodic (box c = 4 n_periods
    a/sqrt(3)): the top Si bonds straight up to the C of the next period's
    bottom bilayer. 16 nx ny n_periods atoms, ideal positions."""
    P = a / math.sqrt(3.0)
    s = sic_4h_slab(nx, ny, 4 * n_periods, a=a, n_frozen_bilayers=0)
    x = s.x.copy()
    x[:, 2] -= x[:, 2].min()
    box = np.array([s.box[0], s.box[1], 4 * n_periods * P])
    return Structure(f"4H-SiC bulk {nx}x{ny}x{n_periods}", x, s.types, box, np.array([True, True, True]))


# --------------------------------------------------------------------------
# 4H-SiC(0001) Si-face slabs
# --------------------------------------------------------------------------
# In-plane sites of a hexagonal close-packed plane, in units of the
# orthorhombic cell (a_h, sqrt(3) a_h); two lattice points per cell.
_SITE = {
    "A": np.array([[0.0, 0.0], [0.5, 0.5]]),
    "B": np.array([[0.5, 1.0 / 6.0], [0.0, 2.0 / 3.0]]),
    "C": np.array([[0.0, 1.0 / 3.0], [0.5, 5.0 / 6.0]]),
}
_STACK_4H = "ABCB"


def sic_4h_slab(nx: int, ny: int, n_bilayers: int, a: float = 4.36,
                step: str | None = None, n_frozen_bilayers: int = 2,
                vacuum: float = 15.0) -> Structure:
    """4H-SiC(0001) Si-terminated slab, periodic in x/y, open in z.

    Orthorhombic in-plane cell a_h x sqrt(3) a_h with a_h = a/sqrt(2), four
    atoms per bilayer per cell. Bilayer m holds a C plane on stacking site
    S_m at z = m P and a Si plane on site S_(m+1) at z = m P + P/4
    (P = a/sqrt(3)); the Si of bilayer m bonds straight up to the C of
    bilayer m+1 (length 3P/4). The top plane is Si (Si face).

    step: None (flat), "strip" (top bilayer kept only for x < Lx/2: two step
    edges along y), or "staircase" (strip s = floor(4x/Lx) loses its top s
    bilayers: three one-bilayer down-steps and one three-bilayer step at the
    periodic boundary).
    Bottom n_frozen_bilayers bilayers are marked frozen.
    """
    ah = a / math.sqrt(2.0)
    P = a / math.sqrt(3.0)
    Lx, Ly = nx * ah, ny * ah * math.sqrt(3.0)
    gx, gy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    cells = np.stack([gx.ravel(), gy.ravel()], -1).astype(np.float64)
    xs, ts, layer = [], [], []
    for m in range(n_bilayers):
        for plane, (typ, site, dz) in enumerate(
                ((C, _STACK_4H[m % 4], 0.0), (SI, _STACK_4H[(m + 1) % 4], P / 4.0))):
            pts = (cells[:, None, :] + _SITE[site][None, :, :]).reshape(-1, 2)
            xy = pts * np.array([ah, ah * math.sqrt(3.0)])
            z = np.full((len(xy), 1), m * P + dz)
            xs.append(np.concatenate([xy, z], 1))
            ts.append(np.full(len(xy), typ, dtype=np.int32))
            layer.append(np.full(len(xy), m, dtype=np.int32))
    x = np.concatenate(xs)
    types = np.concatenate(ts)
    layer = np.concatenate(layer)
    keep = np.ones(len(x), dtype=bool)
    if step == "strip":
        keep &= ~((layer == n_bilayers - 1) & (x[:, 0] >= 0.5 * Lx))
    elif step == "staircase":
        strip = np.minimum((4.0 * x[:, 0] / Lx).astype(int), 3)
        keep &= layer < (n_bilayers - strip)
    elif step is not None:
        raise ValueError(f"unknown step pattern {step!r}")
    x, types, layer = x[keep], types[keep], layer[keep]
    x[:, 2] += 1.0
    frozen = layer < n_frozen_bilayers
    thick = (n_bilayers - 1) * P + P / 4.0
    box = np.array([Lx, Ly, thick + 2.0 + vacuum])
    s = Structure(f"4H-SiC(0001) {nx}x{ny}x{n_bilayers} step={step}", x, types,
                  box, np.array([True, True, False]), frozen)
    s.meta["bilayer"] = layer
    s.meta["atoms_per_bilayer"] = 4 * nx * ny
    return s


def add_adatoms(s: Structure, count: int, zmin: float = 1.5, zmax: float = 3.0,
                min_sep: float = 1.2, typ: int = C, seed: int = 3,
                lateral_radius: float = 3.0) -> Structure:
    """Place `count` adatoms uniformly in-plane, zmin..zmax above the highest
    atom within `lateral_radius` (periodic in x/y), rejecting any closer than
    min_sep to an existing atom or to an earlier adatom."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    Lx, Ly = s.box[0], s.box[1]
    xy_tree = cKDTree(np.mod(s.x[:, :2], [Lx, Ly]), boxsize=[Lx, Ly])
    zshift = -s.x[:, 2].min() + 10.0
    big = 1.0e6
    pts = np.mod(s.x, [Lx, Ly, big]) + [0, 0, zshift]
    tree3 = cKDTree(pts, boxsize=[Lx, Ly, big])
    new = []
    tries = 0
    while len(new) < count:
        tries += 1
        if tries > 200 * count + 1000:
            raise RuntimeError("could not place adatoms")
        p = rng.uniform([0, 0], [Lx, Ly])
        idx = xy_tree.query_ball_point(p, lateral_radius)
        if not idx:
            continue
        z = s.x[idx, 2].max() + rng.uniform(zmin, zmax)
        cand = np.array([p[0], p[1], z])
        q = np.mod(cand, [Lx, Ly, big]) + [0, 0, zshift]
        if tree3.query_ball_point(q, min_sep):
            continue
        if new:
            d = np.array(new) - cand
            d[:, :2] -= np.round(d[:, :2] / [Lx, Ly]) * [Lx, Ly]
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep ** 2:
                continue
        new.append(cand)
    x = np.concatenate([s.x, np.array(new).reshape(-1, 3)])
    types = np.concatenate([s.types, np.full(count, typ, dtype=np.int32)])
    frozen = np.concatenate([s.frozen, np.zeros(count, dtype=bool)])
    box = s.box.copy()
    box[2] = max(box[2], x[:, 2].max() + 10.0)
    out = Structure(s.name + f" +{count} adatoms", x, types, box, s.pbc.copy(), frozen)
    out.meta = dict(s.meta)
    if "bilayer" in out.meta:
        out.meta["bilayer"] = np.concatenate([s.meta["bilayer"], np.full(count, -1)])
    return out


# --------------------------------------------------------------------------
# Fitting-set / annealing-ensemble shapes (Sec. 2: SiC crystals with
# defects, amorphous carbon, graphene on SiC)
# --------------------------------------------------------------------------
def _slab_dims(n_target: int, n_bilayers: int):
    """In-plane cells (nx, ny) of a 4H slab closest to n_target atoms."""
    per_cell = 4 * n_bilayers
    cells = max(1, round(n_target / per_cell))
    ny = max(1, int(round(math.sqrt(cells / math.sqrt(3.0)))))
    nx = max(1, int(round(cells / ny)))
    return nx, ny


def slab_with_vacancies(n_target: int, vac_frac: float, seed: int, n_bilayers: int = 4) -> Structure:
    """4H-SiC(0001) slab of about n_target atoms (periodic in x/y, bottom
    bilayer frozen) with a fraction vac_frac of its Si atoms removed at
    random."""
    rng = np.random.default_rng(seed)
    nx, ny = _slab_dims(n_target / max(1e-9, 1.0 - 0.5 * vac_frac), n_bilayers)
    s = sic_4h_slab(nx, ny, n_bilayers, n_frozen_bilayers=1)
    si = np.nonzero(s.types == SI)[0]
    drop = rng.choice(si, int(round(vac_frac * len(si))), replace=False)
    keep = np.ones(s.n, dtype=bool)
    keep[drop] = False
    out = Structure(f"4H-SiC slab {nx}x{ny}x{n_bilayers}, {vac_frac:.0%} Si vacancies", s.x[keep],
                    s.types[keep], s.box, s.pbc, s.frozen[keep])
    return out


def _pack_sphere(n: int, n_rho: float, rng, min_sep: float) -> np.ndarray:
    """n points by random sequential addition in the sphere (centred at 0)
    that holds them at number density n_rho (per A^3), no two closer than
    min_sep."""
    R = (3.0 * n / (4.0 * math.pi * n_rho)) ** (1.0 / 3.0)
    cell = min_sep
    grid: dict = {}
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 2000 * n:
            raise RuntimeError("could not pack the cluster")
        p = rng.uniform(-R, R, 3)
        if p @ p > R * R:
            continue
        k = tuple(np.floor(p / cell).astype(int))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for q in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        d = p - q
                        if d @ d < min_sep * min_sep:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        grid.setdefault(k, []).append(p)
        pts.append(p)
    return np.array(pts), R


def amorphous_carbon_cluster(n: int, density_gcc: float, seed: int, min_sep: float = 1.2) -> Structure:
    """n C atoms placed by random sequential addition in a sphere holding
    them at density_gcc (g/cm^3), no two closer than min_sep; open box."""
    rng = np.random.default_rng(seed)
    n_rho = density_gcc * 0.602214076 / MASS[C]          # atoms per A^3
    pts, R = _pack_sphere(n, n_rho, rng, min_sep)
    edge = 2.0 * R + 30.0
    x = pts + edge / 2.0
    return Structure(f"amorphous C cluster n={n} rho={density_gcc:.2f}", x, np.full(n, C, dtype=np.int32),
                     np.full(3, edge), np.array([False] * 3))


def random_sic_cluster(n: int, n_rho: float, seed: int, min_sep: float = 1.2) -> Structure:
    """n atoms of random type (Si or C with equal odds) packed like
    amorphous_carbon_cluster at number density n_rho (per A^3), no two
    closer than min_sep; open box."""
    rng = np.random.default_rng(seed)
    pts, R = _pack_sphere(n, n_rho, rng, min_sep)
    types = rng.integers(0, 2, n).astype(np.int32)
    edge = 2.0 * R + 30.0
    return Structure(f"random Si/C cluster n={n}", pts + edge / 2.0, types, np.full(3, edge),
                     np.array([False] * 3))


def graphene_flake(n: int, seed: int, vac_frac: float = 0.03, n_stone_wales: int = 2) -> np.ndarray:
    """Positions (z = 0) of a roughly circular graphene flake (C-C 1.42 A)
    of about n atoms, with a fraction vac_frac of its atoms removed and
    n_stone_wales Stone-Wales defects (a C-C bond rotated by 90 degrees about
    its midpoint, turning four hexagons into two pentagons and two
    heptagons)."""
    rng = np.random.default_rng(seed)
    b = 1.42
    a = b * math.sqrt(3.0)
    R = math.sqrt(n / (math.pi * 4.0 / (math.sqrt(3.0) * a * a)))
    m = int(R / a) + 3
    pts = []
    for i in range(-2 * m, 2 * m + 1):
        for j in range(-2 * m, 2 * m + 1):
            o = np.array([i * a + j * a / 2.0, j * a * math.sqrt(3.0) / 2.0])
            pts.append(o)
            pts.append(o + np.array([a / 2.0, a / (2.0 * math.sqrt(3.0))]))
    xy = np.array(pts)
    xy = xy[np.einsum("ij,ij->i", xy, xy) <= R * R]
    # Stone-Wales: rotate interior bonds by 90 degrees
    from scipy.spatial import cKDTree
    for _ in range(n_stone_wales):
        tree = cKDTree(xy)
        inner = np.nonzero(np.einsum("ij,ij->i", xy, xy) < (0.6 * R) ** 2)[0]
        if len(inner) == 0:
            break
        i = rng.choice(inner)
        nb = [j for j in tree.query_ball_point(xy[i], 1.05 * b) if j != i]
        if not nb:
            continue
        j = rng.choice(nb)
        mid = 0.5 * (xy[i] + xy[j])
        old = xy[[i, j]].copy()
        for k in (i, j):
            d = xy[k] - mid
            xy[k] = mid + np.array([-d[1], d[0]])
        # keep the rotation only if the moved pair stays clear of every other atom
        others = np.ones(len(xy), dtype=bool)
        others[[i, j]] = False
        dmin = min(np.min(np.linalg.norm(xy[others] - xy[k], axis=1)) for k in (i, j))
        if dmin < 1.2:
            xy[[i, j]] = old
    keep = rng.random(len(xy)) >= vac_frac
    return xy[keep]


def graphene_sheet(n_target: int, seed: int, n_stone_wales: int = 1, disp: float = 0.05) -> Structure:
    """Periodic graphene (C-C 1.42 A) in the x/y plane, open in z, of about
    n_target atoms: rectangular cells sqrt(3) b x 3 b with four atoms each,
    about as many cells along y as x / sqrt(3), so the sheet is roughly
    square. n_stone_wales bonds are rotated by 90 degrees about their
    midpoints (each turns four hexagons into two pentagons and two
    heptagons); a rotation that would bring the pair within 1.2 A of another
    atom or periodic image is undone. Every coordinate is then displaced by
    U(-disp, +disp)."""
    rng = np.random.default_rng(seed)
    b = 1.42
    ax, ay = math.sqrt(3.0) * b, 3.0 * b
    cells = max(1, round(n_target / 4))
    ny = max(2, int(round(math.sqrt(cells / math.sqrt(3.0)))))
    nx = max(2, int(round(cells / ny)))
    basis = np.array([[0.0, 0.0], [ax / 2, b / 2], [ax / 2, 1.5 * b], [0.0, 2.0 * b]])
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    org = np.stack([ii.ravel() * ax, jj.ravel() * ay], 1)
    xy = (org[:, None, :] + basis[None, :, :]).reshape(-1, 2)
    L = np.array([nx * ax, ny * ay])

    def mic(d):
        return d - np.round(d / L) * L

    for _ in range(n_stone_wales):
        i = int(rng.integers(len(xy)))
        d = mic(xy - xy[i])
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        nb = np.nonzero((r > 0.1) & (r < 1.05 * b))[0]
        j = int(rng.choice(nb))
        mid = xy[i] + 0.5 * mic(xy[j] - xy[i])
        old = xy[[i, j]].copy()
        for k in (i, j):
            dk = mic(xy[k] - mid)
            xy[k] = np.mod(mid + np.array([-dk[1], dk[0]]), L)
        others = np.ones(len(xy), dtype=bool)
        others[[i, j]] = False
        dmin = min(np.min(np.linalg.norm(mic(xy[others] - xy[k]), axis=1)) for k in (i, j))
        if dmin < 1.2:
            xy[[i, j]] = old
    n = len(xy)
    x = np.concatenate([xy, np.full((n, 1), 15.0)], 1) + rng.uniform(-disp, disp, size=(n, 3))
    box = np.array([L[0], L[1], 30.0])
    x[:, :2] = np.mod(x[:, :2], L)
    return Structure(f"graphene {nx}x{ny}, {n_stone_wales} Stone-Wales", x, np.full(n, C, dtype=np.int32), box,
                     np.array([True, True, False]))


def graphene_on_sic(n_target: int, seed: int) -> Structure:
    """A defected graphene flake (about 20% of the atoms) 2.5-3.0 A above a
    3-bilayer 4H-SiC(0001) slab whose periodic cell is at least the flake's
    diameter + 6 A wide, so the flake never meets its periodic images."""
    rng = np.random.default_rng(seed)
    flake = graphene_flake(max(20, int(0.2 * n_target)), seed + 1)
    diam = 2.0 * np.sqrt(np.einsum("ij,ij->i", flake, flake).max()) + 6.0
    ah = 4.36 / math.sqrt(2.0)
    nx, ny = int(math.ceil(diam / ah)), int(math.ceil(diam / (ah * math.sqrt(3.0))))
    slab = sic_4h_slab(nx, ny, 3, n_frozen_bilayers=1)
    h = rng.uniform(2.5, 3.0)
    c = slab.box[:2] / 2.0
    z = slab.x[:, 2].max() + h
    fx = np.concatenate([flake + c, np.full((len(flake), 1), z)], 1)
    x = np.concatenate([slab.x, fx])
    types = np.concatenate([slab.types, np.full(len(fx), C, dtype=np.int32)])
    frozen = np.concatenate([slab.frozen, np.zeros(len(fx), dtype=bool)])
    box = slab.box.copy()
    box[2] = x[:, 2].max() + 15.0
    return Structure(f"graphene flake ({len(fx)}) on SiC slab ({slab.n})", x, types, box, slab.pbc.copy(), frozen)


def annealing_ensemble(n_replicas: int = 256, seed: int = 4, n_min: int = 200, n_max: int = 3000):
    """Independent replicas of uneven size (uniform n_min..n_max atoms) in
    three kinds taken in turn: SiC slabs with 0-30% Si vacancies, amorphous C
    clusters at 1.8-2.3 g/cm^3, defected graphene flakes on SiC. Returns the
    structures and a temperature (K) for each, uniform in 1500-3000."""
    rng = np.random.default_rng(seed)
    out, temps = [], []
    for r in range(n_replicas):
        n = int(rng.integers(n_min, n_max + 1))
        k = r % 3
        if k == 0:
            s = slab_with_vacancies(n, float(rng.uniform(0.0, 0.3)), seed * 1000 + r)
        elif k == 1:
            s = amorphous_carbon_cluster(n, float(rng.uniform(1.8, 2.3)), seed * 1000 + r)
        else:
            s = graphene_on_sic(n, seed * 1000 + r)
        out.append(s)
        temps.append(float(rng.uniform(1500.0, 3000.0)))
    return out, temps


def differentiation_batch(n_configs: int = 1024, seed: int = 5, n_min: int = 64, n_max: int = 512):
    """Configurations for force matching, of uneven size (uniform
    n_min..n_max atoms), in three kinds taken in turn: 3C-SiC supercells of
    n1 x n2 x n3 cubic cells (n_k in 2..4, the shape closest to the drawn
    size) under a random diagonal strain of up to +-5%; periodic graphene
    with 1-3 Stone-Wales defects; random Si/C clusters at 0.05-0.10 atoms
    per A^3 with no two atoms closer than 1.2 A. The 64-atom cells are
    8.72 A wide, under twice the charge cutoff, so their lists hold several
    images of the same atom."""
    rng = np.random.default_rng(seed)
    shapes = [(p, q, r) for p in (2, 3, 4) for q in (2, 3, 4) for r in (2, 3, 4)]
    out = []
    for c in range(n_configs):
        n = int(rng.integers(n_min, n_max + 1))
        sub = seed * 100000 + c
        k = c % 3
        if k == 0:
            gap = [abs(8 * p * q * r - n) for p, q, r in shapes]
            best = [sh for sh, g in zip(shapes, gap) if g == min(gap)]
            shape = best[int(rng.integers(len(best)))]
            eps = rng.uniform(-0.05, 0.05, 3)
            s = sic_3c(shape, 4.36, 0.05, sub, strain=np.diag(eps))
        elif k == 1:
            s = graphene_sheet(n, sub, n_stone_wales=int(rng.integers(1, 4)))
        else:
            s = random_sic_cluster(n, float(rng.uniform(0.05, 0.10)), sub)
        out.append(s)
    return out


def perturbed_params(params: dict, seed: int, rel: float = 0.02) -> dict:
    """A copy of a parameter set with the pair prefactors and decay rates
    (A, B, lambda1, lambda2) and the self-energy coefficients (chi, J) each
    scaled by 1 + U(-rel, +rel): the parameters a force-matching target is
    generated with when no reference forces exist."""
    rng = np.random.default_rng(seed)
    out = json.loads(json.dumps(params))
    for name in sorted(out["pair"]):
        for k in ("A", "B", "lambda1", "lambda2"):
            out["pair"][name][k] *= 1.0 + rng.uniform(-rel, rel)
    for k in ("chi", "J"):
        out["self"][k] = [v * (1.0 + rng.uniform(-rel, rel)) for v in out["self"][k]]
    out["note"] = params.get("note", "") + f" (perturbed, seed {seed}, rel {rel})"
    return out


# --------------------------------------------------------------------------
# Workloads with the shapes of the benchmark configurations
# --------------------------------------------------------------------------
def bulk_3c_512(seed: int = 1) -> Structure:
    """512-atom 3C-SiC, 4x4x4 cubic cells, a = 4.36 A, +-0.05 A displacements."""
    return sic_3c(4, 4.36, 0.05, seed)


def stepped_slab_20k() -> Structure:
    """4H-SiC(0001) slab 24x14 cells x 15 bilayers with half the top bilayer
    removed (two step edges): 19,488 atoms, bottom two bilayers frozen."""
    return sic_4h_slab(24, 14, 15, step="strip")


def stepped_slab_1m(seed: int = 3) -> Structure:
    """4H-SiC(0001) slab 96x48 cells x 56 bilayers, staircase of three
    one-bilayer steps, plus C adatoms numbering 5% of a bilayer's sites,
    1.5-3 A above the surface: 1,005,466 atoms."""
    s = sic_4h_slab(96, 48, 56, step="staircase")
    n_ad = int(round(0.05 * s.meta["atoms_per_bilayer"]))
    return add_adatoms(s, n_ad, seed=seed)


def stepped_slab_250k(seed: int = 3) -> Structure:
    """A quarter-area version of the 1M-atom slab (48x24 cells x 56 bilayers,
    same staircase and adatom density): about 251k atoms."""
    s = sic_4h_slab(48, 24, 56, step="staircase")
    n_ad = int(round(0.05 * s.meta["atoms_per_bilayer"]))
    return add_adatoms(s, n_ad, seed=seed)


def stepped_slab_small(nx: int = 12, ny: int = 6, n_bilayers: int = 8,
                       seed: int = 3) -> Structure:
    """A small stand-in with the same shape as the 1M-atom slab (staircase +
    5% C adatoms), used where a full-size evaluation is too costly."""
    s = sic_4h_slab(nx, ny, n_bilayers, step="staircase")
    n_ad = max(1, int(round(0.05 * s.meta["atoms_per_bilayer"])))
    return add_adatoms(s, n_ad, seed=seed)


# --------------------------------------------------------------------------
# Velocities
# --------------------------------------------------------------------------
def maxwell_boltzmann(types: np.ndarray, T: float, seed: int,
                      frozen: np.ndarray | None = None) -> np.ndarray:
    """Maxwell-Boltzmann velocities (A/fs) at exactly temperature T.

    Each mobile component ~ N(0, kT/m). Frozen atoms get v = 0. The centre-of-
    mass velocity is removed only when no atom is frozen. The draw is then
    rescaled so that 2 KE / (dof k_B) = T with dof = 3 N_mobile (- 3 if the
    centre-of-mass motion was removed).
    """
    types = np.asarray(types)
    n = len(types)
    frozen = np.zeros(n, bool) if frozen is None else np.asarray(frozen, bool)
    m = MASS[types]
    rng = np.random.default_rng(seed)
    sd = np.sqrt(KB_EV * T / m * EV_PER_U_TO_A2_FS2)
    v = rng.standard_normal((n, 3)) * sd[:, None]
    v[frozen] = 0.0
    mob = ~frozen
    dof = 3 * int(mob.sum())
    if not frozen.any() and n > 1:
        vcm = (m[:, None] * v).sum(0) / m.sum()
        v -= vcm
        dof -= 3
    if T > 0 and dof > 0:
        ke = 0.5 * np.sum(m[:, None] * v * v) / EV_PER_U_TO_A2_FS2
        t_now = 2.0 * ke / (dof * KB_EV)
        v *= math.sqrt(T / t_now)
    return v
