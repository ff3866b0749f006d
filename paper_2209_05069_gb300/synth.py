"""Seeded synthetic inputs: pocket grids and ligand databases.

This module builds inputs only.  It holds none of the docking method's arithmetic (no scoring,
no pose moves, no clash test, no moving-set computation), so the FP64 oracle and the CUDA
library can both be fed from it without sharing any of the method's code.

The paper docks MEDIATE ligand libraries against real protein pockets (Section 5); neither is
available, so the shapes of those workloads are reproduced synthetically:

* Pocket (the read-only 3-D grid of Section 4.1, "texture" indexed by atom coordinates): a G^3
  voxel field, x fastest, voxel (i, j, k) at origin + h*(i, j, k) with origin = -h(G-1)/2 on every
  axis (pocket centre at the coordinate origin).  Value 1 - (r/R)^2 + U(0, noise) for r < R, 0
  outside, so the field is 0 on the grid boundary when R < h(G-1)/2.
* Ligand (atoms + bonds, Section 1 and Section 4): a random tree of maximum degree 4 with 1.5 A
  bonds placed by the natural-extension reference frame construction (NeRF) at tetrahedral bond
  angles: the first child of an atom takes a uniform random dihedral, later children sit 120 and
  240 degrees from it.  A placement that lands closer than 2.0 A to an atom more than two bonds
  away is retried with another parent (up to 20 draws).  Rotatable bonds (bonds whose removal splits the ligand in two, Section 1) are sampled
  without replacement among tree edges with at least two atoms on each side, and are oriented
  (a, b) so that the side containing b is the smaller one (ties: the side without atom 0).
"""
from __future__ import annotations

import dataclasses
import math
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from typing import Dict, List, Optional

import numpy as np

BASE_SEED = 20905069

BOND_LENGTH = 1.5
BOND_ANGLE_DEG = 109.5
PLACEMENT_CLEARANCE = 2.0
PLACEMENT_RETRIES = 20
MAX_DEGREE = 4


@dataclasses.dataclass
class Pocket:
    """A pocket grid: ``values[k, j, i]`` (x fastest in memory) at ``origin + spacing*(i, j, k)``."""

    values: np.ndarray          # float32, shape (nz, ny, nx), C-contiguous
    spacing: float
    origin: np.ndarray          # float64 (3,)

    @property
    def dims(self):
        nz, ny, nx = self.values.shape
        return nx, ny, nz

    def integer(self, scale: float = 1000.0) -> "Pocket":
        """The integer-valued pocket of an integer grid: every value times ``scale``, rounded to
        the nearest integer (float32 holding integers; scale 1000 keeps them within int16)."""
        return Pocket(np.ascontiguousarray(np.rint(self.values.astype(np.float64) * scale).astype(np.float32)),
                      self.spacing, self.origin)


@dataclasses.dataclass
class LigandDB:
    """Ligands in CSR form; atom, bond and rotatable-bond indices are local to each ligand."""

    atom_off: np.ndarray        # int32 (n_lig+1,)
    xyz: np.ndarray             # float32 (n_atoms_total, 3)
    bond_off: np.ndarray        # int32 (n_lig+1,)
    bonds: np.ndarray           # int32 (n_bonds_total, 2)
    rot_off: np.ndarray         # int32 (n_lig+1,)
    rot: np.ndarray             # int32 (n_rot_total, 2), oriented (a, b): b's side moves
    ids: np.ndarray             # uint64 (n_lig,)
    clipped: int = 0            # ligands whose rotatable-bond draw exceeded the eligible edges

    @property
    def n_lig(self) -> int:
        return int(self.atom_off.shape[0] - 1)

    def n_atoms(self, l: int) -> int:
        return int(self.atom_off[l + 1] - self.atom_off[l])

    def n_rot(self, l: int) -> int:
        return int(self.rot_off[l + 1] - self.rot_off[l])

    def ligand(self, l: int):
        """(xyz (n,3) float32, bonds (nb,2) int32, rot (B,2) int32, id) of ligand l."""
        a0, a1 = self.atom_off[l], self.atom_off[l + 1]
        b0, b1 = self.bond_off[l], self.bond_off[l + 1]
        r0, r1 = self.rot_off[l], self.rot_off[l + 1]
        return self.xyz[a0:a1], self.bonds[b0:b1], self.rot[r0:r1], int(self.ids[l])

    def subset(self, idx) -> "LigandDB":
        return from_ligands([self.ligand(int(l)) for l in idx])

    def slice(self, l0: int, l1: int, ids=None) -> "LigandDB":
        """Ligands [l0, l1) as a new database (array slices, no per-ligand copies); optional new ids."""
        a0, a1 = int(self.atom_off[l0]), int(self.atom_off[l1])
        b0, b1 = int(self.bond_off[l0]), int(self.bond_off[l1])
        r0, r1 = int(self.rot_off[l0]), int(self.rot_off[l1])
        return LigandDB(atom_off=self.atom_off[l0:l1 + 1] - a0, xyz=self.xyz[a0:a1],
                        bond_off=self.bond_off[l0:l1 + 1] - b0, bonds=self.bonds[b0:b1],
                        rot_off=self.rot_off[l0:l1 + 1] - r0, rot=self.rot[r0:r1],
                        ids=self.ids[l0:l1] if ids is None else np.asarray(ids, np.uint64))


def from_ligands(ligs) -> LigandDB:
    """Packs a list of (xyz, bonds, rot, id) tuples into a LigandDB."""
    atom_off, bond_off, rot_off = [0], [0], [0]
    xyz, bonds, rot, ids = [], [], [], []
    for (x, b, r, i) in ligs:
        x = np.asarray(x, np.float32).reshape(-1, 3)
        b = np.asarray(b, np.int32).reshape(-1, 2)
        r = np.asarray(r, np.int32).reshape(-1, 2)
        xyz.append(x); bonds.append(b); rot.append(r); ids.append(i)
        atom_off.append(atom_off[-1] + x.shape[0])
        bond_off.append(bond_off[-1] + b.shape[0])
        rot_off.append(rot_off[-1] + r.shape[0])
    return LigandDB(
        atom_off=np.asarray(atom_off, np.int32),
        xyz=np.ascontiguousarray(np.concatenate(xyz) if xyz else np.zeros((0, 3), np.float32), np.float32),
        bond_off=np.asarray(bond_off, np.int32),
        bonds=np.ascontiguousarray(np.concatenate(bonds) if bonds else np.zeros((0, 2), np.int32), np.int32),
        rot_off=np.asarray(rot_off, np.int32),
        rot=np.ascontiguousarray(np.concatenate(rot) if rot else np.zeros((0, 2), np.int32), np.int32),
        ids=np.asarray(ids, np.uint64),
    )


# ----------------------------------------------------------------------------------------------
# Pocket grids
# ----------------------------------------------------------------------------------------------

def make_pocket(G: int, spacing: float, radius: float, noise: float, seed: int) -> Pocket:
    """Sphere pocket 1-(r/R)^2 (+U(0,noise) inside), 0 outside, on a G^3 grid centred at 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    origin = np.full(3, -spacing * (G - 1) / 2.0)
    ax = origin[0] + spacing * np.arange(G)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    inside = r < radius
    v = np.where(inside, 1.0 - (r / radius) ** 2, 0.0)
    if noise > 0:
        v = v + np.where(inside, rng.random(v.shape) * noise, 0.0)
    return Pocket(values=np.ascontiguousarray(v.astype(np.float32)), spacing=float(spacing), origin=origin)


def make_field_pocket(dims, spacing: float, origin, fn) -> Pocket:
    """Grid sampled from an arbitrary field fn(X, Y, Z) (used for analytic test grids)."""
    nx, ny, nz = dims
    o = np.asarray(origin, np.float64)
    X = o[0] + spacing * np.arange(nx)
    Y = o[1] + spacing * np.arange(ny)
    Z = o[2] + spacing * np.arange(nz)
    zz, yy, xx = np.meshgrid(Z, Y, X, indexing="ij")
    v = np.broadcast_to(fn(xx, yy, zz), zz.shape)
    return Pocket(values=np.ascontiguousarray(np.asarray(v, np.float32)), spacing=float(spacing), origin=o)


# ----------------------------------------------------------------------------------------------
# Ligands
# ----------------------------------------------------------------------------------------------

def _unit(v):
    n = math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    return (v[0] / n, v[1] / n, v[2] / n)


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _nerf(A, B, C, bond, angle, dihedral):
    """Position D with |CD| = bond, angle BCD = angle, dihedral ABCD = dihedral."""
    bc = _unit((C[0] - B[0], C[1] - B[1], C[2] - B[2]))
    ab = (B[0] - A[0], B[1] - A[1], B[2] - A[2])
    n = _cross(ab, bc)
    nn = math.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
    if nn < 1e-8:  # A, B, C collinear: any perpendicular reference
        t = (1.0, 0.0, 0.0) if abs(bc[0]) < 0.9 else (0.0, 1.0, 0.0)
        n = _cross(t, bc)
        nn = math.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
    n = (n[0] / nn, n[1] / nn, n[2] / nn)
    m = _cross(n, bc)
    d0 = -bond * math.cos(angle)
    d1 = bond * math.sin(angle) * math.cos(dihedral)
    d2 = bond * math.sin(angle) * math.sin(dihedral)
    return (C[0] + d0 * bc[0] + d1 * m[0] + d2 * n[0],
            C[1] + d0 * bc[1] + d1 * m[1] + d2 * n[1],
            C[2] + d0 * bc[2] + d1 * m[2] + d2 * n[2])


def make_ligand(rng: np.random.Generator, n: int, n_rot: int):
    """One random tree ligand; returns (xyz float32 (n,3), bonds (n-1,2), rot (B,2), clipped).

    The tree and its geometry grow together: atom i picks a random parent among placed atoms with
    a free valence, takes the next dihedral slot of that parent (the first child of an atom gets a
    random dihedral, later children sit 120 and 240 degrees from it, so every bond angle is
    tetrahedral) and keeps the position if it is at least 2.0 A from every atom more than two bonds
    away; otherwise another parent is drawn (up to 20 draws, then the last position is kept).
    """
    assert n >= 2
    theta = math.radians(BOND_ANGLE_DEG)
    parent = [-1] * n
    nbrs: List[List[int]] = [[] for _ in range(n)]
    pos = np.zeros((n, 3), np.float64)
    phi0 = [0.0] * n            # dihedral of the first child placed on each atom
    slots_used: List[List[int]] = [[] for _ in range(n)]
    frame = [None] * n          # (dihedral reference point, angle partner g) per parent atom

    def attach(i, p, D, slot, phi):
        parent[i] = p
        nbrs[p].append(i)
        nbrs[i].append(p)
        pos[i] = D
        if slot == 0:
            phi0[p] = phi
        slots_used[p].append(slot)

    # atom 1 on +x from atom 0 fixes the frame
    pos[1] = (BOND_LENGTH, 0.0, 0.0)
    parent[1] = 0
    nbrs[0].append(1)
    nbrs[1].append(0)
    for i in range(2, n):
        last = None
        for _ in range(PLACEMENT_RETRIES):
            open_ = [a for a in range(i) if len(nbrs[a]) < MAX_DEGREE]
            p = open_[int(rng.integers(len(open_)))]
            if frame[p] is None:
                # g: the neighbour the new bond makes 109.5 degrees with (p's parent; for atom 0
                # its first child)
                g = parent[p] if parent[p] >= 0 else min(nbrs[p])
                ref = next((c for c in nbrs[g] if c != p), -1)
                A = tuple(pos[ref]) if ref >= 0 else (pos[g][0] + 1.0, pos[g][1] + 0.7, pos[g][2] - 0.3)
                frame[p] = (A, g)
            A, g = frame[p]
            if not slots_used[p]:
                slot, phi = 0, float(rng.random()) * 2 * math.pi
            else:
                slot = next(s_ for s_ in (1, 2) if s_ not in slots_used[p])
                phi = phi0[p] + slot * 2 * math.pi / 3
            D = _nerf(A, tuple(pos[g]), tuple(pos[p]), BOND_LENGTH, theta, phi)
            last = (p, D, slot, phi)
            near = set([p] + nbrs[p])  # atoms one or two bonds away from the new atom
            far = [a for a in range(i) if a not in near]
            if far:
                d = pos[far] - np.asarray(D)
                if np.min(np.einsum("ij,ij->i", d, d)) < PLACEMENT_CLEARANCE ** 2:
                    continue
            break
        attach(i, *last)

    # subtree sizes (atom 0 is the root of the tree)
    size = [1] * n
    for i in range(n - 1, 0, -1):
        size[parent[i]] += size[i]
    eligible = [i for i in range(1, n) if size[i] >= 2 and n - size[i] >= 2]
    clipped = n_rot > len(eligible)
    k = min(n_rot, len(eligible))
    pick = rng.choice(len(eligible), size=k, replace=False) if k > 0 else []
    rot = []
    for e in pick:
        c = eligible[int(e)]
        p = parent[c]
        # b's side moves: the smaller side; the subtree of c never holds atom 0, so ties keep (p, c)
        rot.append((p, c) if size[c] <= n - size[c] else (c, p))
    bonds = [(parent[i], i) for i in range(1, n)]
    return (pos.astype(np.float32), np.asarray(bonds, np.int32).reshape(-1, 2),
            np.asarray(rot, np.int32).reshape(-1, 2), clipped)


# ----------------------------------------------------------------------------------------------
# Workload recipes
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    """One seeded workload: pocket recipe, ligand-size distribution and docking parameters."""

    name: str
    key: int                      # seeds: pocket p -> BASE+100*key+p, ligands -> BASE+100*key+50
    n_lig: int
    grid: int
    spacing: float
    radius: float
    noise: float
    restarts: int
    align_steps: int
    torsion_steps: int
    clash_dist: float
    atoms: tuple                  # ("uniform", lo, hi) | ("lognormal", median, sigma, lo, hi)
    rot: tuple                    # ("uniform", lo, hi) | ("poisson", mean, lo, hi)
    grid_dtype: str = "f32"
    n_pockets: int = 1


WORKLOADS: Dict[str, Workload] = {
    "tiny": Workload("tiny", 1, 32, 40, 0.5, 8.0, 0.1, 8, 30, 64, 2.0,
                     ("uniform", 20, 30), ("uniform", 3, 5)),
    "uneven": Workload("uneven", 2, 10_000, 64, 0.375, 8.0, 0.1, 30, 30, 256, 2.0,
                       ("lognormal", 35, 0.4, 10, 80), ("poisson", 6, 0, 20)),
    "large": Workload("large", 3, 20_000, 96, 0.375, 12.0, 0.1, 30, 30, 256, 2.0,
                      ("uniform", 80, 150), ("uniform", 20, 40)),
    "serving": Workload("serving", 4, 10_000, 64, 0.375, 8.0, 0.1, 30, 30, 256, 2.0,
                        ("lognormal", 35, 0.4, 10, 80), ("poisson", 6, 0, 20), n_pockets=4),
    "plateau": Workload("plateau", 5, 1_000_000, 128, 0.375, 12.0, 0.1, 30, 30, 256, 2.0,
                        ("lognormal", 35, 0.4, 10, 80), ("poisson", 6, 0, 20), grid_dtype="f16"),
}


def pocket_seed(w: Workload, p: int = 0) -> int:
    return BASE_SEED + 100 * w.key + p


def ligand_seed(w: Workload) -> int:
    return BASE_SEED + 100 * w.key + 50


def workload_pocket(w: Workload, p: int = 0) -> Pocket:
    return make_pocket(w.grid, w.spacing, w.radius, w.noise, pocket_seed(w, p))


def _draw_size(rng, w: Workload):
    a = w.atoms
    if a[0] == "uniform":
        n = int(rng.integers(a[1], a[2] + 1))
    else:
        n = int(np.clip(np.rint(rng.lognormal(math.log(a[1]), a[2])), a[3], a[4]))
    r = w.rot
    if r[0] == "uniform":
        b = int(rng.integers(r[1], r[2] + 1))
    else:
        b = int(np.clip(rng.poisson(r[1]), r[2], r[3]))
    return n, b


def _make_range(args):
    w, seed, first_id, l0, l1 = args
    out, clipped = [], 0
    for l in range(l0, l1):
        # one stream per ligand keeps every ligand independent of the database size and chunking
        lrng = np.random.Generator(np.random.PCG64([seed, l]))
        n, b = _draw_size(lrng, w)
        xyz, bonds, rot, c = make_ligand(lrng, n, b)
        clipped += int(c)
        out.append((xyz, bonds, rot, first_id + l))
    return out, clipped


def make_db(w: Workload, n_lig: Optional[int] = None, seed: Optional[int] = None, first_id: int = 0,
            workers: Optional[int] = None) -> LigandDB:
    """The workload's ligand database (or its first ``n_lig`` ligands: the draw is prefix-stable).

    ``workers`` > 1 generates with a pool of worker processes started with ``spawn`` (safe in a
    process that already uses the GPU; the calling script needs the usual ``__main__`` guard); the
    result does not depend on the worker count.
    """
    n_lig = w.n_lig if n_lig is None else n_lig
    seed = ligand_seed(w) if seed is None else seed
    workers = 1 if workers is None else max(1, int(workers))
    chunks = max(1, min(workers * 4, n_lig // 250 or 1))
    edges = np.linspace(0, n_lig, chunks + 1).astype(int)
    jobs = [(w, seed, first_id, int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
    if workers > 1 and len(jobs) > 1:
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_make_range, jobs))
    else:
        parts = [_make_range(j) for j in jobs]
    ligs = [x for p in parts for x in p[0]]
    db = from_ligands(ligs)
    db.clipped = sum(p[1] for p in parts)
    return db


def default_workers() -> int:
    return min(os.cpu_count() or 1, 16)


def tile_db(pool: LigandDB, n_lig: int, first_id: int = 0) -> LigandDB:
    """A database of ``n_lig`` ligands cycling through ``pool`` with fresh ids first_id, first_id+1, ...

    The ids key the restart orientations, so repeated geometries are docked as new work."""
    reps = -(-n_lig // pool.n_lig)
    L = pool.n_lig
    na, nb, nr = int(pool.atom_off[-1]), int(pool.bond_off[-1]), int(pool.rot_off[-1])

    def offs(o, total):
        base = np.concatenate([o[:-1] + k * total for k in range(reps)] + [[reps * total]])
        return base[:n_lig + 1].astype(np.int64)

    atom_off, bond_off, rot_off = offs(pool.atom_off, na), offs(pool.bond_off, nb), offs(pool.rot_off, nr)
    return LigandDB(atom_off=atom_off.astype(np.int32), xyz=np.tile(pool.xyz, (reps, 1))[:atom_off[-1]],
                    bond_off=bond_off.astype(np.int32), bonds=np.tile(pool.bonds, (reps, 1))[:bond_off[-1]],
                    rot_off=rot_off.astype(np.int32), rot=np.tile(pool.rot, (reps, 1))[:rot_off[-1]],
                    ids=np.arange(first_id, first_id + n_lig, dtype=np.uint64))


def poisson_arrivals(rate_per_s: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative sums of exponential gaps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
