"""ctypes binding of the FP64 docking oracle (``dock_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``.  The product library never imports it.

Every function follows the method of arXiv 2209.05069 Alg. 1 as restated in the header of
``dock_oracle.cpp`` (score = sum of trilinear pocket lookups, Section 4.1; rigid alignment,
Alg. 1's two rotation loops; sequential torsion sweep with bump check, its fragment loop).
Each step is pinned by the tests; the end-to-end docking of a ligand has no published worked
example and is "parity unpinned" beyond those component pins.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dock_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdock_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle (plain g++, IEEE double, no FMA contraction) and returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("spacing", C.c_double),
                ("origin", C.c_double * 3), ("values", C.POINTER(C.c_double)), ("mode", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("restarts", C.c_int32), ("align_steps", C.c_int32), ("torsion_steps", C.c_int32),
                ("post_align", C.c_int32), ("clash_dist", C.c_double), ("seed", C.c_uint64),
                ("eps_clash", C.c_double), ("eps_voxel", C.c_double)]


_OUT_FIELDS = [
    ("best_score", "f8", "1"), ("best_restart", "i4", "1"), ("restart_score", "f8", "R"),
    ("align_idx", "i4", "R"), ("post_idx", "i4", "R"), ("torsion_idx", "i4", "RB"), ("rejected", "i4", "RB"),
    ("clash", "i4", "R"), ("restart_xyz", "f8", "Rn3"),
    ("align_best", "f8", "R"), ("align_second", "f8", "R"), ("align_forced", "f8", "R"),
    ("post_best", "f8", "R"), ("post_second", "f8", "R"), ("post_forced", "f8", "R"),
    ("tors_best", "f8", "RB"), ("tors_second", "f8", "RB"), ("tors_best_robust", "f8", "RB"),
    ("tors_forced", "f8", "RB"), ("tors_forced_margin", "f8", "RB"), ("tors_max_margin", "f8", "RB"),
    ("tors_ambiguous", "i4", "RB"), ("tors_robust_valid", "i4", "RB"), ("clash_margin", "f8", "R"),
    ("align_robust", "i4", "R"), ("align_possible", "i4", "R"), ("post_robust", "i4", "R"),
    ("post_possible", "i4", "R"), ("tors_robust", "i4", "RB"), ("tors_possible", "i4", "RB"),
    ("score_lo", "f8", "R"), ("score_hi", "f8", "R"),
]


class _Out(C.Structure):
    _fields_ = [(name, C.POINTER(C.c_double if t == "f8" else C.c_int32)) for name, t, _ in _OUT_FIELDS]


def build_source(source: str, path: str) -> str:
    """Compiles oracle source text to a shared library at `path` (used by tests that plant mistakes
    in a copy of the oracle to check that the pins catch them)."""
    src = path + ".cpp"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                           "-o", path, src])
    return path


def use_library(path: Optional[str] = None):
    """Routes every call to the library at `path` (None: back to the oracle built from this folder)."""
    global _lib
    with _lock:
        _lib = _configure(C.CDLL(path)) if path else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(C.CDLL(build()))
    return _lib


def _configure(L):
    """Declares the argument and result types of the oracle's C functions."""
    P = C.POINTER
    L.oracle_dock_ligand.argtypes = [P(_Grid), C.c_int32, P(C.c_float), C.c_int32, P(C.c_int32), C.c_int32,
                                     P(C.c_int32), C.c_uint64, P(_Params), P(C.c_int32), P(C.c_int32),
                                     P(C.c_int32), P(_Out)]
    L.oracle_dock_ligand.restype = C.c_int
    L.oracle_score.argtypes = [P(_Grid), C.c_int32, P(C.c_double)]
    L.oracle_score.restype = C.c_double
    L.oracle_score_range.argtypes = [P(_Grid), C.c_int32, P(C.c_double), C.c_double, P(C.c_double), P(C.c_double)]
    L.oracle_score_range.restype = C.c_double
    L.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    L.oracle_splitmix64.restype = C.c_uint64
    L.oracle_restart_rotation.argtypes = [C.c_uint64, C.c_uint64, C.c_int32, P(C.c_double)]
    L.oracle_restart_rotation.restype = None
    L.oracle_align_pose.argtypes = [C.c_int32, P(C.c_double), C.c_int32, C.c_int32, C.c_int32, P(C.c_double)]
    L.oracle_align_pose.restype = None
    L.oracle_moving_set.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), C.c_int32, C.c_int32, P(C.c_int32)]
    L.oracle_moving_set.restype = C.c_int
    L.oracle_torsion_pose.argtypes = [C.c_int32, P(C.c_double), C.c_int32, P(C.c_int32), C.c_int32,
                                      C.c_int32, C.c_int32, C.c_int32, P(C.c_double)]
    L.oracle_torsion_pose.restype = C.c_int
    L.oracle_rejected_angles.argtypes = [C.c_int32, P(C.c_double), C.c_int32, P(C.c_int32), C.c_int32,
                                         C.c_int32, C.c_int32, C.c_double]
    L.oracle_rejected_angles.restype = C.c_int
    L.oracle_clash_count.argtypes = [C.c_int32, P(C.c_double), C.c_int32, P(C.c_int32), C.c_double]
    L.oracle_clash_count.restype = C.c_int
    L.oracle_select_poses.argtypes = [C.c_int32, C.c_int32, P(C.c_double), P(C.c_double), C.c_int32, C.c_double,
                                      P(C.c_int32), P(C.c_double), P(C.c_double)]
    L.oracle_select_poses.restype = C.c_int
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


@dataclasses.dataclass
class Params:
    """Docking parameters (names follow Alg. 1): restarts N, alignment angles per axis, torsion
    angles per rotatable bond, bump threshold d_c (A), post-optimisation alignment flag, seed."""

    restarts: int = 8
    align_steps: int = 30
    torsion_steps: int = 64
    clash_dist: float = 2.0
    post_align: int = 1
    seed: int = 0
    eps_clash: float = 1e-4
    eps_voxel: float = 1e-4   # grid units (integer grid only)


class GridView:
    """Keeps the float64 copy of a grid alive while the oracle reads it.  ``mode`` 0 interpolates
    trilinearly; mode 1 reads the nearest voxel (integer grid)."""

    def __init__(self, values, spacing, origin, mode: int = 0):
        v = np.ascontiguousarray(np.asarray(values, np.float64))
        assert v.ndim == 3
        self.values = v
        self.mode = mode
        nz, ny, nx = v.shape
        self.c = _Grid(nx, ny, nz, float(spacing), (C.c_double * 3)(*[float(o) for o in origin]),
                       _ptr(v, C.c_double), mode)

    @classmethod
    def of(cls, pocket, fp16: bool = False, nearest: bool = False):
        v = pocket.values.astype(np.float16).astype(np.float64) if fp16 else pocket.values
        return cls(v, pocket.spacing, pocket.origin, 1 if nearest else 0)


def dock_ligand(grid: GridView, xyz, bonds, rot, lig_id: int, p: Params, forced_align=None, forced_post=None,
                forced_tors=None) -> dict:
    """Docks one ligand (all restarts); returns a dict of numpy arrays (see oracle_out)."""
    xyz = np.ascontiguousarray(np.asarray(xyz, np.float32).reshape(-1, 3))
    bonds = np.ascontiguousarray(np.asarray(bonds, np.int32).reshape(-1, 2))
    rot = np.ascontiguousarray(np.asarray(rot, np.int32).reshape(-1, 2))
    n, B, R = xyz.shape[0], rot.shape[0], p.restarts
    sizes = {"1": 1, "R": R, "RB": max(R * B, 1), "Rn3": R * n * 3}
    arrs = {name: np.zeros(sizes[s], dtype=t) for name, t, s in _OUT_FIELDS}
    out = _Out(**{name: _ptr(arrs[name], C.c_double if t == "f8" else C.c_int32) for name, t, _ in _OUT_FIELDS})
    cp = _Params(p.restarts, p.align_steps, p.torsion_steps, p.post_align, p.clash_dist, p.seed, p.eps_clash,
                 p.eps_voxel)

    def opt(a, size):
        if a is None:
            return None, None
        a = np.ascontiguousarray(np.asarray(a, np.int32).reshape(-1))
        assert a.size >= size
        return a, _ptr(a, C.c_int32)

    fa, fa_p = opt(forced_align, R)
    fp, fp_p = opt(forced_post, R)
    ft, ft_p = opt(forced_tors, R * B)
    rc = lib().oracle_dock_ligand(C.byref(grid.c), n, _ptr(xyz, C.c_float), bonds.shape[0], _ptr(bonds, C.c_int32),
                                  B, _ptr(rot, C.c_int32), C.c_uint64(int(lig_id)), C.byref(cp), fa_p, fp_p, ft_p,
                                  C.byref(out))
    if rc != 0:
        raise ValueError(f"oracle_dock_ligand failed with code {rc}")
    res = {k: v for k, v in arrs.items()}
    res["best_score"] = float(arrs["best_score"][0])
    res["best_restart"] = int(arrs["best_restart"][0])
    for k in [name for name, _, s in _OUT_FIELDS if s == "RB"]:
        res[k] = arrs[k][:R * B].reshape(R, B)
    res["restart_xyz"] = arrs["restart_xyz"].reshape(R, n, 3)
    return res


def dock_db(grid: GridView, db, p: Params, threads: int = 1, forced: Optional[dict] = None, indices=None):
    """Docks ligands of a LigandDB; ``threads`` > 1 runs ligands concurrently (ctypes drops the GIL).

    ``forced`` (replay) maps 'align', 'post', 'tors' to per-ligand lists of forced decisions.
    """
    idx = list(range(db.n_lig)) if indices is None else list(indices)

    def one(l):
        xyz, bonds, rot, lid = db.ligand(l)
        kw = {}
        if forced is not None:
            kw = dict(forced_align=forced["align"][l], forced_post=forced["post"][l], forced_tors=forced["tors"][l])
        return dock_ligand(grid, xyz, bonds, rot, lid, p, **kw)

    if threads <= 1:
        return [one(l) for l in idx]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, idx))


# ---- building blocks -------------------------------------------------------------------------------

def score_range(grid: GridView, xyz, eps: float):
    """Integer-grid score of a pose and its (lo, hi) range over coordinates within eps grid units."""
    a = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    lo, hi = C.c_double(), C.c_double()
    s = lib().oracle_score_range(C.byref(grid.c), a.shape[0], _ptr(a, C.c_double), float(eps), C.byref(lo),
                                 C.byref(hi))
    return s, lo.value, hi.value


def score(grid: GridView, xyz) -> float:
    x = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    return float(lib().oracle_score(C.byref(grid.c), x.shape[0], _ptr(x, C.c_double)))


def splitmix64(state: int, k: int) -> int:
    return int(lib().oracle_splitmix64(C.c_uint64(state), C.c_uint64(k)))


def restart_rotation(lig_id: int, seed: int, r: int) -> np.ndarray:
    R = np.zeros(9, np.float64)
    lib().oracle_restart_rotation(C.c_uint64(lig_id), C.c_uint64(seed), r, _ptr(R, C.c_double))
    return R.reshape(3, 3)


def align_pose(xyz, N: int, i: int, j: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    out = np.zeros_like(x)
    lib().oracle_align_pose(x.shape[0], _ptr(x, C.c_double), N, i, j, _ptr(out, C.c_double))
    return out


def moving_set(n: int, bonds, a: int, b: int) -> np.ndarray:
    bonds = np.ascontiguousarray(np.asarray(bonds, np.int32).reshape(-1, 2))
    m = np.zeros(n, np.int32)
    rc = lib().oracle_moving_set(n, bonds.shape[0], _ptr(bonds, C.c_int32), a, b, _ptr(m, C.c_int32))
    if rc:
        raise ValueError(f"moving_set failed with code {rc}")
    return m.astype(bool)


def torsion_pose(xyz, bonds, a: int, b: int, A: int, k: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    bonds = np.ascontiguousarray(np.asarray(bonds, np.int32).reshape(-1, 2))
    out = np.zeros_like(x)
    rc = lib().oracle_torsion_pose(x.shape[0], _ptr(x, C.c_double), bonds.shape[0], _ptr(bonds, C.c_int32), a, b,
                                   A, k, _ptr(out, C.c_double))
    if rc:
        raise ValueError(f"torsion_pose failed with code {rc}")
    return out


def rejected_angles(xyz, bonds, a: int, b: int, A: int, dc: float) -> int:
    x = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    bonds = np.ascontiguousarray(np.asarray(bonds, np.int32).reshape(-1, 2))
    return int(lib().oracle_rejected_angles(x.shape[0], _ptr(x, C.c_double), bonds.shape[0],
                                            _ptr(bonds, C.c_int32), a, b, A, dc))


def clash_count(xyz, bonds, dc: float) -> int:
    x = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    bonds = np.ascontiguousarray(np.asarray(bonds, np.int32).reshape(-1, 2))
    return int(lib().oracle_clash_count(x.shape[0], _ptr(x, C.c_double), bonds.shape[0], _ptr(bonds, C.c_int32), dc))


def select_poses(score, xyz, K: int, thr: float) -> dict:
    """Select Poses over one ligand's restarts (Alg. 1, after the restart loop): ``score`` [R] final
    scores, ``xyz`` [R, n, 3] final poses.  Returns {"sel": [K] kept restarts (-1 past the end),
    "n_kept", "rmsd_margin", "score_margin"}."""
    score = np.ascontiguousarray(np.asarray(score, np.float64).reshape(-1))
    R = score.shape[0]
    xyz = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(R, -1, 3))
    sel = np.zeros(K, np.int32)
    rm, sm = C.c_double(), C.c_double()
    nk = lib().oracle_select_poses(R, xyz.shape[1], _ptr(score, C.c_double), _ptr(xyz, C.c_double), K, float(thr),
                                   _ptr(sel, C.c_int32), C.byref(rm), C.byref(sm))
    if nk < 0:
        raise ValueError(f"oracle_select_poses failed with code {nk}")
    return {"sel": sel, "n_kept": nk, "rmsd_margin": rm.value, "score_margin": sm.value}
