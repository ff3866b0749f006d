"""ctypes binding of libdock.so (the C-ABI declared in include/dock.h).

Argument marshalling only: every step of docking runs in the library's CUDA kernels.  There is no
Python or CPU fallback; if the library cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import threading
from typing import Optional

import numpy as np

from . import build as _build

DOCK_OK = 0
DOCK_PENDING = 1
DOCK_ERR_INVALID = -1
DOCK_ERR_NOMEM = -2
DOCK_ERR_BUSY = -3
DOCK_ERR_NOPOCKET = -4
DOCK_ERR_UNKNOWN_TICKET = -5
DOCK_ERR_TIMEOUT = -6
DOCK_ERR_CUDA = -7

DOCK_GRID_F32 = 0
DOCK_GRID_F16 = 1
DOCK_GRID_I16 = 2
GRID_DTYPES = {"f32": DOCK_GRID_F32, "f16": DOCK_GRID_F16, "i16": DOCK_GRID_I16}
DOCK_OUTPUT_FULL = 0
DOCK_OUTPUT_BEST = 1
DOCK_FORM_BATCHED = 0
DOCK_FORM_PER_LIGAND = 1
DOCK_FORM_LATENCY = 2

SYMBOLS = ["dock_create", "dock_destroy", "dock_last_error", "dock_load_pocket", "dock_unload_pocket",
           "dock_validate_ligands", "dock_get_stats",
           "dock_submit_ligands", "dock_poll", "dock_results", "dock_batch_create", "dock_batch_launch",
           "dock_batch_results", "dock_batch_destroy", "dock_batch_work", "dock_batch_launch_noalloc", "dock_set_launch", "dock_batch_wait",
           "dock_get_launch", "dock_gather_peak", "dock_exec_counters"]

NOALLOC_SCRATCH_BYTES = 16 << 20
DEVICE_RESULT_FIELDS = ["score", "best_restart", "xyz", "clash_count", "restart_score", "restart_clash", "align_idx",
                        "post_idx", "torsion_idx", "rejected"]


class DockConfig(C.Structure):
    _fields_ = [("device", C.c_int32), ("n_streams", C.c_int32), ("hbm_budget_bytes", C.c_uint64),
                ("max_batch_ligands", C.c_int32), ("max_queued_ligands", C.c_int32), ("serve_off", C.c_int32),
                ("stall_timeout_ms", C.c_int32), ("serve_latency_items", C.c_int32),
                ("serve_latency_form", C.c_int32), ("reserved", C.c_int32)]


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("spacing", C.c_float),
                ("origin", C.c_float * 3), ("dtype", C.c_int32)]


class Params(C.Structure):
    """dock_params: restarts, align_steps, torsion_steps, clash_dist, post_align, early_exit, seed,
    select_k and select_rmsd (Select Poses: up to select_k poses per ligand, pairwise RMSD >= select_rmsd)."""

    _fields_ = [("restarts", C.c_int32), ("align_steps", C.c_int32), ("torsion_steps", C.c_int32),
                ("clash_dist", C.c_float), ("post_align", C.c_int32), ("early_exit", C.c_int32),
                ("seed", C.c_uint64), ("select_k", C.c_int32), ("select_rmsd", C.c_float), ("outputs", C.c_int32)]

    @classmethod
    def make(cls, restarts=30, align_steps=30, torsion_steps=256, clash_dist=2.0, post_align=1, early_exit=1,
             seed=0, select_k=1, select_rmsd=2.0, outputs=DOCK_OUTPUT_FULL):
        return cls(restarts, align_steps, torsion_steps, clash_dist, post_align, early_exit, seed, select_k,
                   select_rmsd, outputs)

    @property
    def k(self) -> int:
        """Poses Select Poses keeps per ligand."""
        return max(1, self.select_k)


_P = C.POINTER


class LigandBatch(C.Structure):
    _fields_ = [("n_lig", C.c_int32), ("atom_off", _P(C.c_int32)), ("xyz", _P(C.c_float)),
                ("bond_off", _P(C.c_int32)), ("bonds", _P(C.c_int32)), ("rot_off", _P(C.c_int32)),
                ("rot_bonds", _P(C.c_int32)), ("ids", _P(C.c_uint64))]


class ResultBuffers(C.Structure):
    _fields_ = [("score", _P(C.c_float)), ("best_restart", _P(C.c_int32)), ("xyz", _P(C.c_float)),
                ("clash_count", _P(C.c_int32)), ("restart_score", _P(C.c_float)), ("restart_clash", _P(C.c_int32)),
                ("align_idx", _P(C.c_int32)), ("post_idx", _P(C.c_int32)), ("torsion_idx", _P(C.c_int32)),
                ("rejected", _P(C.c_int32)), ("latency_ns", _P(C.c_int64)), ("select_restart", _P(C.c_int32)),
                ("select_score", _P(C.c_float)), ("select_xyz", _P(C.c_float))]


class DeviceResults(C.Structure):
    """dock_device_results: caller-owned device buffers (raw device addresses)."""

    _fields_ = [(name, C.c_void_p) for name in DEVICE_RESULT_FIELDS]


class LaunchShape(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("smem_carveout_pct", C.c_int32), ("persistent", C.c_int32),
                ("warps_per_item", C.c_int32), ("pose_tile", C.c_int32)]


class Status(C.Structure):
    _fields_ = [("pending", C.c_int32), ("n_done", C.c_int32), ("n_total", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("ligands_submitted", C.c_uint64), ("ligands_done", C.c_uint64), ("batches", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("graph_launches", C.c_uint64), ("prep_ns", C.c_uint64), ("fill_ns", C.c_uint64),
                ("scatter_ns", C.c_uint64), ("latency_batches", C.c_uint64),
                ("slot_grows", C.c_uint64), ("slot_grow_ns", C.c_uint64), ("latency_form_batches", C.c_uint64)]


class Work(C.Structure):
    _fields_ = [("items", C.c_uint64), ("lookups_align", C.c_uint64), ("lookups_torsion", C.c_uint64),
                ("lookups_final", C.c_uint64)]


class ExecWork(C.Structure):
    """dock_exec_work: work the kernels executed (counter build only)."""

    _fields_ = [(k, C.c_uint64) for k in ("items", "align_poses", "torsion_angles", "angles_accepted", "lookups",
                                          "loads", "sectors", "pair_tests", "lines")]


class DockError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dock error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_libs = {}


def lib_path(counters: bool = False) -> str:
    return _build.LIB_COUNT if counters else _build.LIB


def lib(counters: bool = False):
    """Loads libdock.so (``counters``: libdock_count.so, the counter build), building it first if it
    is missing or stale."""
    with _lock:
        if counters not in _libs:
            path = _build.build(counters=counters)
            L = C.CDLL(path)
            vp = C.c_void_p
            L.dock_create.argtypes = [_P(DockConfig), _P(vp)]
            L.dock_destroy.argtypes = [vp]
            L.dock_last_error.argtypes = [vp]
            L.dock_last_error.restype = C.c_char_p
            L.dock_load_pocket.argtypes = [vp, _P(GridDesc), _P(C.c_float), _P(C.c_int32)]
            L.dock_unload_pocket.argtypes = [vp, C.c_int32]
            L.dock_submit_ligands.argtypes = [vp, C.c_int32, _P(LigandBatch), _P(Params), _P(C.c_uint64)]
            L.dock_poll.argtypes = [vp, C.c_uint64, C.c_int32, _P(Status)]
            L.dock_results.argtypes = [vp, C.c_uint64, _P(ResultBuffers)]
            L.dock_batch_create.argtypes = [vp, _P(LigandBatch), _P(Params), _P(vp)]
            L.dock_batch_launch.argtypes = [vp, C.c_int32, vp, C.c_int32, vp]
            L.dock_batch_results.argtypes = [vp, vp, _P(ResultBuffers)]
            L.dock_batch_destroy.argtypes = [vp, vp]
            L.dock_get_stats.argtypes = [vp, _P(Stats)]
            L.dock_batch_work.argtypes = [vp, _P(Work)]
            L.dock_batch_wait.argtypes = [vp, vp]
            L.dock_set_launch.argtypes = [vp, C.c_int32, _P(LaunchShape)]
            L.dock_get_launch.argtypes = [vp, C.c_int32, _P(LaunchShape)]
            L.dock_batch_launch_noalloc.argtypes = [vp, C.c_int32, vp, _P(DeviceResults), vp]
            L.dock_gather_peak.argtypes = [vp, C.c_int32, _P(C.c_double)]
            L.dock_validate_ligands.argtypes = [_P(LigandBatch), _P(Params), C.c_char_p, C.c_size_t]
            L.dock_exec_counters.argtypes = [vp, _P(ExecWork), C.c_int32]
            for s in SYMBOLS:
                if s != "dock_last_error":
                    getattr(L, s).restype = C.c_int
            _libs[counters] = L
    return _libs[counters]


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct)) if a is not None else None


class _Ligands:
    """Keeps contiguous copies of a LigandDB's arrays alive and exposes them as dock_ligand_batch."""

    def __init__(self, db):
        self.atom_off = np.ascontiguousarray(db.atom_off, np.int32)
        self.xyz = np.ascontiguousarray(db.xyz, np.float32).reshape(-1)
        self.bond_off = np.ascontiguousarray(db.bond_off, np.int32)
        self.bonds = np.ascontiguousarray(db.bonds, np.int32).reshape(-1)
        self.rot_off = np.ascontiguousarray(db.rot_off, np.int32)
        self.rot = np.ascontiguousarray(db.rot, np.int32).reshape(-1)
        self.ids = np.ascontiguousarray(db.ids, np.uint64)
        self.n_lig = int(self.atom_off.shape[0] - 1)
        self.c = LigandBatch(self.n_lig, _ptr(self.atom_off, C.c_int32), _ptr(self.xyz, C.c_float),
                             _ptr(self.bond_off, C.c_int32), _ptr(self.bonds, C.c_int32),
                             _ptr(self.rot_off, C.c_int32), _ptr(self.rot, C.c_int32), _ptr(self.ids, C.c_uint64))


def validate(db, params: Params):
    """Host-only validation of ligands and params (dock_validate_ligands); returns '' or the error."""
    lig = _Ligands(db)
    buf = C.create_string_buffer(512)
    rc = lib().dock_validate_ligands(C.byref(lig.c), C.byref(params), buf, 512)
    return "" if rc == DOCK_OK else buf.value.decode()


class Results(dict):
    """Result arrays of one docked batch (see dock_result_buffers)."""


def _alloc_results(n_lig, n_atoms, n_rot, R, K=1, minimal=False):
    if minimal:   # the per-ligand outputs only
        r = Results(score=np.zeros(n_lig, np.float32), best_restart=np.zeros(n_lig, np.int32),
                    xyz=np.zeros((n_atoms, 3), np.float32), clash_count=np.zeros(n_lig, np.int32),
                    latency_ns=np.zeros(n_lig, np.int64), select_restart=np.zeros(n_lig * K, np.int32),
                    select_score=np.zeros(n_lig * K, np.float32), select_xyz=np.zeros((n_atoms * K, 3), np.float32))
        c = ResultBuffers(score=_ptr(r["score"], C.c_float), best_restart=_ptr(r["best_restart"], C.c_int32),
                          xyz=_ptr(r["xyz"], C.c_float), clash_count=_ptr(r["clash_count"], C.c_int32),
                          latency_ns=_ptr(r["latency_ns"], C.c_int64),
                          select_restart=_ptr(r["select_restart"], C.c_int32),
                          select_score=_ptr(r["select_score"], C.c_float), select_xyz=_ptr(r["select_xyz"], C.c_float))
        return r, c
    r = Results(
        score=np.zeros(n_lig, np.float32), best_restart=np.zeros(n_lig, np.int32),
        xyz=np.zeros((n_atoms, 3), np.float32), clash_count=np.zeros(n_lig, np.int32),
        restart_score=np.zeros(n_lig * R, np.float32), restart_clash=np.zeros(n_lig * R, np.int32),
        align_idx=np.zeros(n_lig * R, np.int32), post_idx=np.zeros(n_lig * R, np.int32),
        torsion_idx=np.zeros(n_rot * R, np.int32), rejected=np.zeros(n_rot * R, np.int32),
        latency_ns=np.zeros(n_lig, np.int64), select_restart=np.zeros(n_lig * K, np.int32),
        select_score=np.zeros(n_lig * K, np.float32), select_xyz=np.zeros((n_atoms * K, 3), np.float32))
    types = dict(score=C.c_float, best_restart=C.c_int32, xyz=C.c_float, clash_count=C.c_int32,
                 restart_score=C.c_float, restart_clash=C.c_int32, align_idx=C.c_int32, post_idx=C.c_int32,
                 torsion_idx=C.c_int32, rejected=C.c_int32, latency_ns=C.c_int64, select_restart=C.c_int32,
                 select_score=C.c_float, select_xyz=C.c_float)
    c = ResultBuffers(**{k: _ptr(r[k], t) for k, t in types.items()})
    return r, c


class Batch:
    """A device-resident prepared batch (dock_batch)."""

    def __init__(self, handle, lig: _Ligands, params: Params):
        self.handle = handle
        self.lig = lig
        self.params = params


class Context:
    """One dock_ctx on one GPU."""

    def __init__(self, device: int = 0, n_streams: int = 0, hbm_budget_bytes: int = 0, max_batch_ligands: int = 0,
                 max_queued_ligands: int = 0, serve: bool = True, stall_timeout_ms: int = 0,
                 serve_latency_items: int = 0, counters: bool = False, serve_latency_form: int = 0):
        """``counters``: the context runs on the counter build (libdock_count.so), whose kernels count
        the work they execute (:meth:`exec_counters`); meant for measurement, not for timing."""
        self._lib = lib(counters)
        cfg = DockConfig(device, n_streams, hbm_budget_bytes, max_batch_ligands, max_queued_ligands,
                         0 if serve else 1, stall_timeout_ms, serve_latency_items, serve_latency_form)
        h = C.c_void_p()
        rc = self._lib.dock_create(C.byref(cfg), C.byref(h))
        if rc != DOCK_OK:
            raise DockError(rc, "dock_create failed")
        self.h = h
        self._tickets = {}

    def _check(self, rc):
        if rc < 0:
            raise DockError(rc, self._lib.dock_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self._lib.dock_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_launch(self, bucket: int, warps_per_block: int, smem_carveout_pct: int = -1, persistent: int = 0,
                   warps_per_item: int = 1, pose_tile: int = 1):
        sh = LaunchShape(warps_per_block, smem_carveout_pct, int(persistent), warps_per_item, pose_tile)
        self._check(self._lib.dock_set_launch(self.h, bucket, C.byref(sh)))

    def gather_peak(self, pocket_id: int) -> float:
        """dock_gather_peak: the stand-alone pocket-gather rate (lookups/s) on this GPU."""
        v = C.c_double()
        self._check(self._lib.dock_gather_peak(self.h, pocket_id, C.byref(v)))
        return v.value

    def reset_launch(self, bucket: Optional[int] = None):
        """Restores the default launch shape of one bucket (all buckets if None)."""
        for b in (range(5) if bucket is None else [bucket]):
            self._check(self._lib.dock_set_launch(self.h, b, None))

    def get_launch(self, bucket: int) -> dict:
        sh = LaunchShape()
        self._check(self._lib.dock_get_launch(self.h, bucket, C.byref(sh)))
        return {k: int(getattr(sh, k)) for k, _ in LaunchShape._fields_}

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.dock_get_stats(self.h, C.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in Stats._fields_}

    def last_error(self) -> str:
        return self._lib.dock_last_error(self.h).decode()

    # pockets
    def load_pocket(self, values, spacing, origin, dtype: str = "f32") -> int:
        """dtype "f32" / "f16": trilinear grid; "i16": integer grid (integer values, nearest voxel)."""
        v = np.ascontiguousarray(values, np.float32)
        nz, ny, nx = v.shape
        g = GridDesc(nx, ny, nz, float(spacing), (C.c_float * 3)(*[float(o) for o in origin]), GRID_DTYPES[dtype])
        pid = C.c_int32()
        self._check(self._lib.dock_load_pocket(self.h, C.byref(g), _ptr(v, C.c_float), C.byref(pid)))
        return pid.value

    def load(self, pocket, dtype: str = "f32") -> int:
        return self.load_pocket(pocket.values, pocket.spacing, pocket.origin, dtype)

    def unload_pocket(self, pid: int):
        self._check(self._lib.dock_unload_pocket(self.h, pid))

    # asynchronous docking
    def submit(self, pocket_id: int, db, params: Params) -> int:
        lig = _Ligands(db)
        t = C.c_uint64()
        self._check(self._lib.dock_submit_ligands(self.h, pocket_id, C.byref(lig.c), C.byref(params), C.byref(t)))
        self._tickets[t.value] = (lig.n_lig, int(lig.atom_off[-1]), int(lig.rot_off[-1]), params.restarts, params.k,
                                  params.outputs)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        st = Status()
        rc = self._check(self._lib.dock_poll(self.h, ticket, timeout_ms, C.byref(st)))
        return rc, (st.pending, st.n_done, st.n_total)

    def results(self, ticket: int, minimal: bool = False) -> Optional[Results]:
        """Copies a finished ticket's results; ``minimal`` fetches only the per-ligand outputs (score,
        best restart, pose, clash count, latency, Select Poses), as every ticket submitted with
        ``outputs=DOCK_OUTPUT_BEST`` does."""
        n_lig, n_atoms, n_rot, R, K, outputs = self._tickets.get(ticket, (0, 0, 0, 1, 1, DOCK_OUTPUT_FULL))
        r, c = _alloc_results(n_lig, n_atoms, n_rot, R, K, minimal or outputs == DOCK_OUTPUT_BEST)
        rc = self._check(self._lib.dock_results(self.h, ticket, C.byref(c)))
        if rc == DOCK_PENDING:
            return None
        self._tickets.pop(ticket, None)
        return r

    def dock(self, pocket_id: int, db, params: Params, timeout_ms: int = -1) -> Results:
        t = self.submit(pocket_id, db, params)
        rc, _ = self.poll(t, timeout_ms)
        if rc != DOCK_OK:
            raise DockError(DOCK_ERR_TIMEOUT, "ticket not finished")
        return self.results(t)

    # device-resident batches
    def batch_create(self, db, params: Params) -> Batch:
        lig = _Ligands(db)
        h = C.c_void_p()
        self._check(self._lib.dock_batch_create(self.h, C.byref(lig.c), C.byref(params), C.byref(h)))
        return Batch(h, lig, params)

    def batch_launch(self, pocket_id: int, b: Batch, form: int = DOCK_FORM_BATCHED, stream: int = 0) -> int:
        return self._check(self._lib.dock_batch_launch(self.h, pocket_id, b.handle, form,
                                                       C.c_void_p(stream) if stream else None))

    def batch_wait(self, b: Batch):
        self._check(self._lib.dock_batch_wait(self.h, b.handle))

    def batch_results(self, b: Batch) -> Results:
        r, c = _alloc_results(b.lig.n_lig, int(b.lig.atom_off[-1]), int(b.lig.rot_off[-1]), b.params.restarts,
                              b.params.k, b.params.outputs == DOCK_OUTPUT_BEST)
        self._check(self._lib.dock_batch_results(self.h, b.handle, C.byref(c)))
        return r

    def batch_launch_noalloc(self, pocket_id: int, b: Batch, out_ptrs: dict, stream: int = 0) -> int:
        """dock_batch_launch_noalloc: results go to the caller's device buffers, given as raw device
        addresses keyed like DEVICE_RESULT_FIELDS; the library allocates nothing for the call."""
        out = DeviceResults(**{k: C.c_void_p(int(out_ptrs[k])) for k in DEVICE_RESULT_FIELDS})
        return self._check(self._lib.dock_batch_launch_noalloc(self.h, pocket_id, b.handle, C.byref(out),
                                                               C.c_void_p(stream) if stream else None))

    def batch_work(self, b: Batch) -> dict:
        w = Work()
        self._check(self._lib.dock_batch_work(b.handle, C.byref(w)))
        return {k: int(getattr(w, k)) for k, _ in Work._fields_}

    def exec_counters(self, reset: bool = False) -> dict:
        """dock_exec_counters: executed work summed over this context's launches (counter build)."""
        w = ExecWork()
        self._check(self._lib.dock_exec_counters(self.h, C.byref(w), int(reset)))
        return {k: int(getattr(w, k)) for k, _ in ExecWork._fields_}

    def batch_destroy(self, b: Batch):
        if b.handle:
            self._check(self._lib.dock_batch_destroy(self.h, b.handle))
            b.handle = None
