"""A plain C11 program compiled against include/dock.h (tests/c/dock_abi_test.c) uses the boundary.

CPU: the C compiler's sizeof / offsetof of every struct of the C-ABI equal those of the Python
binding's ctypes mirrors, field by field, so a field added on one side only cannot shift the later
ones silently.  GPU: the C program docks the tiny workload through dock_create, dock_load_pocket,
dock_submit_ligands, dock_poll and dock_results, and its results equal the Python binding's bit
for bit.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_2209_05069_gb300 import dock, synth

from .c import build_abi_test

MIRRORS = {"dock_config": dock.DockConfig, "dock_grid_desc": dock.GridDesc, "dock_params": dock.Params,
           "dock_ligand_batch": dock.LigandBatch, "dock_result_buffers": dock.ResultBuffers,
           "dock_status": dock.Status, "dock_stats": dock.Stats, "dock_launch_shape": dock.LaunchShape,
           "dock_work": dock.Work, "dock_device_results": dock.DeviceResults, "dock_exec_work": dock.ExecWork}


@pytest.fixture(scope="module")
def exe():
    return build_abi_test.build(dock.lib_path() if os.path.exists(dock.lib_path()) else dock._build.build())


def c_layout(exe):
    out = subprocess.run([exe, "layout"], capture_output=True, text=True, check=True).stdout
    sizes, fields = {}, {}
    for line in out.splitlines():
        name, off, size = line.split()
        if "." in name:
            s, f = name.split(".")
            fields.setdefault(s, {})[f] = (int(off), int(size))
        else:
            sizes[name] = int(size)
    return sizes, fields


def test_struct_layouts_match_the_binding(exe):
    sizes, fields = c_layout(exe)
    assert set(sizes) == set(MIRRORS)
    for name, cls in MIRRORS.items():
        assert sizes[name] == C.sizeof(cls), name
        py = {f: (getattr(cls, f).offset, getattr(cls, f).size) for f, _ in cls._fields_}
        assert py == fields[name], name


def write_input(path, pk, db, prm, dtype=0):
    nz, ny, nx = pk.values.shape
    with open(path, "wb") as f:
        np.array([nx, ny, nz, dtype], np.int32).tofile(f)
        np.array([pk.spacing, *pk.origin], np.float32).tofile(f)
        np.ascontiguousarray(pk.values, np.float32).tofile(f)
        np.array([prm.restarts, prm.align_steps, prm.torsion_steps, prm.post_align, prm.early_exit, prm.select_k,
                  prm.outputs], np.int32).tofile(f)
        np.array([prm.clash_dist, prm.select_rmsd], np.float32).tofile(f)
        np.array([prm.seed], np.uint64).tofile(f)
        np.array([db.n_lig], np.int32).tofile(f)
        np.asarray(db.atom_off, np.int32).tofile(f)
        np.asarray(db.xyz, np.float32).tofile(f)
        np.asarray(db.bond_off, np.int32).tofile(f)
        np.asarray(db.bonds, np.int32).tofile(f)
        np.asarray(db.rot_off, np.int32).tofile(f)
        np.asarray(db.rot, np.int32).tofile(f)
        np.asarray(db.ids, np.uint64).tofile(f)


def read_output(path, db, R):
    n, atoms, nrot = db.n_lig, int(db.atom_off[-1]), int(db.rot_off[-1])
    raw = np.fromfile(path, np.uint8)
    spec = [("score", np.float32, n), ("best_restart", np.int32, n), ("xyz", np.float32, 3 * atoms),
            ("clash_count", np.int32, n), ("restart_score", np.float32, n * R), ("restart_clash", np.int32, n * R),
            ("align_idx", np.int32, n * R), ("post_idx", np.int32, n * R), ("torsion_idx", np.int32, nrot * R),
            ("rejected", np.int32, nrot * R)]
    out, o = {}, 0
    for name, t, cnt in spec:
        out[name] = raw[o:o + 4 * cnt].view(t)
        o += 4 * cnt
    assert o == raw.size
    out["xyz"] = out["xyz"].reshape(-1, 3)
    return out


@pytest.mark.gpu
def test_c_client_docks_like_the_binding(exe, tmp_path):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w)
    prm = dock.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                           clash_dist=w.clash_dist, seed=41)
    write_input(tmp_path / "in.bin", pk, db, prm)
    subprocess.run([exe, "dock", str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], check=True, timeout=300)
    got = read_output(tmp_path / "out.bin", db, prm.restarts)
    with dock.Context() as ctx:
        ref = ctx.dock(ctx.load(pk), db, prm)
    for k, v in got.items():
        assert np.array_equal(np.asarray(ref[k]).reshape(v.shape), v), k
