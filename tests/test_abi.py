"""The C-ABI library builds, loads and exports what include/dock.h declares; host validation (CPU)."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2209_05069_gb300 import dock, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dock.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const\s+char\s*\*)\s*(dock_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("dock_load_pocket", "dock_submit_ligands", "dock_poll", "dock_results"):
        assert n in names
    assert sorted(dock.SYMBOLS) == names


def test_library_exports_every_declared_symbol():
    lib = dock.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", dock.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dock_\w+)", out))
    for n in declared():
        assert n in exported, n
        assert getattr(lib, n) is not None


def _db():
    return synth.make_db(synth.WORKLOADS["tiny"], 4)


def _params(**kw):
    base = dict(restarts=8, align_steps=30, torsion_steps=64, clash_dist=2.0, post_align=1, early_exit=1, seed=1)
    base.update(kw)
    return dock.Params.make(**base)


def test_validation_accepts_generated_ligands():
    db = synth.make_db(synth.WORKLOADS["uneven"], 50)
    assert dock.validate(db, _params()) == ""


def test_validation_rejects_ring_rotatable_bond():
    ring = synth.from_ligands([(np.arange(15, dtype=np.float32).reshape(5, 3), [(0, 1), (1, 2), (2, 3), (3, 0), (3, 4)],
                                [(3, 4), (0, 1)], 7)])
    msg = dock.validate(ring, _params())
    assert "ligand 0" in msg and "rot_bonds[1]" in msg and "bridge" in msg


@pytest.mark.parametrize("mutate, expect", [
    (lambda d: d.bonds.__setitem__((0, 1), 99), "bonds[0]"),
    (lambda d: d.rot.__setitem__((0, 0), d.rot[0, 1]), "rot_bonds[0]"),
    (lambda d: d.xyz.__setitem__((3, 1), np.nan), "not finite"),
])
def test_validation_names_the_bad_field(mutate, expect):
    db = _db()
    mutate(db)
    msg = dock.validate(db, _params())
    assert expect in msg and "ligand 0" in msg


def test_validation_rejects_oversized_ligand_and_bad_params():
    big = synth.from_ligands([(np.zeros((161, 3), np.float32), [(i, i + 1) for i in range(160)], [], 0)])
    assert "atoms=161" in dock.validate(big, _params())
    db = _db()
    assert "restarts" in dock.validate(db, _params(restarts=0))
    assert "torsion_steps" in dock.validate(db, _params(torsion_steps=2000))
    assert "align_steps" in dock.validate(db, _params(align_steps=0))
    assert "clash_dist" in dock.validate(db, _params(clash_dist=float("nan")))
    assert "early_exit" in dock.validate(db, _params(early_exit=2))
    assert "select_k" in dock.validate(db, _params(select_k=17))
    assert "select_k" in dock.validate(db, _params(restarts=4, select_k=5))
    assert "select_rmsd" in dock.validate(db, _params(select_k=2, select_rmsd=float("nan")))
    assert "select_rmsd" in dock.validate(db, _params(select_k=2, select_rmsd=-1.0))
    assert dock.validate(db, _params(restarts=4, select_k=4, select_rmsd=0.0)) == ""
    assert "outputs" in dock.validate(db, _params(outputs=2))
    assert dock.validate(db, _params(outputs=dock.DOCK_OUTPUT_BEST)) == ""


def test_validation_accepts_edge_sizes():
    one = synth.from_ligands([(np.zeros((1, 3), np.float32), [], [], 0)])
    assert dock.validate(one, _params()) == ""
    empty = synth.from_ligands([])
    assert dock.validate(empty, _params()) == ""
    chain = synth.from_ligands([(np.arange(480, dtype=np.float32).reshape(160, 3), [(i, i + 1) for i in range(159)],
                                 [(i, i + 1) for i in range(1, 65)], 3)])
    assert dock.validate(chain, _params()) == ""


def test_validation_of_large_submissions_names_the_first_bad_ligand():
    """Submissions of more than 512 ligands are prepared by several host threads; the error must
    still name the first bad ligand, whichever thread found it."""
    one = synth.make_db(synth.WORKLOADS["tiny"], 1)
    db = synth.tile_db(one, 5000, first_id=1)
    assert dock.validate(db, _params()) == ""
    for bad in ([4321, 1700], [4999], [0, 2600]):
        d = synth.tile_db(one, 5000, first_id=1)
        for l in bad:
            d.xyz[d.atom_off[l] + 1, 2] = np.inf
        msg = dock.validate(d, _params())
        assert f"ligand {min(bad)}:" in msg and "not finite" in msg, (bad, msg)


def test_validation_with_out_of_range_counts_names_the_first_bad_ligand():
    """Ingest sizes its arrays from the ligand counts before the threads run; a ligand whose atom
    count is out of range gets no room and must fail before writing, wherever it sits among other
    errors."""
    one = synth.make_db(synth.WORKLOADS["tiny"], 1)
    xyz, bonds, rot, _ = one.ligand(0)
    big = (np.arange(3 * 161, dtype=np.float32).reshape(161, 3), np.zeros((0, 2), np.int32),
           np.zeros((0, 2), np.int32), 7)
    not_a_bond = (xyz, bonds, np.array([[0, 0]], np.int32), 8)
    for cases, first, what in [({2000: big, 2500: not_a_bond}, 2000, "atoms=161"),
                               ({100: big, 2900: not_a_bond}, 100, "atoms=161"),
                               ({700: not_a_bond, 1500: big}, 700, "is not a bond")]:
        ligs = [one.ligand(0)] * 3000
        for l, lig in cases.items():
            ligs[l] = lig
        msg = dock.validate(synth.from_ligands(ligs), _params())
        assert f"ligand {first}:" in msg and what in msg, (cases.keys(), msg)


def _validate_in_child(db, q):
    q.put(dock.validate(db, _params()))


@pytest.mark.filterwarnings("ignore::DeprecationWarning")   # fork of a multi-threaded process, on purpose
def test_validation_in_a_forked_child():
    """Ingest runs on a process-wide pool of host threads; a child forked after the pool started
    inherits none of its threads and must validate on its own instead of waiting for them."""
    import multiprocessing as mp
    one = synth.make_db(synth.WORKLOADS["tiny"], 1)
    db = synth.tile_db(one, 3000, first_id=1)
    assert dock.validate(db, _params()) == ""   # starts the pool in this process
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_validate_in_child, args=(db, q))
    p.start()
    p.join(60)
    if p.is_alive():
        p.kill()
        p.join()
        pytest.fail("validation in a forked child did not return")
    assert p.exitcode == 0 and q.get(timeout=10) == ""
