"""The latency form (DOCK_FORM_LATENCY, the paper's Section 4.1 design): one ligand at a time over
the whole GPU.

Its kernels score every pose with the batched kernel's own device functions and reduce the best
pose exactly, so its results must equal the batched form's bit for bit; they are also compared
with the FP64 oracle (direct and replay, tests/parity.py) on the tiny workload and on a sample of
the uneven database, and the serving loop's use of it for lone ligands is checked.
"""
import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

from . import parity
from .test_gpu_parity import _lig, assert_report, oparams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    from paper_2209_05069_gb300 import dock
    return dock


@pytest.fixture(scope="module")
def ctx(dk):
    c = dk.Context(serve=False)
    yield c
    c.close()


def run(ctx, pid, db, prm, form):
    b = ctx.batch_create(db, prm)
    n = ctx.batch_launch(pid, b, form)
    r = ctx.batch_results(b)
    ctx.batch_destroy(b)
    return r, n


def same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("grid_dtype", ["f32", "f16", "i16"])
def test_latency_form_equals_batched_form(ctx, dk, grid_dtype):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    if grid_dtype == "i16":
        pk = pk.integer(1000)
    db = synth.make_db(w)
    pid = ctx.load(pk, grid_dtype)
    for prm in [dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                               clash_dist=w.clash_dist, seed=13),
                dk.Params.make(restarts=5, align_steps=7, torsion_steps=40, seed=14, post_align=0, early_exit=0),
                dk.Params.make(restarts=8, align_steps=30, torsion_steps=64, seed=15, select_k=3, select_rmsd=1.0)]:
        ref, _ = run(ctx, pid, db, prm, dk.DOCK_FORM_BATCHED)
        got, n = run(ctx, pid, db, prm, dk.DOCK_FORM_LATENCY)
        assert n == 2 * db.n_lig + (prm.select_k > 1)
        same(ref, got)


def test_latency_form_edge_cases_equal_batched_form(ctx, dk):
    """1-atom and 2-atom ligands, every atom bucket up to 160 atoms and 64 rotatable bonds, one
    restart, one alignment angle, 1024 restarts and 128 x 128 alignment poses with 1024 angles."""
    rng = np.random.Generator(np.random.PCG64(71))
    ligs = [(np.zeros((1, 3), np.float32), np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32), 100),
            (np.array([[0, 0, 0], [1.5, 0, 0]], np.float32), [(0, 1)], np.zeros((0, 2), np.int32), 101)]
    for i, (n, b) in enumerate([(12, 3), (33, 5), (64, 10), (97, 20), (130, 30), (160, 64)]):
        xyz, bonds, rot = _lig(rng, n, b)
        ligs.append((xyz, bonds, rot, 300 + i))
    db = synth.from_ligands(ligs)
    pid = ctx.load(synth.workload_pocket(synth.WORKLOADS["tiny"]))
    for prm in [dk.Params.make(restarts=3, align_steps=7, torsion_steps=12, seed=1),
                dk.Params.make(restarts=1, align_steps=1, torsion_steps=100, seed=2, post_align=0),
                dk.Params.make(restarts=2, align_steps=5, torsion_steps=40, clash_dist=6.0, seed=4)]:
        same(run(ctx, pid, db, prm, dk.DOCK_FORM_BATCHED)[0], run(ctx, pid, db, prm, dk.DOCK_FORM_LATENCY)[0])
    small = db.slice(2, 4)
    for prm in [dk.Params.make(restarts=1024, align_steps=4, torsion_steps=64, seed=7),
                dk.Params.make(restarts=2, align_steps=128, torsion_steps=1024, seed=8)]:
        same(run(ctx, pid, small, prm, dk.DOCK_FORM_BATCHED)[0], run(ctx, pid, small, prm, dk.DOCK_FORM_LATENCY)[0])


def test_latency_form_oracle_parity(ctx, dk, oracle):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=17)
    res, _ = run(ctx, ctx.load(pk), db, prm, dk.DOCK_FORM_LATENCY)
    rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.85, min_exact=0.7, min_best=0.75, label="latency form, tiny: ")
    u = synth.WORKLOADS["uneven"]
    upk = synth.workload_pocket(u)
    udb = synth.make_db(u, 96, seed=18)
    uprm = dk.Params.make(restarts=u.restarts, align_steps=u.align_steps, torsion_steps=u.torsion_steps,
                          clash_dist=u.clash_dist, seed=2209)
    pid = ctx.load(upk)
    res, _ = run(ctx, pid, udb, uprm, dk.DOCK_FORM_LATENCY)
    same(run(ctx, pid, udb, uprm, dk.DOCK_FORM_BATCHED)[0], res)
    rep = parity.check(oracle, oracle.GridView.of(upk), udb, res, oparams(oracle, uprm))
    assert_report(rep, min_comparable=0.6, min_exact=0.45, min_best=0.6, label="latency form, uneven 96: ")


def test_serving_docks_lone_ligands_in_the_latency_form(dk):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 6, seed=19)
    prm = dk.Params.make(restarts=8, align_steps=30, torsion_steps=64, seed=3)
    with dk.Context(serve=False) as c0:
        ref, _ = run(c0, c0.load(pk), db, prm, dk.DOCK_FORM_BATCHED)
    for form_ligands, expect in [(0, True), (-1, False)]:
        with dk.Context(n_streams=1, serve_latency_form=form_ligands) as ctx:
            pid = ctx.load(pk)
            got = []
            for l in range(db.n_lig):       # one ligand per submission, each docked alone
                got.append(ctx.dock(pid, db.slice(l, l + 1), prm))
            st = ctx.stats()
        assert (st["latency_form_batches"] == db.n_lig) == expect, st
        for l, g in enumerate(got):
            a0, a1 = db.atom_off[l], db.atom_off[l + 1]
            assert g["score"][0] == ref["score"][l] and g["best_restart"][0] == ref["best_restart"][l]
            assert np.array_equal(g["xyz"], ref["xyz"][a0:a1])
            assert np.array_equal(g["restart_score"], ref["restart_score"][l * 8:(l + 1) * 8])
