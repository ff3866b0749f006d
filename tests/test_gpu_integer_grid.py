"""Integer pocket grids (DOCK_GRID_I16: nearest-voxel score, exact integer sums) on the GPU
against the oracle's integer mode.

Scores are exact integers on both sides, so comparable trajectories must match bit for bit,
scores included; decisions that an atom near a half-way plane between voxels could flip are
checked by replay (see tests/parity.py).
"""
import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

from . import parity

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


def run(ctx, pid, db, prm, form=0):
    b = ctx.batch_create(db, prm)
    assert ctx.batch_launch(pid, b, form) >= 0
    r = ctx.batch_results(b)
    ctx.batch_destroy(b)
    return r


def oparams(oracle, prm):
    return oracle.Params(restarts=prm.restarts, align_steps=prm.align_steps, torsion_steps=prm.torsion_steps,
                         clash_dist=float(np.float32(prm.clash_dist)), post_align=prm.post_align, seed=prm.seed)


def assert_report(rep, min_comparable, min_exact=0.0, min_best=0.0, label=""):
    """No failure, and coverage floors: trajectories compared bit for bit (every decision the only
    possible one), decisions whose only possible choice was compared exactly, best poses compared
    directly, each as a fraction of its total.  Prints the coverage line."""
    print(f"\n{label}{rep.summary()}")
    assert not rep.failures, "\n".join(rep.failures)
    assert rep.comparable >= min_comparable * rep.trajectories, (rep.comparable, rep.trajectories)
    assert rep.decisions_exact >= min_exact * rep.decisions, (rep.decisions_exact, rep.decisions)
    assert rep.ligands_comparable >= min_best * rep.ligands, (rep.ligands_comparable, rep.ligands)


@pytest.mark.parametrize("seed", [5, 6])
def test_tiny_workload_integer_grid_parity(ctx, dk, oracle, seed):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w).integer(1000)
    db = synth.make_db(w)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=seed)
    res = run(ctx, ctx.load(pk, "i16"), db, prm)
    assert (res["restart_score"] == np.rint(res["restart_score"])).all()
    rep = parity.check(oracle, oracle.GridView.of(pk, nearest=True), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.9, min_exact=0.9, min_best=0.75, label=f"tiny, integer grid, seed {seed}: ")


def test_constant_integer_grid(ctx, dk):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 8, seed=3)
    prm = dk.Params.make(restarts=4, align_steps=8, torsion_steps=16, clash_dist=w.clash_dist, seed=1)
    res = run(ctx, ctx.load_pocket(np.full(pk.values.shape, -7.0, np.float32), pk.spacing, pk.origin, "i16"), db,
              prm)
    n = np.diff(db.atom_off)
    assert (res["restart_score"].reshape(-1, 4) == -7.0 * n[:, None]).all()
    assert (res["align_idx"] == 0).all() and (res["post_idx"] == 0).all() and (res["torsion_idx"] == 0).all()
    assert (res["best_restart"] == 0).all()


def test_all_zero_integer_grid(ctx, dk):
    """Nothing nonzero to store: every lookup lands on the zero border, every score is 0 and every
    decision is the tie rule's lowest index."""
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 6, seed=4)
    prm = dk.Params.make(restarts=3, align_steps=6, torsion_steps=8, clash_dist=w.clash_dist, seed=2)
    res = run(ctx, ctx.load_pocket(np.zeros(pk.values.shape, np.float32), pk.spacing, pk.origin, "i16"), db, prm)
    assert (res["restart_score"] == 0).all() and (res["score"] == 0).all()
    assert (res["align_idx"] == 0).all() and (res["post_idx"] == 0).all() and (res["torsion_idx"] == 0).all()


def test_integer_grid_values_are_checked(ctx, dk):
    v = np.zeros((4, 4, 4), np.float32)
    for bad in (0.5, 32768.0, -32769.0):
        v[1, 2, 3] = bad
        with pytest.raises(dk.DockError) as e:
            ctx.load_pocket(v, 0.5, (0, 0, 0), "i16")
        assert e.value.code == dk.DOCK_ERR_INVALID and "int16" in str(e.value)
    v[1, 2, 3] = -32768.0
    v[0, 0, 0] = 32767.0
    ctx.unload_pocket(ctx.load_pocket(v, 0.5, (0, 0, 0), "i16"))


def test_integer_grid_edges_and_ligands_sticking_out(ctx, dk, oracle):
    """A small grid that is nonzero up to its faces: atoms within half a voxel outside the last
    voxel centre still read it, farther ones read 0."""
    rng = np.random.default_rng(8)
    v = rng.integers(1, 40, size=(14, 14, 14)).astype(np.float32)
    pk = synth.Pocket(v, 0.5, np.array([-3.25, -3.25, -3.25]))
    db = synth.make_db(synth.WORKLOADS["tiny"], 10)
    prm = dk.Params.make(restarts=3, align_steps=10, torsion_steps=32, seed=6)
    res = run(ctx, ctx.load(pk, "i16"), db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk, nearest=True), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.5, min_exact=0.7, label="integer grid edges: ")


def test_integer_grid_launch_shapes_are_bit_identical(ctx, dk):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w).integer(1000)
    db = synth.make_db(w, seed=12)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=12)
    pid = ctx.load(pk, "i16")
    ref = run(ctx, pid, db, prm)
    got = [run(ctx, pid, db, prm, form=dk.DOCK_FORM_PER_LIGAND)]
    try:
        for wpb, ps, g, tl in [(2, 0, 1, 1), (8, 1, 2, 1), (8, 0, 8, 1), (4, 1, 4, 1), (4, 1, 1, 2), (8, 1, 2, 2)]:
            ctx.set_launch(0, wpb, -1, ps, g, tl)
            got.append(run(ctx, pid, db, prm))
    finally:
        ctx.reset_launch(0)
    for r in got:
        for k in ref:
            assert np.array_equal(r[k], ref[k]), k


def test_uneven_database_integer_grid_full_size_sampled(ctx, dk, oracle):
    """The 10,000-ligand uneven database at full parameters on the integer grid: properties on
    every ligand, 64 sampled ligands against the oracle."""
    w = synth.WORKLOADS["uneven"]
    pk = synth.workload_pocket(w).integer(1000)
    db = synth.make_db(w, workers=synth.default_workers())
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    res = run(ctx, ctx.load(pk, "i16"), db, prm)
    R = prm.restarts
    rs = res["restart_score"].reshape(-1, R)
    assert (rs == np.rint(rs)).all()
    assert np.array_equal(res["best_restart"], np.argmax(rs, axis=1))
    assert np.array_equal(res["score"], rs[np.arange(db.n_lig), res["best_restart"]])
    sample = np.random.Generator(np.random.PCG64(19)).choice(db.n_lig, 64, replace=False)
    rep = parity.check(oracle, oracle.GridView.of(pk, nearest=True), db, res, oparams(oracle, prm), indices=sample)
    assert_report(rep, min_comparable=0.6, min_exact=0.85, min_best=0.6, label="uneven 10,000, integer grid, 64 sampled: ")


def test_large_molecules_integer_grid_sampled(ctx, dk, oracle):
    w = synth.WORKLOADS["large"]
    pk = synth.workload_pocket(w).integer(1000)
    db = synth.make_db(w, 24)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    res = run(ctx, ctx.load(pk, "i16"), db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk, nearest=True), db, res, oparams(oracle, prm),
                       indices=[0, 3, 6, 9, 12, 15, 18, 21])
    assert_report(rep, min_comparable=0.1, min_exact=0.5, label="large molecules, integer grid, 8 of 24: ")
