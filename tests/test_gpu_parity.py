"""GPU (CUDA path through the C-ABI) vs the FP64 oracle, element by element.

Every test calls libdock.so through its C-ABI and checks the results with tests/parity.py:
direct comparison on trajectories whose decisions FP32 cannot flip, and a double-precision replay
of the GPU's own decisions for every trajectory.
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


def run(ctx, dk, pid, db, prm, form=0):
    b = ctx.batch_create(db, prm)
    n = ctx.batch_launch(pid, b, form)
    assert n >= 0
    r = ctx.batch_results(b)
    ctx.batch_destroy(b)
    return r


def oparams(oracle, prm):
    return oracle.Params(restarts=prm.restarts, align_steps=prm.align_steps, torsion_steps=prm.torsion_steps,
                         clash_dist=float(np.float32(prm.clash_dist)), post_align=prm.post_align, seed=prm.seed)


def assert_report(rep, min_comparable=0.85, min_exact=0.0, min_best=0.0, label=""):
    """No failure, and coverage floors: trajectories compared directly (clear of 1e-6 ties), decisions
    clear of the benchmark spec's 1e-4 ties (compared exactly) and best poses compared directly, each
    as a fraction of its total.  Prints the coverage line (pytest -s shows it)."""
    print(f"\n{label}{rep.summary()}")
    msg = "\n".join(rep.failures)
    assert not rep.failures, msg
    assert rep.comparable >= min_comparable * rep.trajectories, (rep.comparable, rep.trajectories)
    assert rep.decisions_exact >= min_exact * rep.decisions, (rep.decisions_exact, rep.decisions)
    assert rep.ligands_comparable >= min_best * rep.ligands, (rep.ligands_comparable, rep.ligands)


def tiny_setup(dk, w=synth.WORKLOADS["tiny"], seed=5):
    pk = synth.workload_pocket(w)
    db = synth.make_db(w)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, post_align=1, early_exit=1, seed=seed)
    return pk, db, prm


def test_tiny_workload_parity(ctx, dk, oracle):
    pk, db, prm = tiny_setup(dk)
    pid = ctx.load(pk)
    res = run(ctx, dk, pid, db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.85, min_exact=0.7, min_best=0.75, label="tiny, FP32 grid: ")


def test_tiny_workload_parity_fp16_grid(ctx, dk, oracle):
    pk, db, prm = tiny_setup(dk, seed=6)
    pid = ctx.load(pk, "f16")
    res = run(ctx, dk, pid, db, prm)
    # the oracle reads the same FP16-rounded voxel values
    rep = parity.check(oracle, oracle.GridView.of(pk, fp16=True), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.85, min_exact=0.7, min_best=0.75, label="tiny, FP16 grid: ")
    # score error of the FP16 grid on the GPU's final poses, against the FP32 grid in FP64
    g32 = oracle.GridView.of(pk)
    for l in range(db.n_lig):
        a0, a1 = db.atom_off[l], db.atom_off[l + 1]
        s32 = oracle.score(g32, res["xyz"][a0:a1])
        assert abs(res["score"][l] - s32) <= 2e-3 * max(abs(s32), 1.0)


def test_no_bump_early_exit_changes_nothing(ctx, dk):
    pk, db, prm = tiny_setup(dk, seed=7)
    pid = ctx.load(pk)
    a = run(ctx, dk, pid, db, prm)
    prm.early_exit = 0
    b = run(ctx, dk, pid, db, prm)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_per_ligand_form_equals_batched_form(ctx, dk):
    pk, db, prm = tiny_setup(dk, seed=8)
    pid = ctx.load(pk)
    a = run(ctx, dk, pid, db, prm, form=dk.DOCK_FORM_BATCHED)
    b = run(ctx, dk, pid, db, prm, form=dk.DOCK_FORM_PER_LIGAND)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    try:   # the latency-oriented shape: one launch per ligand, 8 warps per ligand-restart
        ctx.set_launch(0, 8, -1, 0, 8)
        c = run(ctx, dk, pid, db, prm, form=dk.DOCK_FORM_PER_LIGAND)
        for k in a:
            assert np.array_equal(a[k], c[k]), k
    finally:
        ctx.set_launch(0, 4, -1, 0, 1)


def test_repeated_launches_are_identical(ctx, dk):
    pk, db, prm = tiny_setup(dk, seed=9)
    pid = ctx.load(pk)
    b = ctx.batch_create(db, prm)
    ctx.batch_launch(pid, b)
    r1 = ctx.batch_results(b)
    ctx.batch_launch(pid, b)
    ctx.batch_launch(pid, b)
    r2 = ctx.batch_results(b)
    ctx.batch_destroy(b)
    for k in r1:
        assert np.array_equal(r1[k], r2[k]), k


def test_constant_grid_ties_pick_lowest_indices(ctx, dk):
    c = 0.25
    pk = synth.make_field_pocket((48, 48, 48), 0.5, (-11.75,) * 3, lambda x, y, z: c + 0 * x)
    db = synth.make_db(synth.WORKLOADS["tiny"], 8)
    prm = dk.Params.make(restarts=4, align_steps=30, torsion_steps=64, seed=3)
    res = run(ctx, dk, ctx.load(pk), db, prm)
    n = np.diff(db.atom_off)
    assert np.array_equal(res["score"], (n * c).astype(np.float32))
    assert (res["best_restart"] == 0).all()
    assert (res["align_idx"] == 0).all() and (res["post_idx"] == 0).all()
    assert (res["torsion_idx"] == 0).all()


def test_affine_grid_parity(ctx, dk, oracle):
    # trilinear interpolation is exact on an affine field
    gv = np.array([0.8, -0.35, 0.5])
    pk = synth.make_field_pocket((64, 64, 64), 0.5, (-15.75,) * 3,
                                 lambda x, y, z: gv[0] * x + gv[1] * y + gv[2] * z + 3.0)
    db = synth.make_db(synth.WORKLOADS["tiny"], 12)
    prm = dk.Params.make(restarts=3, align_steps=12, torsion_steps=48, clash_dist=2.0, seed=4)
    res = run(ctx, dk, ctx.load(pk), db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm))
    # a rigid rotation about the centroid leaves an affine field's score unchanged, so every
    # alignment pose ties and no whole trajectory is tie-free; the torsion decisions are not ties
    assert_report(rep, min_comparable=0.0, min_exact=0.35, label="affine grid: ")


def _lig(rng, n, b):
    while True:
        xyz, bonds, rot, clipped = synth.make_ligand(rng, n, b)
        if not clipped:
            return xyz, bonds, rot


def test_edge_cases(ctx, dk, oracle):
    rng = np.random.Generator(np.random.PCG64(11))
    ligs = [(np.zeros((1, 3), np.float32), np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32), 100),
            (np.array([[0, 0, 0], [1.5, 0, 0]], np.float32), [(0, 1)], np.zeros((0, 2), np.int32), 101)]
    for i, (n, b) in enumerate([(4, 1), (12, 0), (33, 5), (64, 10), (65, 12), (97, 20), (130, 30), (160, 40),
                                (160, 64)]):
        xyz, bonds, rot = _lig(rng, n, b) if n < 160 or b <= 40 else _lig(rng, n, b)
        ligs.append((xyz, bonds, rot, 200 + i))
    db = synth.from_ligands(ligs)
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    pid = ctx.load(pk)
    for prm in [dk.Params.make(restarts=3, align_steps=7, torsion_steps=12, clash_dist=2.0, seed=1),
                dk.Params.make(restarts=1, align_steps=1, torsion_steps=100, clash_dist=2.0, seed=2, post_align=0),
                dk.Params.make(restarts=2, align_steps=5, torsion_steps=33, clash_dist=0.0, seed=3),
                dk.Params.make(restarts=2, align_steps=5, torsion_steps=40, clash_dist=6.0, seed=4)]:
        res = run(ctx, dk, pid, db, prm)
        rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm))
        assert_report(rep, min_comparable=0.35, min_exact=0.45, min_best=0.35,
                      label=f"edge cases R {prm.restarts} N {prm.align_steps} A {prm.torsion_steps} "
                            f"d_c {prm.clash_dist}: ")


def test_maximum_parameter_sizes(ctx, dk, oracle):
    """The largest restarts (1024), alignment angles per axis (128) and torsion angles (1024) the
    C-ABI accepts, on small ligands the oracle docks in seconds."""
    rng = np.random.Generator(np.random.PCG64(21))
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    pid = ctx.load(pk)
    # floors: 1024 restarts of a small ligand are nearly all tie-free; 128 x 128 alignment poses
    # (2.8 degree steps) and 1024 torsion angles put near-ties in every trajectory of the second case
    for (n, b), prm, floors in [
            ((10, 2), dk.Params.make(restarts=1024, align_steps=4, torsion_steps=64, seed=7), (0.9, 0.8, 1.0)),
            ((14, 2), dk.Params.make(restarts=2, align_steps=128, torsion_steps=1024, seed=8), (0.0, 0.5, 0.0))]:
        xyz, bonds, rot = _lig(rng, n, b)
        db = synth.from_ligands([(xyz, bonds, rot, 900 + n)])
        res = run(ctx, dk, pid, db, prm)
        rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm))
        assert_report(rep, *floors, label=f"R {prm.restarts} N {prm.align_steps} A {prm.torsion_steps}: ")


def test_ligands_sticking_out_of_a_small_grid(ctx, dk, oracle):
    pk = synth.make_pocket(14, 0.5, 3.0, 0.2, 5)   # 6.5 A wide: large ligands leave the grid
    db = synth.make_db(synth.WORKLOADS["tiny"], 10)
    prm = dk.Params.make(restarts=3, align_steps=10, torsion_steps=32, seed=6)
    res = run(ctx, dk, ctx.load(pk), db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.4, min_exact=0.7, min_best=0.4, label="ligands leaving a small grid: ")


def test_empty_batch(ctx, dk):
    pk, _, prm = tiny_setup(dk)
    res = run(ctx, dk, ctx.load(pk), synth.from_ligands([]), prm)
    assert res["score"].size == 0


@pytest.fixture(scope="module")
def uneven_db():
    return synth.make_db(synth.WORKLOADS["uneven"], workers=synth.default_workers())


@pytest.mark.parametrize("grid_dtype", ["f32", "f16"])
def test_uneven_database_full_size_sampled(ctx, dk, oracle, grid_dtype, uneven_db):
    """The 10,000-ligand uneven database at its full parameters (30 restarts, 30x30 alignment,
    256 torsion angles), launched as the benchmark launches it; sampled ligands against the oracle
    and size-free properties on every ligand."""
    w = synth.WORKLOADS["uneven"]
    pk = synth.workload_pocket(w)
    db = uneven_db
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    pid = ctx.load(pk, grid_dtype)
    res = run(ctx, dk, pid, db, prm)
    if grid_dtype == "f32":   # the benchmark's launch configuration: shapes tuned on the database
        from paper_2209_05069_gb300 import autotune
        try:
            autotune.tune(ctx, pid, db.slice(0, 4000), prm)
            tuned = run(ctx, dk, pid, db, prm)
        finally:
            ctx.reset_launch()
        for k in res:
            assert np.array_equal(res[k], tuned[k]), k
    R, A, N = prm.restarts, prm.torsion_steps, prm.align_steps
    rs = res["restart_score"].reshape(-1, R)
    assert np.array_equal(res["best_restart"], np.argmax(rs, axis=1))
    assert np.array_equal(res["score"], rs[np.arange(db.n_lig), res["best_restart"]])
    assert np.array_equal(res["clash_count"], res["restart_clash"].reshape(-1, R)[np.arange(db.n_lig), res["best_restart"]])
    assert ((res["align_idx"] >= 0) & (res["align_idx"] < N * N)).all()
    assert ((res["post_idx"] >= 0) & (res["post_idx"] < N * N)).all()
    assert ((res["torsion_idx"] >= 0) & (res["torsion_idx"] < A)).all()
    assert ((res["rejected"] >= 0) & (res["rejected"] <= A)).all()
    assert np.isfinite(res["xyz"]).all()
    # bond lengths survive every move
    d = np.linalg.norm(res["xyz"][db.bonds[:, 0] + np.repeat(db.atom_off[:-1], np.diff(db.bond_off))]
                       - res["xyz"][db.bonds[:, 1] + np.repeat(db.atom_off[:-1], np.diff(db.bond_off))], axis=1)
    assert np.abs(d - 1.5).max() < 1e-3
    # 1,024 ligands (FP32) / 512 (FP16) against the oracle: about 30 s of oracle on 16 host cores
    n_sample = 1024 if grid_dtype == "f32" else 512
    sample = np.random.Generator(np.random.PCG64(17)).choice(db.n_lig, n_sample, replace=False)
    rep = parity.check(oracle, oracle.GridView.of(pk, fp16=grid_dtype == "f16"), db, res, oparams(oracle, prm),
                       indices=sample)
    assert_report(rep, min_comparable=0.6, min_exact=0.45, min_best=0.6,
                  label=f"uneven 10,000, {grid_dtype} grid, {n_sample} sampled: ")


def test_launch_shapes_and_graph_replay_do_not_change_results(ctx, dk):
    pk, db, prm = tiny_setup(dk, seed=12)
    pid = ctx.load(pk)
    ref = run(ctx, dk, pid, db, prm)
    g0 = ctx.stats()["graph_launches"]
    b = ctx.batch_create(db, prm)
    try:
        for wpb, cv, ps, gi, tl in [(1, -1, 0, 1, 1), (2, 50, 0, 1, 1), (8, 75, 0, 1, 1), (3, 0, 0, 1, 1),
                                    (4, -1, 1, 1, 1), (2, 60, 1, 1, 1), (8, -1, 1, 1, 1), (2, -1, 0, 2, 1),
                                    (4, -1, 0, 4, 1), (8, 60, 1, 4, 1), (8, -1, 0, 8, 1), (8, -1, 1, 2, 1),
                                    (1, -1, 0, 1, 2), (4, -1, 1, 1, 2), (2, -1, 0, 2, 2), (8, -1, 1, 2, 2),
                                    (6, 60, 1, 2, 2)]:
            ctx.set_launch(0, wpb, cv, ps, gi, tl)
            ctx.batch_launch(pid, b)      # captured into a graph
            ctx.batch_launch(pid, b)      # replayed
            got = ctx.batch_results(b)
            for k in ref:
                assert np.array_equal(ref[k], got[k]), (wpb, cv, ps, gi, tl, k)
        with pytest.raises(dk.DockError):  # a tile of 2 needs 1 or 2 warps per item
            ctx.set_launch(0, 8, -1, 1, 4, 2)
    finally:
        ctx.reset_launch(0)
        ctx.batch_destroy(b)
    assert ctx.get_launch(0) == {"warps_per_block": 8, "smem_carveout_pct": -1, "persistent": 1,
                                 "warps_per_item": 2, "pose_tile": 1}   # the default shape, restored
    assert ctx.stats()["graph_launches"] - g0 >= 34


def test_autotuner_picks_a_shape_and_results_stay_identical(ctx, dk):
    from paper_2209_05069_gb300 import autotune
    w = synth.WORKLOADS["uneven"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 300, seed=123)
    prm = dk.Params.make(restarts=4, align_steps=10, torsion_steps=32, seed=1)
    pid = ctx.load(pk)
    ref = run(ctx, dk, pid, db, prm)
    try:
        table = autotune.tune(ctx, pid, db, prm, warps=(2, 4), carveouts=(-1, 60), persistent=(0, 1),
                              warps_per_item=(1, 4), tiles=(1, 2), reps=1)
        assert set(table) <= {0, 1, 2} and len(table) >= 2
        for row in table.values():
            # (2, 1, 1) (2, 1, 2) (4, 1, 1) (4, 1, 2) (4, 4, 1) per carveout and persistent choice
            assert len(row["tried"]) == 20
            if row["joint"]["chosen"] == "library default":   # the joint check also times the defaults
                continue
            assert row["warps_per_block"] in (2, 4) and row["smem_carveout"] in (-1, 60)
            assert row["persistent"] in (0, 1) and row["warps_per_item"] in (1, 4) and row["pose_tile"] in (1, 2)
        got = run(ctx, dk, pid, db, prm)
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k
        table = autotune.confirm(ctx, pid, db, prm, table, reps=1)
        for b, row in table.items():
            assert row["confirm"]["chosen"] in ("tuned", "library default")
            sh = ctx.get_launch(b)
            assert (sh["warps_per_block"], sh["warps_per_item"], sh["pose_tile"]) == (
                row["warps_per_block"], row["warps_per_item"], row["pose_tile"])
        got = run(ctx, dk, pid, db, prm)
        for k in ref:
            assert np.array_equal(ref[k], got[k]), k
    finally:
        for bkt in range(5):
            ctx.reset_launch(bkt)


@pytest.mark.parametrize("grid_dtype", ["f32", "f16"])
def test_large_molecules_full_parameters_sampled(ctx, dk, oracle, grid_dtype):
    """Large-molecule workload (80-150 atoms, 20-40 rotatable bonds, 96^3 grid at 0.375 A, 30
    restarts, 256 angles): a 24-ligand slice of the database docked in one batch, every one
    compared with the oracle in full (FP16: against an oracle reading the FP16-rounded grid)."""
    w = synth.WORKLOADS["large"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 24)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    res = run(ctx, dk, ctx.load(pk, grid_dtype), db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk, fp16=grid_dtype == "f16"), db, res, oparams(oracle, prm))
    # 20-40 bonds of 256 angles each: most trajectories hold some decision within 1e-6 of a tie
    assert_report(rep, min_comparable=0.08, min_exact=0.22, label=f"large molecules 24, {grid_dtype} grid: ")


@pytest.mark.parametrize("grid_dtype", ["f32", "f16"])
def test_large_molecules_score_error_per_ligand(ctx, dk, oracle, grid_dtype):
    """Large-molecule workload, 2,000 ligands at full parameters: every ligand's final score
    against the FP64 oracle's score of the same final pose on the FP32 grid (for the FP16 grid the
    error includes the grid's rounding), the per-ligand score error of the large-molecule stress
    configuration."""
    w = synth.WORKLOADS["large"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 2000, workers=synth.default_workers())
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    res = run(ctx, dk, ctx.load(pk, grid_dtype), db, prm)
    g32 = oracle.GridView.of(pk)
    err = np.empty(db.n_lig)
    for l in range(db.n_lig):
        s64 = oracle.score(g32, res["xyz"][db.atom_off[l]:db.atom_off[l + 1]])
        err[l] = abs(float(res["score"][l]) - s64) / max(abs(s64), 1.0)
    print(f"\n{grid_dtype}: per-ligand relative score error over {db.n_lig} ligands: max {err.max():.2e}, "
          f"p99 {np.quantile(err, 0.99):.2e}, median {np.median(err):.2e}")
    assert err.max() <= (2e-3 if grid_dtype == "f16" else 1e-4)


def _size_free_properties(res, db, prm):
    R = prm.restarts
    rs = res["restart_score"].reshape(-1, R)
    assert np.array_equal(res["best_restart"], np.argmax(rs, axis=1))
    assert np.array_equal(res["score"], rs[np.arange(db.n_lig), res["best_restart"]])
    assert ((res["torsion_idx"] >= 0) & (res["torsion_idx"] < prm.torsion_steps)).all()
    assert np.isfinite(res["xyz"]).all()
    lig_of_bond = np.repeat(np.arange(db.n_lig), np.diff(db.bond_off))
    a0 = db.atom_off[:-1][lig_of_bond]
    d = np.linalg.norm(res["xyz"][db.bonds[:, 0] + a0] - res["xyz"][db.bonds[:, 1] + a0], axis=1)
    assert np.abs(d - 1.5).max() < 1e-3   # every move keeps every bond length


def test_large_molecules_full_size_sampled(ctx, dk, oracle):
    """The large-molecule configuration at its full size: 20,000 ligands of 80-150 atoms and 20-40
    rotatable bonds, docked in one batch with shapes tuned on it; size-free properties on every
    ligand, 64 sampled ligands against the oracle."""
    from paper_2209_05069_gb300 import autotune
    w = synth.WORKLOADS["large"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, workers=synth.default_workers())
    assert db.n_lig == 20_000
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    pid = ctx.load(pk)
    try:
        autotune.tune(ctx, pid, db.slice(0, 2000), prm)
        res = run(ctx, dk, pid, db, prm)
    finally:
        ctx.reset_launch()
    _size_free_properties(res, db, prm)
    sample = np.random.Generator(np.random.PCG64(29)).choice(db.n_lig, 64, replace=False)
    rep = parity.check(oracle, oracle.GridView.of(pk), db, res, oparams(oracle, prm), indices=sample)
    assert_report(rep, min_comparable=0.08, min_exact=0.22, label="large molecules 20,000, 64 sampled: ")


def test_plateau_million_ligands_sampled(ctx, dk, oracle):
    """The plateau sweep's largest database: 10^6 ligands of the uneven size mix through one 128^3
    FP16 pocket in one batch; size-free properties on every ligand, 32 sampled against the oracle."""
    w = synth.WORKLOADS["plateau"]
    pk = synth.workload_pocket(w)
    pool = synth.make_db(w, 10_000, workers=synth.default_workers())
    db = synth.tile_db(pool, 1_000_000, first_id=10_000_000)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209, outputs=dk.DOCK_OUTPUT_FULL)
    res = run(ctx, dk, ctx.load(pk, "f16"), db, prm)
    _size_free_properties(res, db, prm)
    sample = np.concatenate([[0, 999_999], np.random.Generator(np.random.PCG64(31)).choice(
        np.arange(1, 999_999), 30, replace=False)])
    rep = parity.check(oracle, oracle.GridView.of(pk, fp16=True), db, res, oparams(oracle, prm), indices=sample)
    assert_report(rep, min_comparable=0.5, min_exact=0.35, min_best=0.5, label="plateau 10^6, 32 sampled: ")


def test_plateau_grid_fp16_sampled(ctx, dk, oracle):
    """The 128^3 FP16 pocket of the database-size sweep with the uneven size distribution."""
    w = synth.WORKLOADS["plateau"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 200)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209)
    res = run(ctx, dk, ctx.load(pk, "f16"), db, prm)
    rep = parity.check(oracle, oracle.GridView.of(pk, fp16=True), db, res, oparams(oracle, prm))
    assert_report(rep, min_comparable=0.6, min_exact=0.35, min_best=0.6, label="plateau grid, 200 ligands: ")
