"""Select Poses on the GPU against the oracle (Alg. 1, after the restart loop).

The kernel keeps up to K restart poses per ligand, walking the restarts in order of final score
(ties: lowest restart) and keeping a pose whose RMSD to every kept pose is at least the threshold.
Checks:

* selection is post-processing only: every other output equals that of a run with K = 1;
* the outputs are consistent: the first kept pose is the best restart, scores and poses are those
  of the kept restarts, empty slots hold -1 / -inf / zeros;
* replay: the oracle's selection over the GPU's own FP32 scores and the FP64 poses of the GPU's
  decisions equals the GPU's selection wherever no RMSD test is within 1e-3 A of the threshold
  (the pose error bound), and the kept poses match those FP64 poses to 1e-3 A RMSD;
* direct: where every restart's trajectory matches the oracle's free run and neither a score tie
  (1e-4 relative) nor an RMSD test (1e-3 A) is near, the oracle's own selection is the GPU's.
"""
import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

from . import parity

pytestmark = pytest.mark.gpu

KEYS = ["score", "best_restart", "xyz", "clash_count", "restart_score", "restart_clash", "align_idx", "post_idx",
        "torsion_idx", "rejected"]
RMSD_NEAR = 1e-3    # A: an RMSD test this close to the threshold may fall either side in FP32
SCORE_NEAR = 1e-4   # relative: score gaps this small may reorder restarts in FP32


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


def rmsd(a, b):
    return float(np.sqrt(((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2).sum(axis=1).mean()))


def check_selection(oracle, grid_view, db, res, prm, indices, threads=8):
    """Returns (ligands compared by replay, ligands compared directly, ambiguous ligands)."""
    R, K = prm.restarts, prm.k
    thr = float(np.float32(prm.select_rmsd))
    op = oparams(oracle, prm)
    g_all = parity.gpu_split(res, db, R)
    idx = [int(i) for i in indices]
    forced = {"align": {}, "post": {}, "tors": {}}
    for l in idx:
        forced["align"][l] = g_all[l]["align_idx"]
        forced["post"][l] = g_all[l]["post_idx"]
        forced["tors"][l] = g_all[l]["torsion_idx"].reshape(-1)
    replay = oracle.dock_db(grid_view, db, op, threads=threads, indices=idx, forced=forced)
    free = oracle.dock_db(grid_view, db, op, threads=threads, indices=idx)
    n_replay = n_direct = n_ambiguous = 0
    for l, o_rep, o_free in zip(idx, replay, free):
        a0, a1 = db.atom_off[l], db.atom_off[l + 1]
        n = a1 - a0
        sel = res["select_restart"][l * K:(l + 1) * K]
        ssc = res["select_score"][l * K:(l + 1) * K]
        sxyz = res["select_xyz"][a0 * K:a1 * K].reshape(K, n, 3)
        rs = g_all[l]["restart_score"]
        nk = int((sel >= 0).sum())
        # consistency of the outputs
        assert nk >= 1 and (sel[:nk] >= 0).all() and (sel[nk:] == -1).all(), (l, sel)
        assert sel[0] == g_all[l]["best_restart"] and np.array_equal(sxyz[0], g_all[l]["xyz"]), l
        assert np.array_equal(ssc[:nk], rs[sel[:nk]]) and np.isneginf(ssc[nk:]).all(), l
        assert not sxyz[nk:].any(), l
        assert len(set(sel[:nk].tolist())) == nk, l
        # replay: the GPU's scores, the FP64 poses of the GPU's decisions
        o = oracle.select_poses(rs.astype(np.float64), o_rep["restart_xyz"], K, thr)
        for k in range(nk):
            assert rmsd(sxyz[k], o_rep["restart_xyz"][sel[k]]) < parity.RMSD_TOL, (l, k)
        if o["rmsd_margin"] > RMSD_NEAR:
            assert np.array_equal(o["sel"], sel), (l, o["sel"], sel)
            n_replay += 1
        else:
            n_ambiguous += 1
            for i in range(nk):          # still a valid selection up to the threshold's noise
                for j in range(i):
                    assert rmsd(sxyz[i], sxyz[j]) >= thr - RMSD_NEAR, (l, i, j)
        # direct: the oracle's free run, where every trajectory is the GPU's and no decision is near
        same = np.allclose(o_free["restart_score"], rs, rtol=parity.SCORE_REL, atol=parity.SCORE_REL) and all(
            rmsd(o_free["restart_xyz"][r], o_rep["restart_xyz"][r]) < 1e-9 for r in range(R))
        of = oracle.select_poses(o_free["restart_score"], o_free["restart_xyz"], K, thr)
        if same and of["rmsd_margin"] > RMSD_NEAR and of["score_margin"] > SCORE_NEAR * max(1.0, abs(rs).max()):
            assert np.array_equal(of["sel"], sel), (l, of["sel"], sel)
            n_direct += 1
    return n_replay, n_direct, n_ambiguous


def test_tiny_workload_selection(ctx, dk, oracle):
    w = synth.WORKLOADS["tiny"]
    pk, db = synth.workload_pocket(w), synth.make_db(w)
    pid = ctx.load(pk)
    base = dict(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                clash_dist=w.clash_dist, seed=31)
    ref = run(ctx, pid, db, dk.Params.make(**base))
    for K, thr in [(4, 2.0), (8, 1.0), (3, 0.0), (8, 1e6)]:
        prm = dk.Params.make(**base, select_k=K, select_rmsd=thr)
        res = run(ctx, pid, db, prm)
        for k in KEYS:
            assert np.array_equal(res[k], ref[k]), (K, thr, k)
        nr, nd, na = check_selection(oracle, oracle.GridView.of(pk), db, res, prm, range(db.n_lig))
        print(f"\nK={K} thr={thr}: {nr} replay / {nd} direct / {na} ambiguous of {db.n_lig} ligands")
        assert nr >= 0.8 * db.n_lig and nd >= 1
        sel = res["select_restart"].reshape(db.n_lig, K)
        if thr == 0.0:   # top K by score, ties to the lowest restart
            rs = res["restart_score"].reshape(db.n_lig, -1)
            for l in range(db.n_lig):
                assert list(sel[l]) == list(np.lexsort((np.arange(w.restarts), -rs[l]))[:K])
        if thr == 1e6:   # nothing else is far enough
            assert (sel[:, 0] == ref["best_restart"]).all() and (sel[:, 1:] == -1).all()


def test_selection_is_the_same_in_every_launch_form(ctx, dk):
    w = synth.WORKLOADS["tiny"]
    pk, db = synth.workload_pocket(w), synth.make_db(w, seed=8)
    pid = ctx.load(pk)
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=4, select_k=5, select_rmsd=1.5)
    ref = run(ctx, pid, db, prm)
    got = [run(ctx, pid, db, prm, form=dk.DOCK_FORM_PER_LIGAND)]
    try:
        for wpb, ps, g, tl in [(8, 0, 2, 1), (8, 0, 8, 1), (4, 1, 1, 1), (8, 1, 2, 2)]:
            ctx.set_launch(0, wpb, -1, ps, g, tl)
            got.append(run(ctx, pid, db, prm))
    finally:
        ctx.reset_launch(0)
    for r in got:
        for k in KEYS + ["select_restart", "select_score", "select_xyz"]:
            assert np.array_equal(r[k], ref[k]), k
    with dk.Context() as sctx:           # the serving loop scatters the same selection
        served = sctx.dock(sctx.load(pk), db, prm)
    for k in ["select_restart", "select_score", "select_xyz"]:
        assert np.array_equal(served[k], ref[k]), k


def test_uneven_database_selection_sampled(ctx, dk, oracle):
    """The uneven database at its full parameters with K = 16 (the largest K) and a 2 A threshold:
    sampled ligands against the oracle, output consistency on every ligand."""
    w = synth.WORKLOADS["uneven"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 2000, workers=synth.default_workers())
    prm = dk.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                         clash_dist=w.clash_dist, seed=2209, select_k=16, select_rmsd=2.0)
    res = run(ctx, ctx.load(pk), db, prm)
    K, R = prm.k, prm.restarts
    sel = res["select_restart"].reshape(-1, K)
    assert (sel[:, 0] == res["best_restart"]).all()
    nk = (sel >= 0).sum(axis=1)
    assert (nk >= 1).all() and (nk > 1).mean() > 0.5
    rs = res["restart_score"].reshape(-1, R)
    got = np.where(sel >= 0, rs[np.arange(db.n_lig)[:, None], np.maximum(sel, 0)], -np.inf).astype(np.float32)
    assert np.array_equal(res["select_score"].reshape(-1, K), got)
    ss = res["select_score"].reshape(-1, K)
    kept = sel[:, 1:] >= 0   # unused slots hold -inf; compare kept neighbours only
    assert (ss[:, 1:][kept] <= ss[:, :-1][kept]).all()
    sample = np.random.Generator(np.random.PCG64(23)).choice(db.n_lig, 10, replace=False)
    nr, nd, na = check_selection(oracle, oracle.GridView.of(pk), db, res, prm, sample)
    print(f"\n{nr} replay / {nd} direct / {na} ambiguous of {len(sample)} sampled ligands")
    assert nr >= 8
