"""The GPU parity harness (tests/parity.py) can fail (CPU only).

The oracle's own results, laid out the way the GPU library returns them, must pass the harness;
the same results with one planted difference — an alignment index, a torsion index, a rejected
count, a score or a pose off by more than the tolerance — must not, and a score within the
tolerance must still pass.  No GPU is involved: the differences are planted in oracle output.
"""
import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

from . import parity

R, N, A = 4, 12, 32


@pytest.fixture(scope="module")
def case(oracle):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 6, seed=5)
    p = oracle.Params(restarts=R, align_steps=N, torsion_steps=A, clash_dist=2.0, post_align=1, seed=4)
    g = oracle.GridView.of(pk)
    outs = oracle.dock_db(g, db, p, threads=4)
    return db, p, g, outs


def gpu_layout(db, outs, R=R):
    """Oracle results in the flat layout of dock_results (FP32 where the library returns FP32)."""
    L = db.n_lig
    res = {"score": np.zeros(L, np.float32), "best_restart": np.zeros(L, np.int32),
           "xyz": np.zeros((db.atom_off[-1], 3), np.float32), "clash_count": np.zeros(L, np.int32),
           "restart_score": np.zeros(L * R, np.float32), "restart_clash": np.zeros(L * R, np.int32),
           "align_idx": np.zeros(L * R, np.int32), "post_idx": np.zeros(L * R, np.int32),
           "torsion_idx": np.zeros(db.rot_off[-1] * R, np.int32), "rejected": np.zeros(db.rot_off[-1] * R, np.int32)}
    for l, o in enumerate(outs):
        br = int(np.asarray(o["best_restart"]).reshape(-1)[0])
        a0, a1, r0, r1 = db.atom_off[l], db.atom_off[l + 1], db.rot_off[l], db.rot_off[l + 1]
        res["best_restart"][l] = br
        res["restart_score"][l * R:(l + 1) * R] = o["restart_score"]
        res["score"][l] = res["restart_score"][l * R + br]
        res["restart_clash"][l * R:(l + 1) * R] = o["clash"]
        res["clash_count"][l] = o["clash"][br]
        res["align_idx"][l * R:(l + 1) * R] = o["align_idx"]
        res["post_idx"][l * R:(l + 1) * R] = o["post_idx"]
        res["torsion_idx"][r0 * R:r1 * R] = np.asarray(o["torsion_idx"]).reshape(-1)[:(r1 - r0) * R]
        res["rejected"][r0 * R:r1 * R] = np.asarray(o["rejected"]).reshape(-1)[:(r1 - r0) * R]
        res["xyz"][a0:a1] = np.asarray(o["restart_xyz"]).reshape(R, a1 - a0, 3)[br]
    return res


def first_comparable(db, outs, p):
    for l, o in enumerate(outs):
        for r in range(R):
            if parity.trajectory_comparable(o, r, p.post_align) and db.n_rot(l) > 0:
                return l, r
    pytest.skip("no comparable trajectory with a rotatable bond")


def test_oracle_results_pass(oracle, case):
    db, p, g, outs = case
    rep = parity.check(oracle, g, db, gpu_layout(db, outs), p, threads=4)
    assert not rep.failures, rep.failures
    assert rep.comparable > 0 and rep.ligands_comparable > 0


@pytest.mark.parametrize("plant", ["align_idx", "post_idx", "torsion_idx", "rejected", "score", "pose",
                                   "score_within_tolerance"])
def test_planted_differences_fail(oracle, case, plant):
    db, p, g, outs = case
    res = gpu_layout(db, outs)
    l, r = first_comparable(db, outs, p)
    i = l * R + r
    t = db.rot_off[l] * R + r * db.n_rot(l)   # first bond of restart r
    if plant == "align_idx":
        res["align_idx"][i] = (res["align_idx"][i] + 1) % (N * N)
    elif plant == "post_idx":
        res["post_idx"][i] = (res["post_idx"][i] + 1) % (N * N)
    elif plant == "torsion_idx":
        res["torsion_idx"][t] = (res["torsion_idx"][t] + 1) % A
    elif plant == "rejected":
        res["rejected"][t] += 1
    elif plant in ("score", "score_within_tolerance"):
        f = 3e-4 if plant == "score" else 3e-5
        res["restart_score"][i] += np.float32(f * max(1.0, abs(float(res["restart_score"][i]))))
        if res["best_restart"][l] == r:
            res["score"][l] = res["restart_score"][i]
    elif plant == "pose":
        a0 = db.atom_off[l]
        res["xyz"][a0:db.atom_off[l + 1]] += np.float32(0.01)
    rep = parity.check(oracle, g, db, res, p, indices=[l], threads=4)
    if plant == "score_within_tolerance":
        assert not rep.failures, rep.failures
    else:
        assert rep.failures, f"planted {plant} difference was not reported"


@pytest.fixture(scope="module")
def case_int(oracle):
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w).integer(1000)
    db = synth.make_db(w, 6, seed=6)
    p = oracle.Params(restarts=R, align_steps=N, torsion_steps=A, clash_dist=2.0, post_align=1, seed=9)
    g = oracle.GridView.of(pk, nearest=True)
    outs = oracle.dock_db(g, db, p, threads=4)
    return db, p, g, outs


@pytest.mark.parametrize("plant", [None, "align_idx", "torsion_idx", "score"])
def test_integer_grid_harness(oracle, case_int, plant):
    """Integer grids: exact scores and robust decisions must match exactly; a score one unit off or
    a changed index is reported."""
    db, p, g, outs = case_int
    res = gpu_layout(db, outs)
    if plant is not None:
        hit = [(l, r) for l, o in enumerate(outs) for r in range(R)
               if parity.int_trajectory_comparable(o, r, p.post_align) and db.n_rot(l) > 0]
        if not hit:
            pytest.skip("no comparable trajectory with a rotatable bond")
        l, r = hit[0]
        i = l * R + r
        if plant == "align_idx":
            res["align_idx"][i] = (res["align_idx"][i] + 1) % (N * N)
        elif plant == "torsion_idx":
            t = db.rot_off[l] * R + r * db.n_rot(l)
            res["torsion_idx"][t] = (res["torsion_idx"][t] + 1) % A
        else:
            res["restart_score"][i] += np.float32(1.0)
            if res["best_restart"][l] == r:
                res["score"][l] = res["restart_score"][i]
        rep = parity.check(oracle, g, db, res, p, indices=[l], threads=4)
        assert rep.failures, f"planted {plant} difference was not reported"
    else:
        rep = parity.check(oracle, g, db, res, p, threads=4)
        assert not rep.failures, rep.failures
        assert rep.comparable > 0


def test_selection_check_reports_planted_differences(oracle, case):
    """The Select Poses comparison of the GPU tests (check_selection) passes the oracle's own
    selection and rejects a different kept restart or a kept pose 0.017 A off."""
    import types
    from .test_gpu_select import check_selection
    db, p, g, outs = case
    K, thr = 3, 1.0
    prm = types.SimpleNamespace(restarts=R, k=K, select_rmsd=thr, align_steps=N, torsion_steps=A, clash_dist=2.0,
                                post_align=1, seed=4)
    res = gpu_layout(db, outs)
    L = db.n_lig
    res["select_restart"] = np.full(L * K, -1, np.int32)
    res["select_score"] = np.full(L * K, -np.inf, np.float32)
    res["select_xyz"] = np.zeros((db.atom_off[-1] * K, 3), np.float32)
    multi = []
    for l, o in enumerate(outs):
        a0, a1 = db.atom_off[l], db.atom_off[l + 1]
        rs = res["restart_score"][l * R:(l + 1) * R]
        xyz = np.asarray(o["restart_xyz"]).reshape(R, a1 - a0, 3)
        sel = oracle.select_poses(rs.astype(np.float64), xyz, K, float(np.float32(thr)))["sel"]
        nk = int((sel >= 0).sum())
        res["select_restart"][l * K:l * K + nk] = sel[:nk]
        res["select_score"][l * K:l * K + nk] = rs[sel[:nk]]
        res["select_xyz"][a0 * K:a1 * K].reshape(K, a1 - a0, 3)[:nk] = xyz[sel[:nk]]
        res["select_xyz"][a0 * K:a0 * K + (a1 - a0)] = res["xyz"][a0:a1]   # slot 0: the best pose as returned
        if nk >= 2 and nk < R:
            multi.append(l)
    check_selection(oracle, g, db, res, prm, range(L), threads=4)
    if not multi:
        pytest.skip("no ligand keeps between 2 and R - 1 poses")
    l = multi[0]
    a0, a1 = db.atom_off[l], db.atom_off[l + 1]
    n = a1 - a0
    sel = res["select_restart"][l * K:(l + 1) * K]
    other = next(r for r in range(R) if r not in sel.tolist())
    xyz = np.asarray(outs[l]["restart_xyz"]).reshape(R, n, 3)
    bad = {k: v.copy() for k, v in res.items()}
    bad["select_restart"][l * K + 1] = other
    bad["select_score"][l * K + 1] = res["restart_score"][l * R + other]
    bad["select_xyz"][a0 * K + n:a0 * K + 2 * n] = xyz[other]
    with pytest.raises(AssertionError):
        check_selection(oracle, g, db, bad, prm, [l], threads=4)
    bad = {k: v.copy() for k, v in res.items()}
    bad["select_xyz"][a0 * K + n:a0 * K + 2 * n] += np.float32(0.01)
    with pytest.raises(AssertionError):
        check_selection(oracle, g, db, bad, prm, [l], threads=4)


def test_exact_decision_check_reports_a_changed_choice(oracle, case):
    """A torsion choice changed at a decision clear of 1e-4 ties is reported by the per-decision
    check (in the replayed state), and the oracle's own results count exact decisions."""
    db, p, g, outs = case
    res = gpu_layout(db, outs)
    rep = parity.check(oracle, g, db, res, p, threads=4)
    assert not rep.failures and rep.decisions_exact > 0 and rep.rejected_exact > 0
    for l, o in enumerate(outs):
        B = db.n_rot(l)
        for r in range(R):
            for b in range(B):
                best, second = o["tors_best"][r, b], o["tors_second"][r, b]
                if o["tors_ambiguous"][r, b] == 0 and np.isfinite(best) and parity.clear_gap(best, second):
                    t = db.rot_off[l] * R + r * B + b
                    res["torsion_idx"][t] = (res["torsion_idx"][t] + 1) % A
                    rep = parity.check(oracle, g, db, res, p, indices=[l], threads=4)
                    assert any("(exact)" in f for f in rep.failures), rep.failures
                    return
    pytest.skip("no torsion decision clear of 1e-4 ties")
