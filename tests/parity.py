"""GPU-vs-oracle comparison used by the GPU parity tests.

Two checks, both against the FP64 oracle (arXiv 2209.05069 Alg. 1 as restated in
oracle/dock_oracle.cpp):

* direct: on every (ligand, restart) trajectory whose decisions FP32 rounding cannot flip
  (alignment and torsion top-two score gaps above 1e-6 relative, which includes every trajectory
  whose gaps exceed 1e-4 relative, and no angle within 1e-4 A of the bump threshold), every
  integer output must match bit for bit and scores to 1e-4 relative;
* replay: for every trajectory, the oracle follows the GPU's own decisions in double precision
  and each decision must be one the method allows there: the chosen alignment within FP32 noise
  of the best pose; the chosen angle not clearly bumping and within FP32 noise of the best angle
  that is clearly bump-free; the rejected count within the number of angles whose bump decision
  sits on the threshold.  The GPU's scores, clash counts and best pose must then match the replay
  (1e-4 relative, exact where not on the threshold, 1e-3 A RMSD).
* per decision (within the replay, so it covers every trajectory, also after an earlier tie):
  wherever the oracle's top two scores in the state the GPU reached differ by more than 1e-4
  relative (and, for a torsion, no angle sits within 1e-4 A of the bump threshold), the GPU's
  chosen index must be the oracle's argmax exactly; rejected counts of bonds with no angle on the
  threshold must match exactly, and so must clash counts off the threshold.

Integer grids (nearest voxel, oracle mode 1) have exact integer scores, so ties are real and are
broken by the lowest index on both sides.  What FP32 can change is which voxel an atom within
1e-4 grid units of a half-way plane reads; the oracle carries every score's range over such moves
and flags each decision as the only possible one (robust) or as a possible one.  Direct: every
trajectory whose decisions are all robust and whose final score range is a single value must match
bit for bit, scores exactly.  Replay: every GPU decision must be possible and every GPU score must
lie in the replayed score's range.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

SCORE_REL = 1e-4        # score tolerance, relative to max(|s|, 1)
DECISION_REL = 1e-4     # top-two gap (relative) above which the chosen index must match exactly
TIGHT_REL = 1e-6        # tighter tie threshold, still 10x the FP32 score error measured on GB300
                        # (1e-7 relative): trajectories clear of ties at this level must match too
CLASH_EPS = 1e-4        # A: pairs this close to d_c may fall either side in FP32
RMSD_TOL = 1e-3         # A
NOISE_REL = 2e-5        # deficit a GPU choice may have against the FP64 best (FP32 summation noise)


def scale(s):
    return np.maximum(np.abs(s), 1.0)


@dataclasses.dataclass
class Report:
    trajectories: int = 0
    comparable: int = 0         # clear of ties at TIGHT_REL: compared directly
    comparable_1e4: int = 0     # clear of ties at DECISION_REL (a subset of the above)
    ligands: int = 0
    ligands_comparable: int = 0
    max_score_rel: float = 0.0
    max_rmsd: float = 0.0
    replay_max_score_rel: float = 0.0
    replay_max_rmsd: float = 0.0
    decisions: int = 0          # alignment, post-alignment and torsion decisions replayed
    decisions_exact: int = 0    # of which clear of ties at DECISION_REL: index compared exactly
    rejected_exact: int = 0     # bonds with no angle on the bump threshold: rejected count exact
    clash_exact: int = 0        # restarts whose final clash count is off the threshold: exact
    failures: list = dataclasses.field(default_factory=list)

    def merge(self, other: "Report") -> "Report":
        for f in dataclasses.fields(self):
            a, b = getattr(self, f.name), getattr(other, f.name)
            if f.name == "failures":
                a.extend(b[:max(0, 20 - len(a))])
            elif f.name.startswith("max") or f.name.startswith("replay_max"):
                setattr(self, f.name, max(a, b))
            else:
                setattr(self, f.name, a + b)
        return self

    def summary(self) -> str:
        return (f"{self.ligands} ligands; trajectories: {self.comparable}/{self.trajectories} compared directly "
                f"(clear of 1e-6 ties), {self.comparable_1e4} clear of 1e-4 ties; {self.ligands_comparable} best "
                f"poses compared directly; decisions: {self.decisions_exact}/{self.decisions} clear of 1e-4 ties and "
                f"exact, {self.rejected_exact} rejected counts and {self.clash_exact} clash counts exact; max score "
                f"rel err {self.max_score_rel:.2e} (replay {self.replay_max_score_rel:.2e}), max RMSD "
                f"{self.max_rmsd:.2e} A (replay {self.replay_max_rmsd:.2e})")

    def fail(self, msg):
        if len(self.failures) < 20:
            self.failures.append(msg)


def gpu_split(res, db, R):
    """Per-ligand views of the GPU's flat result arrays."""
    out = []
    for l in range(db.n_lig):
        a0, a1 = db.atom_off[l], db.atom_off[l + 1]
        r0, r1 = db.rot_off[l], db.rot_off[l + 1]
        B = r1 - r0
        out.append(dict(
            score=float(res["score"][l]), best_restart=int(res["best_restart"][l]), xyz=res["xyz"][a0:a1],
            clash=int(res["clash_count"][l]),
            restart_score=res["restart_score"][l * R:(l + 1) * R], restart_clash=res["restart_clash"][l * R:(l + 1) * R],
            align_idx=res["align_idx"][l * R:(l + 1) * R], post_idx=res["post_idx"][l * R:(l + 1) * R],
            torsion_idx=res["torsion_idx"][r0 * R:r1 * R].reshape(R, B),
            rejected=res["rejected"][r0 * R:r1 * R].reshape(R, B)))
    return out


def trajectory_comparable(o, r, post_align, rel=TIGHT_REL):
    """True if no decision of oracle restart r is a tie at relative level `rel` or sits on the
    bump threshold (so FP32 rounding cannot flip it)."""
    if (o["align_best"][r] - o["align_second"][r]) <= rel * scale(o["align_best"][r]):
        return False
    if post_align and (o["post_best"][r] - o["post_second"][r]) <= rel * scale(o["post_best"][r]):
        return False
    B = o["torsion_idx"].shape[1] if o["torsion_idx"].ndim == 2 else 0
    for b in range(B):
        if o["tors_ambiguous"][r, b] > 0:
            return False
        best, second = o["tors_best"][r, b], o["tors_second"][r, b]
        if np.isfinite(best) and np.isfinite(second) and best - second <= rel * scale(best):
            return False
    return True


def compare_direct(g, o, R, post_align, rep: Report, lig):
    for r in range(R):
        rep.trajectories += 1
        rep.comparable_1e4 += int(trajectory_comparable(o, r, post_align, DECISION_REL))
        if not trajectory_comparable(o, r, post_align):
            continue
        rep.comparable += 1
        where = f"ligand {lig} restart {r}"
        if g["align_idx"][r] != o["align_idx"][r]:
            rep.fail(f"{where}: align_idx {g['align_idx'][r]} != {o['align_idx'][r]}")
        if g["post_idx"][r] != o["post_idx"][r]:
            rep.fail(f"{where}: post_idx {g['post_idx'][r]} != {o['post_idx'][r]}")
        if not np.array_equal(g["torsion_idx"][r], o["torsion_idx"][r]):
            rep.fail(f"{where}: torsion_idx {g['torsion_idx'][r].tolist()} != {o['torsion_idx'][r].tolist()}")
        if not np.array_equal(g["rejected"][r], o["rejected"][r]):
            rep.fail(f"{where}: rejected {g['rejected'][r].tolist()} != {o['rejected'][r].tolist()}")
        err = abs(g["restart_score"][r] - o["restart_score"][r]) / scale(o["restart_score"][r])
        rep.max_score_rel = max(rep.max_score_rel, float(err))
        if err > SCORE_REL:
            rep.fail(f"{where}: score {g['restart_score'][r]} vs {o['restart_score'][r]}")
        if o["clash_margin"][r] > CLASH_EPS and g["restart_clash"][r] != o["clash"][r]:
            rep.fail(f"{where}: clash {g['restart_clash'][r]} != {o['clash'][r]}")


def compare_best(g, o, o_rep, R, post_align, rep: Report, lig):
    """The best restart and its pose, compared directly where they are unique: the oracle's best
    restart r* followed a trajectory FP32 cannot flip (so the GPU's restart r* is the oracle's) and
    its score beats every restart the GPU actually docked (their double-precision replays) by more
    than 1e-6 relative; the GPU must then pick r* and report the oracle's pose of it."""
    rb = int(o["best_restart"])
    if not trajectory_comparable(o, rb, post_align):
        return
    others = np.delete(np.asarray(o_rep["restart_score"], np.float64), rb)
    top = float(o["restart_score"][rb])
    if others.size and top - others.max() <= TIGHT_REL * scale(top):
        return
    rep.ligands_comparable += 1
    if g["best_restart"] != rb:
        rep.fail(f"ligand {lig}: best_restart {g['best_restart']} != {rb}")
        return
    d = np.sqrt(np.mean(np.sum((g["xyz"] - o["restart_xyz"][rb]) ** 2, axis=1)))
    rep.max_rmsd = max(rep.max_rmsd, float(d))
    if d > RMSD_TOL:
        rep.fail(f"ligand {lig}: best pose RMSD {d}")


def clear_gap(best, second, rel=DECISION_REL):
    """True if `best` beats `second` by more than rel * max(|best|, 1) (or nothing is second)."""
    if not np.isfinite(second):
        return True
    return best - second > rel * scale(best)


def exact_decisions(g, o, R, A, post_align, rep: Report, lig):
    """Spec bar per decision, in the state the GPU reached (the replay): a choice clear of
    ties at DECISION_REL must be the oracle's argmax; counts off the bump threshold must be equal."""
    B = g["torsion_idx"].shape[1]
    for r in range(R):
        where = f"ligand {lig} restart {r} (exact)"
        phases = [("alignment", o["align_best"][r], o["align_second"][r], o["align_forced"][r], g["align_idx"][r])]
        if post_align:
            phases.append(("post alignment", o["post_best"][r], o["post_second"][r], o["post_forced"][r],
                           g["post_idx"][r]))
        for name, best, second, forced, idx in phases:
            rep.decisions += 1
            if clear_gap(best, second):
                rep.decisions_exact += 1
                if forced != best:
                    rep.fail(f"{where}: {name} {idx} scores {forced}, the unique best is {best} (gap "
                             f"{best - second:.3e})")
        for b in range(B):
            rep.decisions += 1
            if int(o["tors_ambiguous"][r, b]) != 0:
                continue
            k, rej = int(g["torsion_idx"][r, b]), int(g["rejected"][r, b])
            rep.rejected_exact += 1
            if rej != int(o["rejected"][r, b]):
                rep.fail(f"{where} bond {b}: rejected {rej} != {o['rejected'][r, b]}")
            best, second = o["tors_best"][r, b], o["tors_second"][r, b]
            if not np.isfinite(best):   # every angle bumps: the conformation is kept (k = 0)
                rep.decisions_exact += 1
                if k != 0:
                    rep.fail(f"{where} bond {b}: every angle bumps but angle {k} was applied")
            elif clear_gap(best, second):
                rep.decisions_exact += 1
                if o["tors_forced"][r, b] != best or o["tors_forced_margin"][r, b] < 0:
                    rep.fail(f"{where} bond {b}: angle {k} scores {o['tors_forced'][r, b]}, the unique best "
                             f"accepted angle scores {best}")
        if o["clash_margin"][r] > CLASH_EPS:
            rep.clash_exact += 1


def compare_replay(g, o, R, A, post_align, rep: Report, lig):
    """`o` is the oracle run forced with the GPU's decisions."""
    exact_decisions(g, o, R, A, post_align, rep, lig)
    for r in range(R):
        where = f"ligand {lig} restart {r} (replay)"
        if o["align_forced"][r] < o["align_best"][r] - NOISE_REL * scale(o["align_best"][r]):
            rep.fail(f"{where}: alignment {g['align_idx'][r]} scores {o['align_forced'][r]} < best {o['align_best'][r]}")
        if post_align and o["post_forced"][r] < o["post_best"][r] - NOISE_REL * scale(o["post_best"][r]):
            rep.fail(f"{where}: post alignment {g['post_idx'][r]} scores {o['post_forced'][r]} < best {o['post_best'][r]}")
        B = g["torsion_idx"].shape[1]
        for b in range(B):
            k, rej = int(g["torsion_idx"][r, b]), int(g["rejected"][r, b])
            amb = int(o["tors_ambiguous"][r, b])
            if abs(rej - int(o["rejected"][r, b])) > amb:
                rep.fail(f"{where} bond {b}: rejected {rej} vs {o['rejected'][r, b]} (+-{amb})")
            if rej == A:
                if k != 0 or o["tors_robust_valid"][r, b] > 0:
                    rep.fail(f"{where} bond {b}: no accepted angle on GPU but oracle has {o['tors_robust_valid'][r, b]}")
                continue
            if o["tors_forced_margin"][r, b] < -CLASH_EPS:
                rep.fail(f"{where} bond {b}: angle {k} bumps (margin {o['tors_forced_margin'][r, b]})")
            br = o["tors_best_robust"][r, b]
            if np.isfinite(br) and o["tors_forced"][r, b] < br - NOISE_REL * scale(br):
                rep.fail(f"{where} bond {b}: angle {k} scores {o['tors_forced'][r, b]} < best {br}")
        err = abs(g["restart_score"][r] - o["restart_score"][r]) / scale(o["restart_score"][r])
        rep.replay_max_score_rel = max(rep.replay_max_score_rel, float(err))
        if err > SCORE_REL:
            rep.fail(f"{where}: score {g['restart_score'][r]} vs replay {o['restart_score'][r]}")
        if o["clash_margin"][r] > CLASH_EPS and g["restart_clash"][r] != o["clash"][r]:
            rep.fail(f"{where}: clash {g['restart_clash'][r]} != replay {o['clash'][r]}")
    # best restart: the GPU's pick scores within tolerance of the best replayed restart, and its
    # reported pose is the replayed pose of that restart
    rs = o["restart_score"]
    br = g["best_restart"]
    if rs[br] < rs.max() - SCORE_REL * scale(rs.max()):
        rep.fail(f"ligand {lig}: best restart {br} ({rs[br]}) below replay best {rs.max()}")
    if abs(g["score"] - g["restart_score"][br]) != 0:
        rep.fail(f"ligand {lig}: score {g['score']} != restart_score[{br}] {g['restart_score'][br]}")
    if g["clash"] != g["restart_clash"][br]:
        rep.fail(f"ligand {lig}: clash {g['clash']} != restart_clash[{br}]")
    d = np.sqrt(np.mean(np.sum((g["xyz"] - o["restart_xyz"][br]) ** 2, axis=1)))
    rep.replay_max_rmsd = max(rep.replay_max_rmsd, float(d))
    if d > RMSD_TOL:
        rep.fail(f"ligand {lig}: best pose RMSD vs replay {d}")


def int_trajectory_comparable(o, r, post_align):
    if o["align_robust"][r] != 1 or (post_align and o["post_robust"][r] != 1):
        return False
    B = o["torsion_idx"].shape[1] if o["torsion_idx"].ndim == 2 else 0
    if B and (o["tors_robust"][r] != 1).any():
        return False
    return o["score_lo"][r] == o["score_hi"][r]


def compare_direct_int(g, o, R, post_align, rep: Report, lig):
    for r in range(R):
        rep.trajectories += 1
        if not int_trajectory_comparable(o, r, post_align):
            continue
        rep.comparable += 1
        rep.comparable_1e4 += 1
        where = f"ligand {lig} restart {r}"
        for k, ok in [("align_idx", g["align_idx"][r] == o["align_idx"][r]),
                      ("post_idx", g["post_idx"][r] == o["post_idx"][r]),
                      ("torsion_idx", np.array_equal(g["torsion_idx"][r], o["torsion_idx"][r])),
                      ("rejected", np.array_equal(g["rejected"][r], o["rejected"][r])),
                      ("score", g["restart_score"][r] == o["restart_score"][r])]:
            if not ok:
                rep.fail(f"{where}: {k} differs (GPU {g[k if k != 'score' else 'restart_score'][r]})")
        err = abs(g["restart_score"][r] - o["restart_score"][r]) / scale(o["restart_score"][r])
        rep.max_score_rel = max(rep.max_score_rel, float(err))
        if o["clash_margin"][r] > CLASH_EPS and g["restart_clash"][r] != o["clash"][r]:
            rep.fail(f"{where}: clash {g['restart_clash'][r]} != {o['clash'][r]}")


def compare_best_int(g, o, o_rep, R, post_align, rep: Report, lig):
    """Integer grid: the oracle's best restart r* followed a trajectory with only possible decisions
    and one possible score, and that score beats the highest possible score of every restart the GPU
    docked (their replays), or equals it for a later restart (ties go to the lowest restart); the
    GPU must then pick r* and report the oracle's pose of it."""
    rb = int(o["best_restart"])
    if not int_trajectory_comparable(o, rb, post_align):
        return
    top = float(o["restart_score"][rb])
    for r in range(R):
        if r != rb and not (top > o_rep["score_hi"][r] or (top >= o_rep["score_hi"][r] and rb < r)):
            return
    rep.ligands_comparable += 1
    if g["best_restart"] != rb:
        rep.fail(f"ligand {lig}: best_restart {g['best_restart']} != {rb}")
        return
    d = np.sqrt(np.mean(np.sum((g["xyz"] - o["restart_xyz"][rb]) ** 2, axis=1)))
    rep.max_rmsd = max(rep.max_rmsd, float(d))
    if d > RMSD_TOL:
        rep.fail(f"ligand {lig}: best pose RMSD {d}")


def compare_replay_int(g, o, R, A, post_align, rep: Report, lig):
    """`o` is the oracle run forced with the GPU's decisions on an integer grid.  A decision whose
    only possible choice in the replayed state is the oracle's (robust) counts as compared exactly:
    the GPU's choice is then possible only if it is that one."""
    B = g["torsion_idx"].shape[1]
    for r in range(R):
        rep.decisions += 1 + bool(post_align) + B
        rep.decisions_exact += int(o["align_robust"][r] == 1) + int(bool(post_align) and o["post_robust"][r] == 1)
        for b in range(B):
            rep.decisions_exact += int(o["tors_robust"][r, b] == 1)
            if int(o["tors_ambiguous"][r, b]) == 0:
                rep.rejected_exact += 1
                if int(g["rejected"][r, b]) != int(o["rejected"][r, b]):
                    rep.fail(f"ligand {lig} restart {r} bond {b}: rejected {g['rejected'][r, b]} != "
                             f"{o['rejected'][r, b]}")
        rep.clash_exact += int(o["clash_margin"][r] > CLASH_EPS)
    for r in range(R):
        where = f"ligand {lig} restart {r} (replay)"
        if o["align_possible"][r] != 1:
            rep.fail(f"{where}: alignment {g['align_idx'][r]} is not a possible choice")
        if post_align and o["post_possible"][r] != 1:
            rep.fail(f"{where}: post alignment {g['post_idx'][r]} is not a possible choice")
        B = g["torsion_idx"].shape[1]
        for b in range(B):
            rej, amb = int(g["rejected"][r, b]), int(o["tors_ambiguous"][r, b])
            if abs(rej - int(o["rejected"][r, b])) > amb:
                rep.fail(f"{where} bond {b}: rejected {rej} vs {o['rejected'][r, b]} (+-{amb})")
            if o["tors_possible"][r, b] != 1:
                rep.fail(f"{where} bond {b}: angle {g['torsion_idx'][r, b]} is not a possible choice")
        s = g["restart_score"][r]
        if not (o["score_lo"][r] <= s <= o["score_hi"][r]):
            rep.fail(f"{where}: score {s} outside replay range [{o['score_lo'][r]}, {o['score_hi'][r]}]")
        rep.replay_max_score_rel = max(rep.replay_max_score_rel,
                                       float(abs(s - o["restart_score"][r]) / scale(o["restart_score"][r])))
        if o["clash_margin"][r] > CLASH_EPS and g["restart_clash"][r] != o["clash"][r]:
            rep.fail(f"{where}: clash {g['restart_clash'][r]} != replay {o['clash'][r]}")
    rs = g["restart_score"]
    br = g["best_restart"]
    if br != int(np.argmax(rs)):
        rep.fail(f"ligand {lig}: best restart {br} is not the first maximum of the GPU's exact scores")
    if g["score"] != rs[br] or g["clash"] != g["restart_clash"][br]:
        rep.fail(f"ligand {lig}: score / clash not those of restart {br}")
    d = np.sqrt(np.mean(np.sum((g["xyz"] - o["restart_xyz"][br]) ** 2, axis=1)))
    rep.replay_max_rmsd = max(rep.replay_max_rmsd, float(d))
    if d > RMSD_TOL:
        rep.fail(f"ligand {lig}: best pose RMSD vs replay {d}")


def check(oracle, grid_view, db, gpu_res, p, indices=None, threads=None) -> Report:
    """Direct and replay comparison of GPU results for the ligands in `indices` (default all).

    ``p`` is an ``oracle.Params`` matching the GPU run.
    """
    idx = list(range(db.n_lig)) if indices is None else [int(i) for i in indices]
    threads = threads or os.cpu_count() or 8
    R, A = p.restarts, p.torsion_steps
    g_all = gpu_split(gpu_res, db, R)
    free = oracle.dock_db(grid_view, db, p, threads=threads, indices=idx)
    forced = {"align": {}, "post": {}, "tors": {}}
    for l in idx:
        g = g_all[l]
        forced["align"][l] = g["align_idx"]
        forced["post"][l] = g["post_idx"] if p.post_align else np.full(R, -1, np.int32)
        forced["tors"][l] = g["torsion_idx"].reshape(-1)
    replay = oracle.dock_db(grid_view, db, p, threads=threads, indices=idx, forced=forced)
    rep = Report()
    integer = getattr(grid_view, "mode", 0) == 1
    for l, o_free, o_rep in zip(idx, free, replay):
        rep.ligands += 1
        if integer:
            compare_direct_int(g_all[l], o_free, R, p.post_align, rep, l)
            compare_best_int(g_all[l], o_free, o_rep, R, p.post_align, rep, l)
            compare_replay_int(g_all[l], o_rep, R, A, p.post_align, rep, l)
        else:
            compare_direct(g_all[l], o_free, R, p.post_align, rep, l)
            compare_best(g_all[l], o_free, o_rep, R, p.post_align, rep, l)
            compare_replay(g_all[l], o_rep, R, A, p.post_align, rep, l)
    return rep
