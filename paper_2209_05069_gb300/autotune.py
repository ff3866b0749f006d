"""Per-bucket launch-shape autotuner for the docking kernel.

For every atom bucket that a sample database fills, the tuner docks that bucket's ligands with each
candidate launch shape (warps per block x preferred shared-memory carveout x persistent form x
warps per ligand-restart x pose tile, the alignment poses and torsion angles one lane scores per
pass), keeps the fastest and applies it to the context (``dock_set_launch``).  Warps per item G and
the pose tile T together set the angle tile, the angles of a bond one ligand-restart has in flight:
32 x G x T.
Launch shapes change speed only: results are identical under every shape (the warps of an item
form every floating-point sum in the same order whatever their number).  The carveout trades resident
blocks against L1 capacity, which matters because the pocket lookups are gathered through L1.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import dock

WARPS = (2, 4, 8)
CARVEOUTS = (-1, 60)
PERSISTENT = (0, 1)
WARPS_PER_ITEM = (1, 2, 4)
TILES = (1, 2)


def _valid(wpb, gi, tile):
    """A shape exists if G divides the block's warps and a tile of 2 goes with 1 or 2 warps per item."""
    return wpb % gi == 0 and (tile == 1 or gi <= 2)


def bucket_of(n_atoms):
    return (np.asarray(n_atoms) - 1) // 32


def tune(ctx: "dock.Context", pocket_id: int, db, params: "dock.Params", warps=WARPS, carveouts=CARVEOUTS,
         persistent=PERSISTENT, warps_per_item=WARPS_PER_ITEM, reps: int = 3, max_ligands: int = 1500,
         joint: bool = True, log=None, tiles=TILES) -> dict:
    """Tunes every bucket present in ``db`` (up to ``max_ligands`` of it) and applies the winners.

    Shapes whose warps per item do not divide warps per block, or with a tile of 2 and more than 2
    warps per item, are skipped.  With ``joint`` the per-bucket winners are then checked against a
    few shapes common to all buckets with the buckets running side by side (see _joint).  Returns
    {bucket: {"warps_per_block", "smem_carveout", "persistent", "warps_per_item", "pose_tile", "ms",
    "ligands", "tried"[, "joint"]}}.
    """
    n = np.diff(db.atom_off)
    table = {}
    samples = []
    for b in range(5):
        idx = np.flatnonzero(bucket_of(n) == b)[:max_ligands]
        if idx.size == 0:
            continue
        batch = ctx.batch_create(db.subset(idx), params)
        tried = []
        try:
            shapes = [(w, c, q, gi, t) for w in warps for c in carveouts for q in persistent for gi in warps_per_item
                      for t in tiles if _valid(w, gi, t)]
            for wpb, cv, ps, gi, tl in shapes:
                ctx.set_launch(b, wpb, cv, ps, gi, tl)
                ctx.batch_launch(pocket_id, batch)   # first launch captures the graph
                ctx.batch_wait(batch)
                best = float("inf")
                for _ in range(reps):
                    t0 = time.perf_counter()
                    ctx.batch_launch(pocket_id, batch)
                    ctx.batch_wait(batch)
                    best = min(best, (time.perf_counter() - t0) * 1e3)
                tried.append((wpb, cv, ps, gi, tl, best))
                if log:
                    log(f"bucket {b}: warps/block {wpb} carveout {cv} persistent {ps} warps/item {gi} tile {tl}: "
                        f"{best:.3f} ms")
        finally:
            ctx.batch_destroy(batch)
        wpb, cv, ps, gi, tl, ms = min(tried, key=lambda t: t[5])
        ctx.set_launch(b, wpb, cv, ps, gi, tl)
        table[b] = {"warps_per_block": wpb, "smem_carveout": cv, "persistent": ps, "warps_per_item": gi,
                    "pose_tile": tl, "ms": ms, "ligands": int(idx.size),
                    "tried": [[w, c, q, g_, t_, round(t, 4)] for w, c, q, g_, t_, t in tried]}
        samples.append(idx)
    if joint and len(table) > 1:
        _joint(ctx, pocket_id, db, params, table, np.concatenate(samples), reps, log)
    return table


def _joint(ctx, pocket_id, db, params, table, idx, reps, log):
    """The buckets of a batch run side by side, so each bucket's fastest shape alone need not be
    the fastest set.  Times the per-bucket winners against the few shapes that did best summed over
    all buckets, each applied to every bucket, and against the library defaults, on the buckets'
    samples docked together; keeps the fastest set."""
    tried = {b: {tuple(t[:5]): t[5] for t in row["tried"]} for b, row in table.items()}
    common = set.intersection(*(set(d) for d in tried.values()))
    ranked = sorted(common, key=lambda sh: sum(tried[b][sh] for b in tried))[:3]
    sets = [("per bucket", {b: _shape(r) for b, r in table.items()})]
    sets += [(f"all {sh}", {b: sh for b in table}) for sh in ranked]
    sets.append(("library default", _defaults(ctx, table)))
    batch = ctx.batch_create(db.subset(idx), params)
    results = []
    try:
        for name, shapes in sets:
            for b, sh in shapes.items():
                ctx.set_launch(b, *sh)
            ctx.batch_launch(pocket_id, batch)
            ctx.batch_wait(batch)
            best = float("inf")
            for _ in range(reps):
                t0 = time.perf_counter()
                ctx.batch_launch(pocket_id, batch)
                ctx.batch_wait(batch)
                best = min(best, (time.perf_counter() - t0) * 1e3)
            results.append((best, name, shapes))
            if log:
                log(f"together, {name}: {best:.3f} ms")
    finally:
        ctx.batch_destroy(batch)
    best, name, shapes = min(results, key=lambda t: t[0])
    for b, sh in shapes.items():
        ctx.set_launch(b, *sh)
        row = table[b]
        _set_shape(row, sh)
        row["joint"] = {"chosen": name, "ms": round(best, 4), "tried": [[n_, round(t, 4)] for t, n_, _ in results]}


def _shape(row):
    """(warps per block, carveout, persistent, warps per item, pose tile) of a table row."""
    return (row["warps_per_block"], row["smem_carveout"], row["persistent"], row["warps_per_item"],
            row.get("pose_tile", 1))


def _set_shape(row, sh):
    row["warps_per_block"], row["smem_carveout"], row["persistent"], row["warps_per_item"], row["pose_tile"] = sh


def _defaults(ctx, buckets):
    """The library's default launch shape of each bucket (what dock_set_launch with NULL restores)."""
    out = {}
    for b in buckets:
        ctx.reset_launch(b)
        g = ctx.get_launch(b)
        out[b] = (g["warps_per_block"], g["smem_carveout_pct"], g["persistent"], g["warps_per_item"], g["pose_tile"])
    return out


def _time_batch(ctx, pocket_id, batch, reps):
    ctx.batch_launch(pocket_id, batch)
    ctx.batch_wait(batch)
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        ctx.batch_launch(pocket_id, batch)
        ctx.batch_wait(batch)
        best = min(best, (time.perf_counter() - t0) * 1e3)
    return best


def confirm(ctx: "dock.Context", pocket_id: int, db, params: "dock.Params", table: dict, reps: int = 3,
            log=None) -> dict:
    """Docks the whole of ``db`` with the tuned table and with the library defaults and keeps the
    faster (the tuner times samples of at most a few thousand ligands per bucket, whose balance
    can differ from the whole database's).  Records both times in every row under "confirm"."""
    if not table:
        return table
    tuned = {b: _shape(r) for b, r in table.items()}
    batch = ctx.batch_create(db, params)
    try:
        apply(ctx, table)
        t_tuned = _time_batch(ctx, pocket_id, batch, reps)
        defaults = _defaults(ctx, table)
        t_default = _time_batch(ctx, pocket_id, batch, reps)
    finally:
        ctx.batch_destroy(batch)
    shapes, chosen = (tuned, "tuned") if t_tuned <= t_default else (defaults, "library default")
    if log:
        log(f"whole database: tuned {t_tuned:.3f} ms, library default {t_default:.3f} ms -> {chosen}")
    for b, sh in shapes.items():
        ctx.set_launch(b, *sh)
        row = table[b]
        _set_shape(row, sh)
        row["confirm"] = {"chosen": chosen, "tuned_ms": round(t_tuned, 4), "default_ms": round(t_default, 4),
                          "ligands": int(db.n_lig)}
    return table


def apply(ctx: "dock.Context", table: dict):
    """Applies a table produced by :func:`tune` (e.g. loaded from JSON)."""
    for b, row in table.items():
        ctx.set_launch(int(b), int(row["warps_per_block"]), int(row["smem_carveout"]), int(row.get("persistent", 0)),
                       int(row.get("warps_per_item", 1)), int(row.get("pose_tile", 1)))


def save(table: dict, path: str, **meta):
    with open(path, "w") as f:
        json.dump({"meta": meta, "buckets": {str(k): v for k, v in table.items()}}, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        return {int(k): v for k, v in json.load(f)["buckets"].items()}
