#!/usr/bin/env python
"""Docking throughput benchmark: docked ligands/s on GB300 (batched form), with end-to-end,
per-ligand-form, roofline and CPU-oracle figures.  Prints one JSON line (rank 0).

Workload (default): the seeded uneven database of 10,000 synthetic ligands (atom counts
log-normal, median 35, clipped to 10-80; rotatable bonds Poisson(6) clipped to 0-20) docked into a
64^3 FP32 pocket grid at 0.375 A with 30 restarts, 30x30 rigid-alignment angles (12 degree steps,
Alg. 1), 256 torsion angles per rotatable bond, bump threshold 2.0 A, post-alignment on.

A step docks the whole database once: one launch of the fused kernel per non-empty atom bucket,
back to back on one stream, inputs already in device memory.  L2 is flushed (a 256 MiB write)
before every timed step, outside the step's events.  Under torchrun every rank docks its own
database of the same recipe (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "docked ligands/sec on 1 GB300 (batched/served vs per-ligand form); p50/p99 ligand latency"
UNIT = "ligands/s"
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3
# FP32 operations of one pocket lookup: rotation into grid coordinates (9 multiply-adds in the
# alignment, 6 in the torsion sweep, 3 scale-shifts for the final pose), 3 fractional parts,
# 7 linear interpolations (a subtract and a multiply-add each), 1 accumulate.
FLOPS_ALIGN, FLOPS_TORSION, FLOPS_FINAL = 18 + 3 + 21 + 1, 12 + 3 + 21 + 1, 6 + 3 + 21 + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven")
    ap.add_argument("--n-lig", type=int, default=0, help="ligands per rank (default: the workload's)")
    ap.add_argument("--grid-dtype", default="", choices=["", "f32", "f16", "i16"],
                    help="f32/f16: trilinear grid; i16: integer grid (round(1000 x value), nearest voxel)")
    ap.add_argument("--per-ligand-sample", type=int, default=200)
    ap.add_argument("--cpu-sample", type=int, default=2048, help="ligands the oracle docks for cpu_baseline")
    ap.add_argument("--select-k", type=int, default=1, help="Select Poses: poses kept per ligand")
    ap.add_argument("--select-rmsd", type=float, default=2.0, help="Select Poses: RMSD threshold (A)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="0 skips the serving measurement")
    ap.add_argument("--serve-warmup", type=float, default=1.0)
    ap.add_argument("--serve-rate", type=float, default=50_000.0, help="offered load, ligands/s (Poisson)")
    ap.add_argument("--serve-pockets", type=int, default=4)
    ap.add_argument("--serve-streams", type=int, default=4, help="streams of the serving context")
    ap.add_argument("--serve-latency-form", type=int, default=0,
                    help="serving batches of at most this many ligands run in the latency form; 0: the library's "
                         "default (1), -1: never")
    ap.add_argument("--serve-warps-per-item", type=int, default=0,
                    help="warps per ligand-restart for every serving batch; 0: the library's adaptive choice "
                         "(8 for small batches, the default shapes for large ones)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="apply this saved tuning table instead of tuning")
    ap.add_argument("--save-tuning", default="", help="save the tuning table the run used")
    ap.add_argument("--mode", default="bench", choices=["bench", "plateau", "classes", "crossover", "serve"],
                    help="plateau: throughput vs database size (128^3 FP16); crossover: latency form vs per-ligand "
                         "vs batched over database size; serve: the serving measurement alone")
    ap.add_argument("--no-counters", action="store_true", help="skip the counter-build pass of the roofline")
    ap.add_argument("--sizes", default="", help="database sizes of the plateau mode (default 10^2..10^6) or the "
                                                "crossover mode (default 1, 10, ..., 10^4)")
    ap.add_argument("--early-exit", default="both", choices=["both", "1", "0"], help="classes mode: bump early exit")
    ap.add_argument("--forms", default="both", choices=["both", "batched"], help="classes mode: forms to run")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        if enabled:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            try:
                self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "200"],
                                             stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            except OSError:
                self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        self.proc.wait(timeout=10)
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload_db(w, n_lig, rank):
    from paper_2209_05069_gb300 import synth
    n = n_lig or w.n_lig
    k = synth.default_workers()
    if rank == 0:
        return synth.make_db(w, n, workers=k)
    return synth.make_db(w, n, seed=synth.ligand_seed(w) + 1000 * rank, first_id=rank * n, workers=k)


def best_outputs(dock, prm):
    """The same parameters with only the per-ligand outputs copied back (what a screening client
    reads: scores, poses, clash counts); the serving and end-to-end measurements use these."""
    q = dock.Params.from_buffer_copy(prm)
    q.outputs = dock.DOCK_OUTPUT_BEST
    return q


def params_for(w, dock, args=None):
    return dock.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                            clash_dist=w.clash_dist, post_align=1, early_exit=1, seed=2209,
                            select_k=getattr(args, "select_k", 1), select_rmsd=getattr(args, "select_rmsd", 2.0))


def kernel_source_sha1(path):
    """SHA-1 of the kernel source with comments and blank lines removed, so that a capture stays
    valid across edits that change no code."""
    import hashlib
    import re
    src = open(path).read()
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(l.rstrip() for l in src.splitlines() if l.strip())
    return hashlib.sha1(code.encode()).hexdigest()


def committed_traffic(grid_dtype, n_lig):
    """DRAM bytes per step from the committed ncu capture, if it was taken on the current kernel."""
    prof = os.path.join(ROOT, "profiles", "dock_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2209_05069_gb300", "csrc", "dock_kernels.cuh")
    try:
        rec = json.load(open(prof))
        sha = kernel_source_sha1(src)
    except (OSError, ValueError):
        return None
    r = rec.get("records", {}).get(grid_dtype)
    if rec.get("kernel_source_sha1") != sha or r is None:
        return None
    return r["bytes_per_ligand"] * n_lig


def dominant_kernel(dock, ctx, pid, db, prm, stream, flush, warmup, steps):
    """The bucket kernel with the most lookups, launched alone on the same stream: its algorithmic
    lookups per launch and its mean launch duration (CUDA events around each launch, L2 flushed
    before each one)."""
    import torch
    n = np.diff(db.atom_off)
    best = None
    for b in range(5):
        idx = np.flatnonzero((n - 1) // 32 == b)
        if idx.size == 0:
            continue
        bt = ctx.batch_create(db.subset(idx), prm)
        wk = ctx.batch_work(bt)
        look = wk["lookups_align"] + wk["lookups_torsion"] + wk["lookups_final"]
        if best is None or look > best[1]:
            if best is not None:
                ctx.batch_destroy(best[2])
            best = (b, look, bt, int(idx.size))
        else:
            ctx.batch_destroy(bt)
    b, look, bt, nb = best
    sptr = stream.cuda_stream
    for _ in range(max(warmup, 1)):
        ctx.batch_launch(pid, bt, dock.DOCK_FORM_BATCHED, sptr)
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 0xff)
            e0[k].record(stream)
            ctx.batch_launch(pid, bt, dock.DOCK_FORM_BATCHED, sptr)
            e1[k].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in zip(e0, e1)) / steps
    ctx.batch_destroy(bt)
    return {"bucket": b, "ligands": nb, "lookups_per_launch": look, "ms_per_launch": ms}


def executed_work(dock, local, pk, grid_dtype, db, prm, bucket, tuning):
    """Work the dominant bucket's kernel executes in one launch, counted by the counter build of the
    library (the same sources compiled with DOCK_COUNT_WORK) on the same ligands, parameters and
    launch shapes: lookups evaluated, loads issued, distinct 32-byte sectors read per warp-wide
    load, bump-pair tests.  Counting changes no result (tested)."""
    from paper_2209_05069_gb300 import autotune
    n = np.diff(db.atom_off)
    idx = np.flatnonzero((n - 1) // 32 == bucket)
    with dock.Context(device=local, serve=False, counters=True) as cctx:
        if tuning:
            autotune.apply(cctx, tuning)
        pid = cctx.load(pk, grid_dtype)
        b = cctx.batch_create(db.subset(idx), prm)
        cctx.batch_launch(pid, b, dock.DOCK_FORM_BATCHED)
        cctx.batch_wait(b)
        c = cctx.exec_counters(reset=True)
        cctx.batch_destroy(b)
    return c


def _bucket_and_grid(kernel):
    """(MAXN, grid type) of a docking-kernel name such as dock_kernel<64, 0, 2, 1>."""
    return tuple(x.strip() for x in kernel.split("<", 1)[1].split(",")[:2])


def committed_kernel_traffic(grid_dtype, kernel, db, bucket, n_in_bucket):
    """DRAM bytes of one launch of `kernel` from the committed capture (2,000-ligand prefix of the
    same database), scaled by the bucket's ligand count; None if the capture does not apply."""
    prof = os.path.join(ROOT, "profiles", "dock_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2209_05069_gb300", "csrc", "dock_kernels.cuh")
    try:
        rec = json.load(open(prof))
        sha = kernel_source_sha1(src)
    except (OSError, ValueError):
        return None
    r = rec.get("records", {}).get(grid_dtype)
    if rec.get("kernel_source_sha1") != sha or r is None:
        return None
    per = r.get("per_kernel", {})
    if kernel not in per:   # same bucket and grid type, another launch shape or entry point: same DRAM reads
        same = [k for k in per if _bucket_and_grid(k) == _bucket_and_grid(kernel)]
        if not same:
            return None
        kernel = same[0]
    m = int(rec.get("captured_ligands", 0))
    if db.n_lig < m:
        return None
    n = np.diff(db.atom_off[:m + 1])
    c = int(((n - 1) // 32 == bucket).sum())
    return per[kernel] / c * n_in_bucket if c else None


def pocket_for(w, grid_dtype, p=0):
    """Pocket p of the workload; the integer grid holds round(1000 x value)."""
    from paper_2209_05069_gb300 import synth
    pk = synth.workload_pocket(w, p)
    return pk.integer(1000) if grid_dtype == "i16" else pk


def oracle_grid(w, grid_dtype):
    from oracle import oracle
    return oracle.GridView.of(pocket_for(w, grid_dtype), fp16=grid_dtype == "f16", nearest=grid_dtype == "i16")


def cpu_baseline(w, db, n_sample, threads, grid_dtype):
    """The FP64 oracle, as it stands, over a bounded sample of the workload on host threads."""
    from oracle import oracle
    g = oracle_grid(w, grid_dtype)
    p = oracle.Params(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                      clash_dist=w.clash_dist, post_align=1, seed=2209)
    idx = list(range(min(n_sample, db.n_lig)))
    t0 = time.perf_counter()
    oracle.dock_db(g, db, p, threads=threads, indices=idx)
    dt = time.perf_counter() - t0
    return len(idx) / dt, dt, len(idx)


def serving_run(dock, synth, w, pool, prm, rate, seconds, warmup_s, n_pockets, device, warps_per_item=0, streams=4,
                grid_dtype="f32", seed=2209, latency_form=0):
    """Poisson arrivals of single ligands (drawn cyclically from `pool`, each with a fresh id) naming
    one of `n_pockets` resident pocket grids at random, served by the continuous-batching loop.

    Requests arriving in the same millisecond for the same pocket go in one submission; latency is
    measured per ligand from its scheduled arrival to the moment the serving loop has its result.
    """
    import threading
    import queue
    prm_best = best_outputs(dock, prm)
    n = int(rate * (seconds + warmup_s))
    arrivals = synth.poisson_arrivals(rate, n, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    which = rng.integers(0, n_pockets, size=n)
    # warps_per_item 0: the library's adaptive choice (the latency-oriented shape for small batches,
    # the context's shapes for large ones); n > 0: n warps per ligand-restart for every batch
    ctx = dock.Context(device=device, n_streams=streams, serve_latency_items=-1 if warps_per_item > 0 else 0,
                       serve_latency_form=latency_form)
    if warps_per_item > 0:
        for bucket in range(5):
            ctx.set_launch(bucket, 8, -1, 0, warps_per_item)
    pids = [ctx.load(pocket_for(w, grid_dtype, p), grid_dtype) for p in range(n_pockets)]
    # groups: (tick end time, pocket, request indices, first pool ligand); each pocket's requests
    # take consecutive pool ligands so one submission is one slice of the pool
    P = pool.n_lig
    tick = np.floor(arrivals * 1e3).astype(np.int64)
    bounds = np.flatnonzero(np.diff(tick)) + 1
    groups = []
    nxt = [0] * n_pockets
    for a, b in zip(np.r_[0, bounds], np.r_[bounds, n]):
        for p in range(n_pockets):
            idx = np.flatnonzero(which[a:b] == p) + a
            if idx.size:
                if nxt[p] + idx.size > P:
                    nxt[p] = 0
                groups.append(((tick[a] + 1) * 1e-3, p, idx, nxt[p]))
                nxt[p] += idx.size
    done_q = queue.Queue()
    lat = np.full(n, np.nan)
    lag = np.full(n, np.nan)

    def submitter(t0):
        for t_end, p, idx, first in groups:
            dt = t0 + t_end - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            sub = pool.slice(first, first + idx.size, ids=idx)
            t_sub = time.perf_counter() - t0
            done_q.put((ctx.submit(pids[p], sub, prm_best), idx, t_sub))
        done_q.put(None)

    def collector():
        while True:
            item = done_q.get()
            if item is None:
                return
            ticket, idx, t_sub = item
            ctx.poll(ticket, -1)
            r = ctx.results(ticket, minimal=True)
            lat[idx] = t_sub - arrivals[idx] + r["latency_ns"] * 1e-9
            lag[idx] = t_sub - arrivals[idx]

    # the client's own pauses are not the server's latency: Python's collector stays off while the
    # two client threads run (a collection pass held both threads for tens of ms)
    import gc
    gc_was_on = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        ts = threading.Thread(target=submitter, args=(t0,))
        tc = threading.Thread(target=collector)
        ts.start()
        tc.start()
        ts.join()
        tc.join()
        wall = time.perf_counter() - t0
    finally:
        if gc_was_on:
            gc.enable()
    st = ctx.stats()
    ctx.close()
    keep = arrivals >= warmup_s
    done = arrivals + lat
    slow = np.flatnonzero(keep & (lat > 5e-3))
    slow_arrivals = [round(float(arrivals[i]), 4) for i in slow[:20]]
    served = np.sum((done >= warmup_s) & (done <= warmup_s + seconds))
    L = lat[keep] * 1e3
    return {"offered_rate": rate, "served_rate": float(served / seconds), "p50_ms": float(np.percentile(L, 50)),
            "p99_ms": float(np.percentile(L, 99)), "max_ms": float(L.max()),
            "client_lag_p50_ms": float(np.percentile(lag[keep] * 1e3, 50)),
            "warps_per_item": warps_per_item if warps_per_item > 0 else "adaptive",
            "latency_shape_batches": f"{st['latency_batches']} of {st['batches']}",
            "latency_form_batches": st["latency_form_batches"],
            "latency_form_ligands": latency_form if latency_form else "library default (1)",
            "slot_grows": st["slot_grows"], "client": "Python garbage collector paused during the run",
            "streams": streams,
            "requests": int(keep.sum()),
            "submissions": len(groups), "pockets": n_pockets, "seconds": seconds, "warmup_s": warmup_s,
            "wall_s": wall, "over_5ms": {"requests": int(slow.size), "first_arrivals_s": slow_arrivals}}


def run_plateau(args):
    """Throughput vs database size (the paper's scaling study, Section 5.3): databases of the uneven
    size distribution (a 10,000-ligand pool cycled with fresh ids) docked through one pocket, per
    size: the batched form on resident inputs, the public submit/poll/results path end to end, and
    the plain per-ligand form on a sample."""
    import torch

    from paper_2209_05069_gb300 import autotune, dock, synth
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload if args.workload != "uneven" else "plateau"]
    grid_dtype = args.grid_dtype or w.grid_dtype
    pool = synth.make_db(w, 10_000, workers=synth.default_workers())
    prm = params_for(w, dock, args)
    ctx = dock.Context(device=local)
    pid = ctx.load(pocket_for(w, grid_dtype), grid_dtype)
    tuning = None if args.no_autotune else autotune.tune(ctx, pid, pool.slice(0, 4000), prm)
    stream = torch.cuda.Stream()
    rows = []
    sub = pool.slice(0, min(args.per_ligand_sample or 200, pool.n_lig))
    b = ctx.batch_create(sub, prm)
    ctx.batch_launch(pid, b, dock.DOCK_FORM_PER_LIGAND, stream.cuda_stream)
    stream.synchronize()
    t0 = time.perf_counter()
    ctx.batch_launch(pid, b, dock.DOCK_FORM_PER_LIGAND, stream.cuda_stream)
    stream.synchronize()
    per_lig = sub.n_lig / (time.perf_counter() - t0)
    ctx.batch_destroy(b)
    # one untimed pass through the serving path: its stream slots are allocated on first use
    ctx.dock(pid, pool.slice(0, 100), best_outputs(dock, prm))
    for size in [int(x) for x in (args.sizes or "100,1000,10000,100000,1000000").split(",")]:
        db = synth.tile_db(pool, size, first_id=10_000_000)
        if not args.no_autotune:   # small databases favour more warps per ligand-restart
            tuning = autotune.tune(ctx, pid, db if size <= 4000 else pool.slice(0, 4000), prm,
                                   warps_per_item=(1, 2, 4, 8), reps=1)
        b = ctx.batch_create(db, prm)
        ctx.batch_launch(pid, b, dock.DOCK_FORM_BATCHED, stream.cuda_stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.batch_launch(pid, b, dock.DOCK_FORM_BATCHED, stream.cuda_stream)
        e1.record(stream)
        stream.synchronize()
        batched = size / (e0.elapsed_time(e1) / 1e3)
        ctx.batch_destroy(b)
        t0 = time.perf_counter()
        ctx.dock(pid, db, best_outputs(dock, prm))
        served = size / (time.perf_counter() - t0)
        rows.append({"ligands": size, "batched": batched, "served_e2e": served, "per_ligand": per_lig,
                     "batched_over_per_ligand": batched / per_lig,
                     "launch": {k: [v["warps_per_block"], v["smem_carveout"], v["persistent"], v["warps_per_item"],
                                    v.get("pose_tile", 1)] for k, v in (tuning or {}).items()}})
        print(json.dumps(rows[-1]), flush=True)
    ctx.close()
    print(json.dumps({"mode": "plateau", "workload": w.name, "grid": f"{w.grid}^3 @ {w.spacing} A",
                      "grid_dtype": grid_dtype, "restarts": w.restarts, "torsion_steps": w.torsion_steps,
                      "unit": UNIT, "rows": rows,
                      "launch": {k: [v["warps_per_block"], v["smem_carveout"], v["persistent"], v["warps_per_item"],
                                     v.get("pose_tile", 1)] for k, v in (tuning or {}).items()}}),
          flush=True)
    return 0


# The paper's profiling classes (Section 5.5): atoms (including hydrogens), rotatable bonds and the
# batch one molecule is duplicated to.
CLASSES = {"small": (48, 1, 1920), "medium": (80, 12, 1600), "large": (128, 20, 960)}


def run_classes(args):
    """Small / Medium / Large molecule classes: one synthetic molecule per class duplicated to the
    paper's batch size (fresh ids, so restart orientations differ), docked by the batched and the
    per-ligand form, with the bump-check early exit on and off."""
    import torch

    from paper_2209_05069_gb300 import dock, synth
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    w = synth.WORKLOADS["uneven"]
    ctx = dock.Context(device=local, serve=False)
    pid = ctx.load(pocket_for(w, args.grid_dtype or "f32"), args.grid_dtype or "f32")
    stream = torch.cuda.Stream()
    rows = []
    for name, (n_atoms, n_rot, batch) in CLASSES.items():
        rng = np.random.Generator(np.random.PCG64([synth.BASE_SEED, n_atoms, n_rot]))
        while True:
            xyz, bonds, rot, clipped = synth.make_ligand(rng, n_atoms, n_rot)
            if not clipped:
                break
        one = synth.from_ligands([(xyz, bonds, rot, 0)])
        db = synth.tile_db(one, batch, first_id=1)
        row = {"class": name, "atoms": n_atoms, "rotatable_bonds": n_rot, "batch": batch}
        if not args.no_autotune:   # the class's own launch shape, as the benchmark tunes its database
            from paper_2209_05069_gb300 import autotune
            prm = dock.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                                   clash_dist=w.clash_dist, seed=2209)
            tuned = autotune.tune(ctx, pid, db, prm, reps=1)
            row["launch"] = {str(b): [t["warps_per_block"], t["smem_carveout"], t["persistent"], t["warps_per_item"],
                                      t.get("pose_tile", 1)] for b, t in tuned.items()}
        modes = (1, 0) if args.early_exit == "both" else (int(args.early_exit),)
        forms = ((dock.DOCK_FORM_BATCHED, "batched", db), (dock.DOCK_FORM_PER_LIGAND, "per_ligand", db.slice(0, 64)))
        for ee in modes:
            prm = dock.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                                   clash_dist=w.clash_dist, early_exit=ee, seed=2209)
            for form, label, sub in forms[:1 if args.forms == "batched" else 2]:
                b = ctx.batch_create(sub, prm)
                for _ in range(args.warmup):
                    ctx.batch_launch(pid, b, form, stream.cuda_stream)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.batch_launch(pid, b, form, stream.cuda_stream)
                e1.record(stream)
                stream.synchronize()
                row[f"{label}_early_exit{ee}"] = sub.n_lig / (e0.elapsed_time(e1) / 1e3)
                ctx.batch_destroy(b)
        for ee in modes:
            if args.forms == "both":
                row[f"batched_over_per_ligand_early_exit{ee}"] = (row[f"batched_early_exit{ee}"]
                                                                  / row[f"per_ligand_early_exit{ee}"])
        rows.append(row)
        print(json.dumps(row), flush=True)
    ctx.close()
    print(json.dumps({"mode": "classes", "unit": UNIT, "grid": f"{w.grid}^3 @ {w.spacing} A",
                      "restarts": w.restarts, "torsion_steps": w.torsion_steps, "rows": rows}), flush=True)
    return 0


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores, each step a bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2209_05069_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    threads = os.cpu_count() or 1
    per_step = max(threads * 2, 16)
    db = synth.make_db(w, per_step * (args.steps + args.warmup), workers=synth.default_workers())
    from oracle import oracle
    g = oracle_grid(w, args.grid_dtype or w.grid_dtype)
    p = oracle.Params(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                      clash_dist=w.clash_dist, post_align=1, seed=2209)
    times = []
    for s in range(args.warmup + args.steps):
        idx = list(range(s * per_step, (s + 1) * per_step))
        t0 = time.perf_counter()
        oracle.dock_db(g, db, p, threads=threads, indices=idx)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    sample = f"{per_step} ligands of the {w.name} database per step (full parameters), {threads} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "ligands_per_step": per_step, "restarts": w.restarts,
                       "align_steps": w.align_steps, "torsion_steps": w.torsion_steps, "grid": w.grid},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_crossover(args):
    """Latency form vs batched form over database size (the paper's Section 5.3 comparison of its two
    designs): databases of the uneven size mix (a 10,000-ligand pool cycled with fresh ids) docked
    into the uneven workload's 64^3 FP32 pocket by the latency form (one ligand at a time over the
    whole GPU), the per-ligand form with 8 warps per ligand-restart, and the batched form (launch
    shapes tuned per size); each timed once with CUDA events after one warm-up launch."""
    import torch

    from paper_2209_05069_gb300 import autotune, dock, synth
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    grid_dtype = args.grid_dtype or w.grid_dtype
    pool = synth.make_db(w, 10_000, workers=synth.default_workers())
    prm = params_for(w, dock, args)
    ctx = dock.Context(device=local, serve=False)
    pid = ctx.load(pocket_for(w, grid_dtype), grid_dtype)
    stream = torch.cuda.Stream()

    def timed(b, form):
        ctx.batch_launch(pid, b, form, stream.cuda_stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.batch_launch(pid, b, form, stream.cuda_stream)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    rows = []
    for size in [int(x) for x in (args.sizes or "1,10,100,1000,10000").split(",")]:
        db = synth.tile_db(pool, size, first_id=20_000_000)
        b = ctx.batch_create(db, prm)
        row = {"ligands": size}
        row["latency_form_ms"] = timed(b, dock.DOCK_FORM_LATENCY)
        for k in range(5):
            ctx.set_launch(k, 8, -1, 0, 8)
        row["per_ligand_8_warps_ms"] = timed(b, dock.DOCK_FORM_PER_LIGAND)
        ctx.reset_launch()
        if not args.no_autotune:
            autotune.tune(ctx, pid, db if size <= 4000 else pool.slice(0, 4000), prm, warps_per_item=(1, 2, 4, 8),
                          reps=1)
        row["batched_ms"] = timed(b, dock.DOCK_FORM_BATCHED)
        ctx.reset_launch()
        ctx.batch_destroy(b)
        for k in ("latency_form", "per_ligand_8_warps", "batched"):
            row[f"{k}_ligands_per_s"] = size / (row[f"{k}_ms"] / 1e3)
        row["batched_over_latency_form"] = row["batched_ligands_per_s"] / row["latency_form_ligands_per_s"]
        rows.append(row)
        print(json.dumps(row), flush=True)
    ctx.close()
    print(json.dumps({"mode": "crossover", "workload": w.name, "grid": f"{w.grid}^3 @ {w.spacing} A",
                      "grid_dtype": grid_dtype, "restarts": w.restarts, "torsion_steps": w.torsion_steps,
                      "unit": UNIT, "rows": rows}), flush=True)
    return 0


def run_serve(args):
    """The serving measurement alone (SURVEY config 4 at its stated length with --serve-seconds 60
    --serve-warmup 5): Poisson arrivals over resident pockets, per-ligand latency p50/p99/max."""
    import torch

    from paper_2209_05069_gb300 import dock, synth
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    w = synth.WORKLOADS[args.workload]
    grid_dtype = args.grid_dtype or w.grid_dtype
    db = workload_db(w, args.n_lig, 0)
    prm = params_for(w, dock, args)
    clocks = Clocks(local, enabled=not args.no_clocks)
    serving = serving_run(dock, synth, w, db, prm, args.serve_rate, args.serve_seconds, args.serve_warmup,
                          args.serve_pockets, local, args.serve_warps_per_item, args.serve_streams, grid_dtype,
                          latency_form=args.serve_latency_form)
    print(json.dumps({"mode": "serve", "workload": w.name, "grid_dtype": grid_dtype, "unit": UNIT,
                      "latency": serving, "clocks": clocks.stop()}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "plateau":
        return run_plateau(args)
    if args.mode == "classes":
        return run_classes(args)
    if args.mode == "crossover":
        return run_crossover(args)
    if args.mode == "serve":
        return run_serve(args)
    import torch

    from paper_2209_05069_gb300 import dock, shard, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = synth.WORKLOADS[args.workload]
    grid_dtype = args.grid_dtype or w.grid_dtype
    db = workload_db(w, args.n_lig, rank)
    prm = params_for(w, dock, args)
    pk = pocket_for(w, grid_dtype)
    ctx = dock.Context(device=local)
    pid = ctx.load(pk, grid_dtype)
    gather_peak = ctx.gather_peak(pid)   # lookups/s, the stand-alone roof on this pocket
    tuning = None
    from paper_2209_05069_gb300 import autotune
    if args.tuning:
        tuning = autotune.load(args.tuning)
        autotune.apply(ctx, tuning)
    elif not args.no_autotune:
        tuning = autotune.tune(ctx, pid, db, prm, max_ligands=3000)   # up to 3,000 ligands of each bucket
        tuning = autotune.confirm(ctx, pid, db, prm, tuning)          # vs the library defaults, whole database
    if args.save_tuning and tuning:
        autotune.save(tuning, args.save_tuning, workload=w.name, grid_dtype=grid_dtype)
    batch = ctx.batch_create(db, prm)
    work = ctx.batch_work(batch)
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        ctx.batch_launch(pid, batch, dock.DOCK_FORM_BATCHED, sptr)
    torch.cuda.synchronize()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local, enabled=(rank == 0 and not args.no_clocks))
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            ev0[k].record(stream)
            launches += ctx.batch_launch(pid, batch, dock.DOCK_FORM_BATCHED, sptr)
            ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    dom = dominant_kernel(dock, ctx, pid, db, prm, stream, flush, args.warmup, args.steps) if rank == 0 else None
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = shard.max_over_ranks(sum(step_ms), dist, device="cuda")
    value = world * db.n_lig * args.steps / (total_ms / 1e3)
    res = ctx.batch_results(batch)

    # plain per-ligand form of the same kernels (one launch per ligand) on a sample
    per_lig = None
    if rank == 0 and args.per_ligand_sample > 0:
        sub = db.subset(range(min(args.per_ligand_sample, db.n_lig)))
        b2 = ctx.batch_create(sub, prm)
        ctx.batch_launch(pid, b2, dock.DOCK_FORM_PER_LIGAND, sptr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.batch_launch(pid, b2, dock.DOCK_FORM_PER_LIGAND, sptr)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        per_lig = {"value": sub.n_lig / (ms / 1e3), "unit": UNIT, "sample": f"first {sub.n_lig} ligands",
                   "launches": sub.n_lig}
        # one ligand at a time with 8 warps per ligand-restart (the latency-oriented shape)
        saved = [ctx.get_launch(k) for k in range(5)]
        for k in range(5):
            ctx.set_launch(k, 8, -1, 0, 8)
        ctx.batch_launch(pid, b2, dock.DOCK_FORM_PER_LIGAND, sptr)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.batch_launch(pid, b2, dock.DOCK_FORM_PER_LIGAND, sptr)
        e1.record(stream)
        torch.cuda.synchronize()
        ms8 = e0.elapsed_time(e1)
        for k, sh in enumerate(saved):
            ctx.set_launch(k, sh["warps_per_block"], sh["smem_carveout_pct"], sh["persistent"], sh["warps_per_item"],
                           sh["pose_tile"])
        per_lig["ms_per_ligand"] = ms / sub.n_lig
        per_lig["ms_per_ligand_8_warps_per_item"] = ms8 / sub.n_lig
        # the latency form (one ligand at a time over the whole GPU), ligand after ligand
        ctx.batch_launch(pid, b2, dock.DOCK_FORM_LATENCY, sptr)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.batch_launch(pid, b2, dock.DOCK_FORM_LATENCY, sptr)
        e1.record(stream)
        torch.cuda.synchronize()
        per_lig["ms_per_ligand_latency_form"] = e0.elapsed_time(e1) / sub.n_lig
        per_lig["latency_form_over_8_warps_per_item"] = ms8 / e0.elapsed_time(e1)
        ctx.batch_destroy(b2)

    # end to end through the public API: submit (host buffers) -> poll -> results
    e2e = None
    if not args.no_e2e:
        prm_best = best_outputs(dock, prm)
        st0 = ctx.stats()
        e2e_times = []
        chunks = [db.slice(a, b) for a, b in zip(np.linspace(0, db.n_lig, 5).astype(int)[:-1],
                                                  np.linspace(0, db.n_lig, 5).astype(int)[1:])]
        for k in range(args.warmup + args.steps):
            barrier()
            t0 = time.perf_counter()
            tickets = [ctx.submit(pid, c, prm_best) for c in chunks]   # a client streaming 4 submissions
            parts = []
            for t in tickets:
                ctx.poll(t, -1)
                parts.append(ctx.results(t))
            dt = time.perf_counter() - t0
            r2 = {"score": np.concatenate([p_["score"] for p_ in parts])}
            if k >= args.warmup:
                e2e_times.append(dt)
        st1 = ctx.stats()
        n_steps = args.warmup + args.steps
        e2e_total = shard.max_over_ranks(sum(e2e_times), dist, device="cuda")
        assert np.array_equal(r2["score"], res["score"]), "served results differ from the batch results"
        e2e = {"value": world * db.n_lig * args.steps / e2e_total, "unit": UNIT,
               "h2d_bytes_per_step": (st1["h2d_bytes"] - st0["h2d_bytes"]) // n_steps,
               "d2h_bytes_per_step": (st1["d2h_bytes"] - st0["d2h_bytes"]) // n_steps,
               "outputs": "per-ligand (score, best restart, pose, clash count, Select Poses): DOCK_OUTPUT_BEST",
               "ms_per_step": 1e3 * e2e_total / args.steps}

    serving = None
    if args.serve_seconds > 0 and rank == 0:
        serving = serving_run(dock, synth, w, db, prm, args.serve_rate, args.serve_seconds, args.serve_warmup,
                              args.serve_pockets, local, args.serve_warps_per_item, args.serve_streams, grid_dtype,
                              latency_form=args.serve_latency_form)

    if rank != 0:
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    lookups = work["lookups_align"] + work["lookups_torsion"] + work["lookups_final"]
    flops = (FLOPS_ALIGN * work["lookups_align"] + FLOPS_TORSION * work["lookups_torsion"]
             + FLOPS_FINAL * work["lookups_final"])
    mean_s = (sum(step_ms) / len(step_ms)) / 1e3
    alu = flops / mean_s / 1e12
    bytes_per_lookup = {"f16": 16, "i16": 2}.get(grid_dtype, 32)
    gt = {"f16": 1, "i16": 2}.get(grid_dtype, 0)
    sh = ctx.get_launch(dom["bucket"])
    entry = "dock_kernel_wide" if gt == 0 and sh["warps_per_item"] == 1 else "dock_kernel"
    kernel = f"{entry}<{32 * (dom['bucket'] + 1)}, {gt}, {sh['warps_per_item']}, {sh['pose_tile']}>"
    launch_s = dom["ms_per_launch"] / 1e3
    # the L1 data pipe's roof at the SM clock measured during the timed steps: one wavefront per SM
    # per clock, and a scattered 32-byte sector (one FP32 corner-packed cell) takes one wavefront
    sm_ghz = (clk["sm_mhz"] / 1e3) if clk and clk.get("sm_mhz") else SM_MAX_GHZ
    peak_gbs = SM_COUNT * sm_ghz * 32
    algo_gbs = dom["lookups_per_launch"] * bytes_per_lookup / launch_s / 1e9
    executed = None if args.no_counters else executed_work(dock, local, pk, grid_dtype, db, prm, dom["bucket"], tuning)
    scattered_gbs = gather_peak * bytes_per_lookup / 1e9
    path_gbs = lookups * bytes_per_lookup / mean_s / 1e9
    if executed:
        achieved = executed["sectors"] * 32 / launch_s / 1e9
        frac_note = ("executed: the launch's distinct 32-byte sectors (counted per warp-wide load by the counter "
                     "build on the same ligands and shapes) x 32 B / mean launch time.  The model (one data-pipe "
                     "wavefront per sector) fits scattered 32-byte cells (FP32; ncu's data-pipe utilisation on this "
                     "kernel agrees); on FP16 and int16 grids neighbouring lanes share lines, a wavefront serves "
                     "several sectors, the figure can exceed 1 and those kernels are issue-bound (see profiles)")
    else:
        achieved = algo_gbs
        frac_note = "algorithmic lookups x bytes per lookup / mean launch time (no counter pass)"
    roofline = {"bound": "l1tex", "kernel": kernel, "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs, "achieved_source": frac_note,
                "traffic": committed_kernel_traffic(grid_dtype, kernel, db, dom["bucket"], dom["ligands"]),
                "peak_source": f"derived: L1 data pipe, one 32-byte sector (wavefront) per SM per clock, "
                               f"{SM_COUNT} SMs x {sm_ghz:.3f} GHz (median SM clock of the timed steps) x 32 B",
                "launch_ms": dom["ms_per_launch"], "launch_ligands": dom["ligands"],
                "executed": dict(executed, loads_per_lookup=executed["loads"] / max(executed["lookups"], 1),
                                 sectors_per_load=executed["sectors"] / max(executed["loads"], 1),
                                 lines_per_load=executed["lines"] / max(executed["loads"], 1),
                                 lookups_per_s=executed["lookups"] / launch_s,
                                 sectors_per_s=executed["sectors"] / launch_s,
                                 line_frac=executed["lines"] / launch_s / (SM_COUNT * sm_ghz * 1e9))
                if executed else None,
                "algorithmic": {"lookups_per_launch": dom["lookups_per_launch"], "bytes_per_lookup": bytes_per_lookup,
                                "achieved": algo_gbs, "frac": algo_gbs / peak_gbs,
                                "note": "every angle of every bond scored, every lookup one cell of bytes_per_lookup"},
                "scattered_gather": {"achieved": scattered_gbs, "lookups_per_s": gather_peak,
                                     "algorithmic_over_scattered": algo_gbs / scattered_gbs,
                                     "source": "measured in this run by dock_gather_peak: the same lookups at "
                                               "independent random positions in the pocket's nonzero box, no "
                                               "other work (no locality between lanes)"},
                "path": {"lookups_per_step": lookups, "lookups_per_s": lookups / mean_s, "achieved": path_gbs,
                         "traffic_per_step": committed_traffic(grid_dtype, db.n_lig),
                         "note": "algorithmic; all bucket kernels of a step running side by side"},
                "alu": {"achieved": alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": alu / FP32_PEAK_TFLOPS,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz; algorithmic FLOPs"}}

    cpu = None
    if not args.no_cpu:
        threads = os.cpu_count() or 1
        v, dt, n = cpu_baseline(w, db, args.cpu_sample, threads, grid_dtype)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {n} ligands of the {w.name} database at full parameters ({dt:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{w.name}: {db.n_lig} ligands/rank, atoms {w.atoms}, rotatable bonds {w.rot}",
                   "ligands_per_rank": db.n_lig, "restarts": w.restarts, "align_steps": w.align_steps,
                   "torsion_steps": w.torsion_steps, "grid": f"{w.grid}^3 @ {w.spacing} A", "grid_dtype": grid_dtype,
                   "select_poses": {"k": prm.k, "rmsd": prm.select_rmsd},
                   "l2": "flushed before each timed step (256 MiB write)", "parallelism": f"ligand shards x{world}",
                   "launch": {b: [t["warps_per_block"], t["smem_carveout"], t["persistent"], t["warps_per_item"],
                                  t.get("pose_tile", 1)] for b, t in tuning.items()}
                   if tuning else "default (8 warps/block, driver carveout, persistent, 2 warps per item, tile 1)",
                   "launch_fields": "warps per block, carveout %, persistent, warps per item, pose tile"},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
        "per_ligand_form": per_lig, "latency": serving,
        "batched_over_per_ligand": (value / world / per_lig["value"]) if per_lig else None,
        "step_ms": step_ms,
    }
    print(json.dumps(line), flush=True)
    ctx.batch_destroy(batch)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
