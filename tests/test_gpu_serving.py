"""Continuous-batching serving loop (dock_submit_ligands / dock_poll / dock_results) on the GPU.

Each ligand is docked by its own warps, so a result must not depend on which other ligands (of
which submissions, sizes or pockets) share its batch: results are compared bit for bit.
"""
import threading

import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

pytestmark = pytest.mark.gpu

KEYS = ["score", "best_restart", "xyz", "clash_count", "restart_score", "restart_clash", "align_idx", "post_idx",
        "torsion_idx", "rejected"]


@pytest.fixture(scope="module")
def dk():
    from paper_2209_05069_gb300 import dock
    return dock


def params(dk, seed=3):
    return dk.Params.make(restarts=8, align_steps=30, torsion_steps=64, clash_dist=2.0, seed=seed)


def batch_results(ctx, pid, db, prm):
    b = ctx.batch_create(db, prm)
    ctx.batch_launch(pid, b)
    r = ctx.batch_results(b)
    ctx.batch_destroy(b)
    return r


def per_ligand(res, db, R):
    """Splits flat result arrays into one dict per ligand."""
    out = []
    for l in range(db.n_lig):
        a0, a1, r0, r1 = db.atom_off[l], db.atom_off[l + 1], db.rot_off[l], db.rot_off[l + 1]
        out.append({"score": res["score"][l], "best_restart": res["best_restart"][l], "xyz": res["xyz"][a0:a1],
                    "clash_count": res["clash_count"][l], "restart_score": res["restart_score"][l * R:(l + 1) * R],
                    "restart_clash": res["restart_clash"][l * R:(l + 1) * R],
                    "align_idx": res["align_idx"][l * R:(l + 1) * R], "post_idx": res["post_idx"][l * R:(l + 1) * R],
                    "torsion_idx": res["torsion_idx"][r0 * R:r1 * R], "rejected": res["rejected"][r0 * R:r1 * R]})
    return out


def assert_same(a, b):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_served_results_equal_batch_results(dk):
    w = synth.WORKLOADS["tiny"]
    db = synth.make_db(w)
    prm = params(dk)
    with dk.Context() as ctx:
        pid = ctx.load(synth.workload_pocket(w))
        ref = batch_results(ctx, pid, db, prm)
        got = ctx.dock(pid, db, prm)
        st = ctx.stats()
    assert_same(ref, got)
    assert (got["latency_ns"] > 0).all()
    # host stage timers: the batch and the submission were prepared, one serving batch was
    # staged and scattered, and its slot grew once from empty
    assert st["prep_ns"] > 0 and st["fill_ns"] > 0 and st["scatter_ns"] > 0
    assert st["slot_grows"] == 1 and st["ligands_done"] == 2 * db.n_lig


def test_result_alone_equals_result_in_a_mix(dk):
    """Ligands docked alone match the same ligands docked while other submissions (other sizes,
    other pockets, many small tickets) share the GPU and the batches."""
    tiny, uneven = synth.WORKLOADS["tiny"], synth.WORKLOADS["uneven"]
    target = synth.make_db(tiny, 12, seed=77)
    others = synth.make_db(uneven, 300, seed=78)
    prm = params(dk, seed=5)
    with dk.Context(n_streams=1) as ctx:
        pid = ctx.load(synth.workload_pocket(tiny))
        alone = ctx.dock(pid, target, prm)
    with dk.Context(n_streams=4, max_batch_ligands=64) as ctx:
        pids = [ctx.load(synth.workload_pocket(uneven, p)) for p in range(3)]
        pid = ctx.load(synth.workload_pocket(tiny))
        tickets = []
        for i in range(30):   # interleave: 10-ligand tickets of the other database, then one target ligand
            lo = 10 * i
            tickets.append(("o", ctx.submit(pids[i % 3], others.slice(lo, lo + 10), prm)))
            if i < target.n_lig:
                tickets.append((i, ctx.submit(pid, target.slice(i, i + 1), prm)))
        mixed = {}
        for tag, t in tickets:
            rc, _ = ctx.poll(t, 60_000)
            assert rc == dk.DOCK_OK
            r = ctx.results(t)
            if tag != "o":
                mixed[tag] = r
        st = ctx.stats()
        assert st["batches"] > 1
    alone_l = per_ligand(alone, target, prm.restarts)
    for i in range(target.n_lig):
        assert_same(alone_l[i], per_ligand(mixed[i], target.slice(i, i + 1), prm.restarts)[0])


def test_concurrent_submitters_and_small_budget(dk):
    """Four host threads submit single ligands while a small device budget forces many batches."""
    w = synth.WORKLOADS["tiny"]
    db = synth.make_db(w, 64, seed=90)
    prm = params(dk, seed=9)
    with dk.Context(serve=False) as c0:
        pid0 = c0.load(synth.workload_pocket(w))
        ref = per_ligand(batch_results(c0, pid0, db, prm), db, prm.restarts)
    with dk.Context(n_streams=3, hbm_budget_bytes=3 << 20, max_batch_ligands=16) as ctx:
        pid = ctx.load(synth.workload_pocket(w))
        out = {}
        lock = threading.Lock()

        def worker(k):
            for l in range(k, db.n_lig, 4):
                t = ctx.submit(pid, db.slice(l, l + 1), prm)
                with lock:
                    out[l] = t
        th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        [t.start() for t in th]
        [t.join() for t in th]
        for l in range(db.n_lig):
            rc, st = ctx.poll(out[l], 60_000)
            assert rc == dk.DOCK_OK and st == (0, 1, 1)
            assert_same(ref[l], per_ligand(ctx.results(out[l]), db.slice(l, l + 1), prm.restarts)[0])
        assert ctx.stats()["batches"] >= 4


def test_error_codes(dk):
    w = synth.WORKLOADS["tiny"]
    db = synth.make_db(w, 4)
    prm = params(dk)
    with dk.Context(max_queued_ligands=5) as ctx:
        pid = ctx.load(synth.workload_pocket(w))
        with pytest.raises(dk.DockError) as e:
            ctx.submit(pid + 100, db, prm)
        assert e.value.code == dk.DOCK_ERR_NOPOCKET
        bad = synth.make_db(w, 2)
        bad.bonds[0, 0] = 999
        with pytest.raises(dk.DockError) as e:
            ctx.submit(pid, bad, prm)
        assert e.value.code == dk.DOCK_ERR_INVALID and "ligand 0" in str(e.value)
        with pytest.raises(dk.DockError) as e:
            ctx.poll(123456789)
        assert e.value.code == dk.DOCK_ERR_UNKNOWN_TICKET
        with pytest.raises(dk.DockError) as e:
            ctx.submit(pid, synth.make_db(w, 6), prm)    # more than max_queued_ligands waiting
        assert e.value.code == dk.DOCK_ERR_BUSY
        t = ctx.submit(pid, db, prm)
        rc, _ = ctx.poll(t, 60_000)
        assert rc == dk.DOCK_OK
        assert ctx.results(t) is not None
        with pytest.raises(dk.DockError) as e:
            ctx.results(t)                                # released by the first results call
        assert e.value.code == dk.DOCK_ERR_UNKNOWN_TICKET
        with pytest.raises(dk.DockError) as e:
            ctx.load_pocket(np.zeros((1, 4, 4), np.float32), 0.5, (0, 0, 0))
        assert e.value.code == dk.DOCK_ERR_INVALID


def test_watchdog_reports_a_stalled_batch(dk):
    """A serving batch that runs past stall_timeout_ms (here 1 ms, for a batch that needs several)
    stops admission and unfinished tickets report DOCK_ERR_TIMEOUT; the kernels themselves run to
    completion and the context is destroyed cleanly.  No GPU fault is involved."""
    w = synth.WORKLOADS["uneven"]
    db = synth.make_db(w, 2000, workers=synth.default_workers())
    prm = dk.Params.make(restarts=30, align_steps=30, torsion_steps=256, seed=4)
    ctx = dk.Context(stall_timeout_ms=1, n_streams=1, max_batch_ligands=2000)
    try:
        pid = ctx.load(synth.workload_pocket(w))
        t = ctx.submit(pid, db, prm)
        with pytest.raises(dk.DockError) as e:
            for _ in range(100):
                rc, _ = ctx.poll(t, 1000)
                if rc == dk.DOCK_OK:
                    break
        assert e.value.code == dk.DOCK_ERR_TIMEOUT and "stall_timeout_ms" in str(e.value)
        t2 = ctx.submit(pid, db.slice(0, 1), prm)   # accepted, but never admitted while stalled
        with pytest.raises(dk.DockError) as e2:
            ctx.poll(t2, 200)
        assert e2.value.code == dk.DOCK_ERR_TIMEOUT
    finally:
        ctx.close()


def test_best_outputs_only(dk):
    """DOCK_OUTPUT_BEST keeps and copies back only the per-ligand outputs: they equal the full run's,
    fewer bytes cross PCIe, and asking for a per-restart output is an error."""
    w = synth.WORKLOADS["tiny"]
    db = synth.make_db(w, 40, seed=31)
    full = dk.Params.make(restarts=8, align_steps=30, torsion_steps=64, clash_dist=2.0, seed=3, select_k=3,
                          select_rmsd=1.0)
    best = dk.Params.make(restarts=8, align_steps=30, torsion_steps=64, clash_dist=2.0, seed=3, select_k=3,
                          select_rmsd=1.0, outputs=dk.DOCK_OUTPUT_BEST)
    keys = ["score", "best_restart", "xyz", "clash_count", "select_restart", "select_score", "select_xyz"]
    with dk.Context() as ctx:
        pid = ctx.load(synth.workload_pocket(w))
        ref = ctx.dock(pid, db, full)
        d0 = ctx.stats()["d2h_bytes"]
        got = ctx.dock(pid, db, best)
        d_best = ctx.stats()["d2h_bytes"] - d0
        assert "restart_score" not in got
        for k in keys:
            assert np.array_equal(ref[k], got[k]), k
        d0 = ctx.stats()["d2h_bytes"]
        ctx.dock(pid, db, full)
        assert d_best < ctx.stats()["d2h_bytes"] - d0
        t = ctx.submit(pid, db, best)
        ctx.poll(t, 60_000)
        with pytest.raises(dk.DockError) as e:
            _full_results(dk, ctx, t, db, best)
        assert e.value.code == dk.DOCK_ERR_INVALID and "DOCK_OUTPUT_BEST" in str(e.value)
        b = ctx.batch_create(db, best)
        ctx.batch_launch(pid, b)
        bres = ctx.batch_results(b)
        for k in keys:
            assert np.array_equal(ref[k], bres[k]), k
        ctx.batch_destroy(b)


def _full_results(dk, ctx, ticket, db, prm):
    """dock_results with every output requested, bypassing the binding's choice of buffers."""
    r, c = dk._alloc_results(db.n_lig, int(db.atom_off[-1]), int(db.rot_off[-1]), prm.restarts, prm.k, False)
    ctx._check(ctx._lib.dock_results(ctx.h, ticket, dk.C.byref(c)))
    return r


def test_adaptive_launch_shape(dk):
    """Small serving batches run with the latency shape (8 warps per ligand-restart), large ones with
    the context's shapes; results are the same bit for bit either way and with the policy off."""
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    db = synth.make_db(w, 32, seed=9)
    prm = params(dk, seed=5)
    got = {}
    for name, items in [("default", 0), ("off", -1), ("always", 1 << 20), ("tiny", 8)]:
        with dk.Context(serve_latency_items=items) as ctx:
            pid = ctx.load(pk)
            ref = batch_results(ctx, pid, db, prm)
            t = ctx.submit(pid, db, prm)
            ctx.poll(t, -1)
            got[name] = ctx.results(t)
            st = ctx.stats()
            # 32 ligands x 8 restarts = 256 items: within the default threshold (2 x 4 x SMs)
            expect_latency = {"default": True, "off": False, "always": True, "tiny": False}[name]
            assert (st["latency_batches"] > 0) == expect_latency, (name, st)
            for k in KEYS:
                assert np.array_equal(got[name][k], ref[k]), (name, k)
    with pytest.raises(dk.DockError):
        dk.Context(n_streams=65)


def test_unload_defers_the_free_and_stalls_nothing(dk):
    """dock_unload_pocket returns at once while another pocket's large ticket is on the GPU (no
    device-wide wait, no lock held across one), the other ticket's polls keep answering, and a
    pocket unloaded while its own ticket is in flight is freed only after that ticket's kernels:
    every result equals a batch run bit for bit."""
    import time
    w = synth.WORKLOADS["uneven"]
    big = synth.make_db(w, 6000, workers=synth.default_workers(), seed=61)
    small = synth.make_db(w, 40, seed=62)
    prm = dk.Params.make(restarts=30, align_steps=30, torsion_steps=256, seed=8)
    with dk.Context(serve=False) as c0:
        ref_big = batch_results(c0, c0.load(synth.workload_pocket(w, 1)), big, prm)
        ref_small = batch_results(c0, c0.load(synth.workload_pocket(w, 2)), small, prm)
    with dk.Context(n_streams=2, max_batch_ligands=2000) as ctx:
        pa = ctx.load(synth.workload_pocket(w, 0))
        pb = ctx.load(synth.workload_pocket(w, 1))
        pc = ctx.load(synth.workload_pocket(w, 2))
        ctx.dock(pb, small.slice(0, 4), prm)            # warm: slots grown, kernels loaded
        t_big = ctx.submit(pb, big, prm)                  # tens of milliseconds of GPU work
        time.sleep(0.005)
        t0 = time.perf_counter()
        ctx.unload_pocket(pa)                             # idle pocket
        t_idle = time.perf_counter() - t0
        t_small = ctx.submit(pc, small, prm)
        time.sleep(0.002)
        t0 = time.perf_counter()
        ctx.unload_pocket(pc)                             # its own ticket may still be running
        t_busy = time.perf_counter() - t0
        t0 = time.perf_counter()
        rc, st = ctx.poll(t_big, 0)                       # answers without waiting for the GPU
        t_poll = time.perf_counter() - t0
        pending_at_unload = st[0]
        rc, _ = ctx.poll(t_big, 120_000)
        assert rc == dk.DOCK_OK
        got_big = ctx.results(t_big)
        rc, _ = ctx.poll(t_small, 120_000)
        assert rc == dk.DOCK_OK
        got_small = ctx.results(t_small)
        with pytest.raises(dk.DockError) as e:
            ctx.submit(pc, small.slice(0, 1), prm)
        assert e.value.code == dk.DOCK_ERR_NOPOCKET
    print(f"\nunload idle {t_idle * 1e3:.3f} ms, unload busy {t_busy * 1e3:.3f} ms, poll {t_poll * 1e3:.3f} ms, "
          f"big ticket pending at unload: {bool(pending_at_unload)}")
    assert pending_at_unload          # the unloads happened while the large ticket was on the GPU
    assert t_idle < 0.02 and t_busy < 0.02 and t_poll < 0.02
    assert_same(ref_big, got_big)
    assert_same(ref_small, got_small)
