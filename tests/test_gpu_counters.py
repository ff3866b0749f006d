"""The counter build (libdock_count.so: the same sources with DOCK_COUNT_WORK) counts the work the
docking kernels execute, without changing a result.

With early exit off and A a multiple of 32 every count the host can derive is checked exactly:
alignment pose lanes (both alignments, whole passes of 32), and lookups evaluated (alignment poses x
atoms + every torsion angle x the moving atoms but b + the final pose), from dock_batch_work's
algorithmic counts.  Loads never exceed lookups, distinct sectors never exceed loads, distinct
128-byte lines never exceed sectors, and with early
exit on the kernels evaluate no more than with it off.
"""
import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    from paper_2209_05069_gb300 import dock
    return dock


def _run(ctx, pid, db, prm):
    b = ctx.batch_create(db, prm)
    ctx.batch_launch(pid, b)
    ctx.batch_wait(b)
    res = ctx.batch_results(b)
    work = ctx.batch_work(b)
    ctx.batch_destroy(b)
    return res, work


@pytest.mark.parametrize("grid_dtype", ["f32", "f16", "i16"])
def test_counter_build_counts_and_changes_nothing(dk, grid_dtype):
    w = synth.WORKLOADS["uneven"]
    pk = synth.workload_pocket(w)
    if grid_dtype == "i16":
        pk = pk.integer(1000)
    db = synth.make_db(w, 300, seed=44)
    R, N, A = 6, 30, 64
    got = {}
    for ee in (0, 1):
        prm = dk.Params.make(restarts=R, align_steps=N, torsion_steps=A, seed=4, early_exit=ee)
        with dk.Context(serve=False) as ctx:
            ref, _ = _run(ctx, ctx.load(pk, grid_dtype), db, prm)
        with dk.Context(serve=False, counters=True) as ctx:
            pid = ctx.load(pk, grid_dtype)
            res, work = _run(ctx, pid, db, prm)
            c = ctx.exec_counters(reset=True)
            assert ctx.exec_counters()["items"] == 0          # reset
        for k in ref:
            assert np.array_equal(ref[k], res[k]), k         # counting changes no result
        got[ee] = (c, work)
    c, work = got[0]
    items = db.n_lig * R
    passes = -(-N * N // 32)
    assert c["items"] == items
    assert c["align_poses"] == 2 * items * 32 * passes
    align_lookups = work["lookups_align"] * 32 * passes // (N * N)
    assert c["lookups"] == align_lookups + work["lookups_torsion"] + work["lookups_final"]
    assert c["torsion_angles"] == R * int(db.rot_off[-1]) * 32 * -(-A // 32)   # every pass of every bond
    assert 0 < c["loads"] <= c["lookups"] and 0 < c["sectors"] <= c["loads"] and 0 < c["lines"] <= c["sectors"]
    assert c["angles_accepted"] <= c["torsion_angles"] and c["pair_tests"] > 0
    c1, _ = got[1]
    assert c1["items"] == items and c1["align_poses"] == c["align_poses"]
    assert c1["lookups"] <= c["lookups"] and c1["pair_tests"] <= c["pair_tests"]
    assert c1["angles_accepted"] == c["angles_accepted"]   # every accepted angle is scored either way
    print(f"\n{grid_dtype}: early exit off {c}\n{grid_dtype}: early exit on  {c1}")


def test_product_build_has_no_counters(dk):
    with dk.Context(serve=False) as ctx:
        with pytest.raises(dk.DockError) as e:
            ctx.exec_counters()
        assert e.value.code == dk.DOCK_ERR_INVALID and "counters" in str(e.value)
