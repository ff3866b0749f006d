"""dock_batch_launch_noalloc: the allocation-free launch matches dock_batch_launch.

Callers that cannot allocate device memory when they dock (their GPU memory is owned by another
allocator, or cudaMalloc/cudaFree would stall a latency-critical loop) hand the library their own
result buffers; the library's kernel scratch then comes from one fixed array inside libdock.so.
This file is named to be collected last, so a run that stops at the first failure has already run
every other test; it passes alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

from paper_2209_05069_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_buffers(torch, db, R):
    n_lig, n_atoms, n_rot = db.n_lig, int(db.atom_off[-1]), int(db.rot_off[-1])
    f32 = dict(dtype=torch.float32, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    return {
        "score": torch.full((n_lig,), -7.0, **f32), "best_restart": torch.full((n_lig,), -7, **i32),
        "xyz": torch.full((n_atoms, 3), -7.0, **f32), "clash_count": torch.full((n_lig,), -7, **i32),
        "restart_score": torch.full((n_lig * R,), -7.0, **f32), "restart_clash": torch.full((n_lig * R,), -7, **i32),
        "align_idx": torch.full((n_lig * R,), -7, **i32), "post_idx": torch.full((n_lig * R,), -7, **i32),
        "torsion_idx": torch.full((n_rot * R,), -7, **i32), "rejected": torch.full((n_rot * R,), -7, **i32),
    }


def _assert_matches(ref, got):
    """The same kernels on the same inputs: every output bit for bit."""
    for k, t in got.items():
        a = np.asarray(ref[k]).reshape(-1)
        b = t.cpu().numpy().reshape(-1)
        assert a.shape == b.shape, k
        assert np.array_equal(a, b), k


def _mixed_db(w, seed):
    """Ligands of 20-150 atoms: every atom bucket (<= 32, ... <= 160) has some, so the call makes
    several launches with nonzero item offsets and the larger ligands' pose offsets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ligs = []
    for i, n in enumerate([24, 30, 40, 55, 63, 70, 90, 100, 125, 150, 28, 60]):
        while True:
            xyz, bonds, rot, clipped = synth.make_ligand(rng, n, 3 + i % 5)
            if not clipped:
                break
        ligs.append((xyz, bonds, rot, 5000 + i))
    return synth.from_ligands(ligs)


def test_noalloc_launch_matches_batch_launch_twice():
    torch = pytest.importorskip("torch")
    from paper_2209_05069_gb300 import dock
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    prm = dock.Params.make(restarts=w.restarts, align_steps=w.align_steps, torsion_steps=w.torsion_steps,
                           clash_dist=w.clash_dist, seed=31)
    with dock.Context(serve=False) as ctx:
        pid = ctx.load(pk)
        stream = torch.cuda.Stream()
        # two calls in a row with different scratch layouts, then a batch spanning every atom bucket
        for db in (synth.make_db(w, 32, seed=1032), synth.make_db(w, 20, seed=1020), _mixed_db(w, 77)):
            batch = ctx.batch_create(db, prm)
            ctx.batch_launch(pid, batch)
            ref = ctx.batch_results(batch)
            out = _device_buffers(torch, db, prm.restarts)
            ptrs = {k: t.data_ptr() for k, t in out.items()}
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            n = ctx.batch_launch_noalloc(pid, batch, ptrs, stream.cuda_stream)
            free1 = torch.cuda.mem_get_info()[0]
            assert n >= 1
            assert free1 == free0, "the allocation-free launch took device memory"
            ctx.batch_destroy(batch)   # waits for the launch's work (its completion event)
            stream.synchronize()
            _assert_matches(ref, out)
        assert n >= 4   # the mixed batch launched one kernel per atom bucket


def test_noalloc_scratch_is_taken_at_context_creation():
    """The fixed array is loaded when the first context on the device is created, so a docking call
    takes no device memory for it; the batch's own launch loads the kernels' code beforehand."""
    torch = pytest.importorskip("torch")
    from paper_2209_05069_gb300 import dock
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    prm = dock.Params.make(restarts=4, align_steps=8, torsion_steps=16, seed=3)
    db = synth.make_db(w, 8, seed=77)
    with dock.Context(serve=False) as ctx:
        pid = ctx.load(pk)
        batch = ctx.batch_create(db, prm)
        ctx.batch_launch(pid, batch)
        ctx.batch_wait(batch)
        out = _device_buffers(torch, db, prm.restarts)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            ctx.batch_launch_noalloc(pid, batch, {k: t.data_ptr() for k, t in out.items()})
            ctx.batch_wait(batch)
        assert torch.cuda.mem_get_info()[0] == free0
        ctx.batch_destroy(batch)


def test_noalloc_rejects_batches_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2209_05069_gb300 import dock
    w = synth.WORKLOADS["tiny"]
    pk = synth.workload_pocket(w)
    # 64 ligands of ~25 atoms at 1024 restarts need about 19 MB of pose scratch, over 16 MiB
    prm = dock.Params.make(restarts=1024, align_steps=1, torsion_steps=1, seed=1)
    db = synth.make_db(w, 64)
    need = ((4 * db.n_lig + 255) // 256) * 256 + 12 * int(db.atom_off[-1]) * prm.restarts
    assert need > dock.NOALLOC_SCRATCH_BYTES
    with dock.Context(serve=False) as ctx:
        pid = ctx.load(pk)
        batch = ctx.batch_create(db, prm)
        out = _device_buffers(torch, db, prm.restarts)
        with pytest.raises(dock.DockError) as ei:
            ctx.batch_launch_noalloc(pid, batch, {k: t.data_ptr() for k, t in out.items()})
        assert ei.value.code == dock.DOCK_ERR_INVALID and "scratch" in str(ei.value)
        ctx.batch_destroy(batch)
