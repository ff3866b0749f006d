"""Multi-process sharding logic on CPU: two gloo ranks split a database and reduce their times."""
import os
import socket

import pytest

from paper_2209_05069_gb300 import shard, synth


def test_rank_range_partitions():
    for n in (0, 1, 7, 100, 10001):
        for world in (1, 2, 3, 8):
            spans = [shard.rank_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.rank_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db = synth.make_db(synth.WORKLOADS["tiny"], 30)
        mine = shard.shard_db(db, rank, world)
        ids = [None] * world
        dist.all_gather_object(ids, [int(i) for i in mine.ids])
        t = shard.max_over_ranks(1.5 + rank, dist)
        q.put((rank, ids, t, int(mine.atom_off[-1]), int(mine.xyz.shape[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_and_reduce():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    all_ids = out[0][1]
    assert out[1][1] == all_ids
    flat = [i for part in all_ids for i in part]
    assert sorted(flat) == list(range(30)) and len(set(flat)) == 30
    assert all(t == 2.5 for _, _, t, _, _ in out)
    assert all(a == x for _, _, _, a, x in out)
