"""Ligand-level data parallelism over several GPUs, one process per GPU.

Ligands are independent (Section 4: the problem is embarrassingly parallel and LiGen splits
ligands across nodes with synchronisation only at I/O), so each rank docks its own share with no
exchange on the data path.  The only collectives are for measurement: a barrier around the timed
region and the maximum of the ranks' times.
"""
from __future__ import annotations


def rank_range(n_total: int, rank: int, world: int):
    """Contiguous share [lo, hi) of n_total ligands for `rank` (sizes differ by at most one)."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} out of [0, {world})")
    q, r = divmod(n_total, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_db(db, rank: int, world: int):
    """This rank's contiguous share of a LigandDB."""
    lo, hi = rank_range(db.n_lig, rank, world)
    return db.slice(lo, hi)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over all ranks (the identity without torch.distributed)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
