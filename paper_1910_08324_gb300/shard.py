"""Several GPUs: DM rows are independent (Sec. 4.4: the search separates by DM
trial), so each process searches a contiguous block of rows on its own GPU and
nothing is exchanged on the data path.  The host-side pieces live here:

* ``row_shard``: the rows of one rank;
* ``max_over_ranks``: the slowest rank's time (the job's time);
* ``gather_candidates``: every rank's candidate records, rows made global,
  concatenated on rank 0 in (row, start) order.

They work with any ``torch.distributed`` backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def row_shard(ndm: int, rank: int, world: int):
    """(first row, row count) of ``rank``: contiguous blocks, the first
    ``ndm % world`` ranks one row longer."""
    if world < 1 or not 0 <= rank < world or ndm < 0:
        raise ValueError("bad shard request: ndm=%d rank=%d world=%d" % (ndm, rank, world))
    base, extra = divmod(ndm, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _device(dist):
    import torch
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(value: float, dist=None) -> float:
    """The largest ``value`` over the ranks (the value itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_candidates(records, first_row: int, dist=None, dst: int = 0):
    """Rank ``dst`` receives every rank's records (numpy structured arrays with a
    ``row`` field, rows local to the rank's shard) with global rows, ordered by
    (row, start); the other ranks receive None."""
    rec = records.copy()
    rec["row"] = rec["row"] + first_row
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return rec[np.lexsort((rec["start"], rec["row"]))]
    parts = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object(rec, parts, dst=dst)
    if dist.get_rank() != dst:
        return None
    out = np.concatenate(parts)
    return out[np.lexsort((out["start"], out["row"]))]
