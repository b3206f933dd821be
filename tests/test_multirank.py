"""Several ranks, on CPU (gloo, world size 2): the rows of a search split into
contiguous shards, the slowest rank's time is the job's, and the candidate
lists gathered on rank 0 equal the single-process search of every row.  Each
rank runs the oracle on its shard (the GPU kernels are per row, so the host
logic is what a CPU run can check)."""
import os
import socket

import numpy as np
import pytest

from paper_1910_08324_gb300 import shard
from paper_1910_08324_gb300._binding import CANDIDATE_DTYPE

torch = pytest.importorskip("torch")

NDM, NT, SEED = 7, 12000, 4242


def _series():
    import spd_synth
    x = spd_synth.gaussian_noise(NDM, NT, SEED, dtype=np.float64)
    tab = spd_synth.pulse_table(10, NDM, NT, SEED + 1, width_range=(1, 200), snr_range=(7.0, 15.0), min_gap=600)
    spd_synth.inject(x, tab)
    return x


def _records(x_rows):
    import oracle
    Y, W, _ = oracle.search(x_rows, oracle.grid_igrid(1, 4, 256))
    tot, rows, starts, widx, snr = oracle.candidates(Y, W, 4.0, 1)
    rec = np.zeros(tot, CANDIDATE_DTYPE)
    rec["row"], rec["start"], rec["width_idx"], rec["snr"] = rows, starts, widx, snr
    return rec


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, n = shard.row_shard(NDM, rank, world)
        rec = _records(_series()[first:first + n])
        allrec = shard.gather_candidates(rec, first, dist)
        slowest = shard.max_over_ranks(10.0 * (rank + 1), dist)
        if rank == 0:
            q.put((allrec, slowest))
        else:
            assert allrec is None
    finally:
        dist.destroy_process_group()


def test_row_shards_cover_every_row_once():
    for ndm in (1, 7, 64, 4097):
        for world in (1, 2, 3, 8):
            spans = [shard.row_shard(ndm, r, world) for r in range(world)]
            assert spans[0][0] == 0 and sum(n for _, n in spans) == ndm
            assert all(a + n == b for (a, n), (b, _) in zip(spans, spans[1:]))
    with pytest.raises(ValueError):
        shard.row_shard(4, 2, 2)


def test_two_gloo_ranks_equal_one_process():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        allrec, slowest = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert slowest == 20.0
    ref = _records(_series())
    assert len(ref) > 5 and np.array_equal(allrec, ref)
