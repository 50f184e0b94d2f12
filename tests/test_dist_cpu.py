"""The benchmark's multi-rank logic on CPU (gloo, world size 2): each rank
works on its own configuration (distinct seeds, no data-path collective), the
barrier holds, and the reported time is the maximum over ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_init()
    assert (w, r) == (ws, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    t = bench.max_over_ranks(10.0 * (rank + 1), w)
    out[rank] = (bench.rank_seed(1000, rank), t)
    dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    seeds = {out[r][0] for r in range(ws)}
    assert len(seeds) == ws                          # distinct configurations
    assert all(out[r][1] == 20.0 for r in range(ws))  # max over ranks
