"""Replica bookkeeping for several GPUs, exercised on CPU with gloo (world size 2)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_03393_gb300 import dist as tdist


def test_shard_by_cells_covers_every_series_once():
    cells = [5, 1, 9, 3, 3, 7, 2]
    for ws in (1, 2, 3):
        parts = tdist.shard_by_cells(cells, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)


def test_replica_seeds_differ_per_rank():
    seeds = {tdist.replica_seed(100, r) for r in range(8)}
    assert len(seeds) == 8 and tdist.replica_seed(100, 0) == 100


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mx, sm = tdist.reduce_max_sum(float(10 + rank), float(rank + 1))
        q.put((rank, mx, sm))
    finally:
        dist.destroy_process_group()


def test_reduce_max_sum_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 11.0, 3.0), (1, 11.0, 3.0)]


def test_reduce_without_process_group_is_identity():
    assert tdist.reduce_max_sum(2.5, 4.0) == (2.5, 4.0)
