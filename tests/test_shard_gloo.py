"""Row-range sharding of the aggregation path across ranks (CPU, gloo, 2 ranks).

Each rank aggregates its contiguous slice of the fact rows with the oracle;
an all-reduce (sum) of the exact int64 partials must equal the aggregate of
the whole table -- integer addition makes the exchange bit-exact in any
order.  This is the identity a row-partitioned multi-GPU run relies on.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import datagen
import oracle

N = 200_000
AGGS = [("sum", [("col", 3)]), ("sum", [("col", 4)]), ("count", None)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cols(lo, hi):
    t = datagen.fact_table(hi - lo, seed=77, row0=lo)
    return [t["date"], t["flag"], t["status"], t["quantity"], t["price"]]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = rank * N // world, (rank + 1) * N // world
    keys, iv, _ = oracle.groupby(_cols(lo, hi), [(0, "le", 2450)], [1, 2], AGGS)
    full = np.zeros((3, 2, len(AGGS)), np.int64)  # dense over the (flag, status) domain
    for k, v in zip(keys, iv):
        full[k[0], k[1]] = v
    t = torch.from_numpy(full.reshape(-1).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        out.put(t.numpy().copy())
    dist.barrier()
    dist.destroy_process_group()


def test_partial_aggregates_all_reduce_to_the_whole():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    keys, iv, _ = oracle.groupby(_cols(0, N), [(0, "le", 2450)], [1, 2], AGGS)
    want = np.zeros((3, 2, len(AGGS)), np.int64)
    for k, v in zip(keys, iv):
        want[k[0], k[1]] = v
    assert np.array_equal(got.reshape(3, 2, len(AGGS)), want)
