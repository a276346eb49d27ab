"""Batch sharding over ranks: the partition, and a world-size-2 gloo run on
CPU in which each rank handles its share (with the oracle as the stand-in parse
function, since there is no GPU here) and rank 0 gathers every document's
result."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import gen
import oracle
from paper_1902_08318_gb300 import shard


def test_partition_balances_bytes_and_covers_all():
    rng = np.random.Generator(np.random.PCG64(1))
    for world in (1, 2, 3, 8):
        sizes = rng.integers(1, 5000, 1000)
        off = np.concatenate([[0], np.cumsum(sizes)])
        parts = shard.partition(off, world)
        assert parts[0][0] == 0 and parts[-1][1] == 1000
        for (a, b), (c, d) in zip(parts, parts[1:]):
            assert b == c and a <= b
        loads = [off[b] - off[a] for a, b in parts]
        assert max(loads) - min(loads) <= 2 * sizes.max()


def test_partition_more_ranks_than_documents():
    parts = shard.partition(np.array([0, 10, 20]), 4)
    assert sum(b - a for a, b in parts) == 2
    assert all(a <= b for a, b in parts)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, buf, off, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi, errs = shard.parse_shard(lambda b, o: oracle.parse_many_errors(b, o), buf, off, rank,
                                     world)
    out = shard.gather_errors(dist, lo, hi, errs, off.size - 1)
    if rank == 0:
        q.put(out.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world_size_2_gathers_every_document():
    buf, off = gen.config3(3000, n_docs=400, invalid_frac=0.05)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, buf, off, q), nprocs=2, join=True,
                       start_method="spawn")
    got = np.array(q.get(timeout=60), dtype=np.int32)
    assert np.array_equal(got, oracle.parse_many_errors(buf, off))
