"""Multi-rank host logic of the replica path on CPU (gloo, world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2509_08383_gb300 import replicas


def test_shard_partitions_units():
    for n in (0, 1, 7, 64, 129):
        for ws in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, ws) for r in range(ws)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    start, stop = replicas.shard(10, rank, ws)
    t = replicas.max_over_ranks(1.0 + rank, dist)
    units = replicas.sum_over_ranks(stop - start, dist)
    dist.barrier()
    q.put((rank, t, units, (start, stop)))
    dist.destroy_process_group()


def test_two_rank_gloo_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]          # max over ranks
    assert [r[2] for r in res] == [10.0, 10.0]        # all units covered once
    assert res[0][3] == (0, 5) and res[1][3] == (5, 10)
