"""The multi-rank path on CPU: gloo, world size 2.  Each rank owns a disjoint
slice of the independent cases; the host reductions give the job's max time
and total case count."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_28203_gb300.shard import reduce_max, reduce_sum, shard_range


def test_shard_range_partition():
    for n in (0, 1, 7, 2379, 2400):
        for w in (1, 2, 3, 8):
            spans = [shard_range(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_range(2379, rank, world)
    t = reduce_max(1.0 + rank, dist)
    n = reduce_sum(hi - lo, dist)
    q.put((rank, lo, hi, t, n))
    dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert res[0][1:3] == (0, 1190) and res[1][1:3] == (1190, 2379)
    assert all(r[3] == 2.0 and r[4] == 2379 for r in res)
