"""World-size-2 gloo run of the bench's multi-rank logic on CPU: every rank
owns a disjoint block of ensemble rows (no data-path collective) and the job
time is the max over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = bench.shard_ids(rank, world, rows=64)
        got = [None] * world
        dist.all_gather_object(got, ids.tolist())
        t = bench.allreduce_max(1.0 + rank * 0.5, world)
        # each rank's rows are independent seeded instances
        from paper_2601_12204_b300 import workloads as W
        e = W.fourier_ensemble(len(ids), 32, ids=ids)
        q.put((rank, got, t, float(e.u0[:32].sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_rows_and_take_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    got = res[0][1]
    a, b = set(got[0]), set(got[1])
    assert not (a & b) and a | b == set(range(128))
    assert res[0][2] == res[1][2] == 1.5
    from paper_2601_12204_b300 import workloads as W
    e1 = W.fourier_ensemble(1, 32, ids=np.array([64]))
    assert res[1][3] == pytest.approx(float(e1.u0.sum()), rel=1e-15)
