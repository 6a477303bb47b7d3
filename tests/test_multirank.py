"""The multi-rank path of bench.py on CPU (gloo, world size 2): ranks repair
disjoint batches and the whole-job rate uses the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle

    progs = bench.shard("single_1x64_s8", 3, rank)
    res = oracle.repair_batch(progs)
    value, t = bench.whole_job(len(progs), 1.0 + rank, world, device="cpu")
    sig = [(int(p.a.sum()), int(p.b.sum()), int(p.op.sum())) for p in progs]
    gathered = [None] * world
    dist.all_gather_object(gathered, sig)
    dist.destroy_process_group()
    q.put((rank, value, t, gathered, [r["status"] for r in res]))


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t, gathered, statuses in out:
        assert t == 2.0  # the slowest rank's time
        assert value == pytest.approx(3 * 2 / 2.0)
        assert gathered[0] != gathered[1]  # disjoint shards
        assert all(s in (0, 1, 2) for s in statuses)
