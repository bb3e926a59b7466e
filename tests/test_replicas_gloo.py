"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): the path is
'replicas only' (one independent simulation per GPU, no collective on the
data path), so what ranks share is the barrier and the max-over-ranks time
that turns per-rank work into the whole-job value."""
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


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r 'took' 1 + r seconds for the same 1e9 units
    bench.barrier(ws)
    m = bench.allmax(1.0 + rank, ws)
    v = bench.replica_value(1e9, 1.0 + rank, ws)
    bench.barrier(ws)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 2.0                      # the slowest rank's time
        assert v == pytest.approx(2 * 1e9 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.allmax(3.5, 1) == 3.5
    assert bench.replica_value(10.0, 2.0, 1) == 5.0
