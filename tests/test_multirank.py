"""Host logic of the N-replica benchmark over two CPU ranks (gloo): whole-job throughput
is the units of all ranks over the slowest rank's time; the reference arm runs on rank 0
only.  Walkers are independent (Alg. 1 line 2), so replicas exchange nothing but these
scalars."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t_local = [2.0, 3.0][rank]
    v = bench.aggregate_value(1000.0, t_local, ws)
    m = bench.reduce_max(float(rank + 10), ws)
    bench.barrier(ws)
    q.put((rank, v, m, bench.dist_env()))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
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
    for rank, v, m, env in out:
        assert v == pytest.approx(2 * 1000.0 / 3.0)   # slowest rank sets the time
        assert m == 11.0
        assert env == (2, rank, rank)


def _sum_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    q.put((rank, bench.reduce_sum([3.0, 4.5][rank], ws)))
    dist.destroy_process_group()


def test_two_rank_sum_gloo():
    """DMC populations differ between ranks: the job's moves are the sum over ranks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_sum_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [v for _, v in out] == [7.5, 7.5]
