"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the path
shards into independent replicas with no data exchange, so the only collective
is the max-over-ranks of the timed region; value = all ranks' steps / that max."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank 0 ran its 100 steps in 200 ms, rank 1 in 300 ms: the job took 300 ms
    value, t_ms = bench.job_throughput(200.0 + 100.0 * rank, 100, world, "cpu")
    q.put((rank, value, t_ms, bench.rank_info()))
    dist.destroy_process_group()


def test_job_throughput_is_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_ms, info in out:
        assert t_ms == 300.0
        assert value == pytest.approx(world * 100 / 0.3)
        assert info == (rank, world, rank)


def test_job_throughput_single_rank():
    import bench

    value, t_ms = bench.job_throughput(250.0, 50, 1)
    assert t_ms == 250.0 and value == pytest.approx(200.0)
