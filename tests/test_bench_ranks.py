"""Host logic of the multi-replica bench on CPU ranks (gloo): the timed
region's length is the maximum over ranks and the job's rate counts every
rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0, 7.0][rank]
    total = bench.max_over_ranks(ms, torch.device("cpu"))
    rate = bench.whole_job_rate(1000, world, total)
    q.put((rank, total, rate))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_whole_job_rate(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = max([12.5, 20.0, 7.0][:world])
    for rank, total, rate in got:
        assert total == want
        assert rate == pytest.approx(1000 * world / (want / 1e3))


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_rate(10, 1, 1000.0) == 10.0
