"""The multi-rank host logic of the benchmark on CPU (gloo, two ranks): the
path does not shard within a domain, so N GPUs run N replicas; the job time
is the slowest rank's and the rate counts the units of every rank.  The
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [12.0, 30.0][rank]
    ms, rate = bench.job_time_and_rate(ms_local, 1000, world, dist, device="cpu")
    # the reference arm: ranks other than 0 return at once without work
    ran = "skipped on rank 0"
    if rank != 0:
        ran = bench.run_reference(type("A", (), {"workload": "ensemble", "steps": 1, "warmup": 0, "gpus": world})())
    q.put((rank, ms, rate, ran))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = root + (os.pathsep + old if old else "")
    try:
        for p in procs:
            p.start()
        res = sorted(q.get(timeout=100) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=30)
        os.environ["PYTHONPATH"] = old
    for rank, ms, rate, ran in res:
        assert ms == 30.0
        assert rate == pytest.approx(1000 * 2 / 0.030)
    assert res[1][3] is None
