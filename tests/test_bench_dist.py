"""Host logic of bench.py's multi-rank path, on CPU with gloo (world size 2): each rank reports
its own time, the job takes the slowest rank's, and throughput counts every rank's work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_env()
    t = bench.reduce_max(1.0 + rank, w)
    bench.barrier(w)
    q.put((r, w, t, bench.job_throughput(10.0, w, t)))
    dist.destroy_process_group()


def test_reduce_max_and_job_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, world, t, thr in res:
        assert world == 2
        assert t == 2.0  # the slower rank's time on both ranks
        assert thr == pytest.approx(10.0 * 2 / 2.0)


def test_reference_arm_refuses_short_warmup():
    import bench

    with pytest.raises(SystemExit):
        bench.main(["--warmup", "1", "--impl", "reference"])
