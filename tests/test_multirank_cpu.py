"""The benchmark's multi-rank bookkeeping on CPU, world size 2 over gloo: ranks run
independent replica batches (no data exchange), the job's time is the slowest
rank's, and the throughput counts every rank's updates.  Nothing here touches a GPU."""
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


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        t_rank = 1.0 + rank            # rank 1 is the slow one
        t_job = bench.max_over_ranks(t_rank, ws, "cpu")
        out[rank] = (t_job, bench.job_throughput(ws, 1000, t_job))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_every_rank():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (2.0, 1000.0)   # 2 ranks x 1000 updates / 2.0 s


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1, 700, 3.5) == 200.0
