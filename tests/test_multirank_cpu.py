"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2):
each rank runs an independent replica (no data-path collective); the job's time
is the slowest rank's, and the rate counts the units of all ranks."""
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


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    env = bench.dist_env()
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    tot = bench.max_over_ranks(local_ms, ws, torch.device("cpu"))
    rate = bench.whole_job_rate(1000, ws, 10, tot)
    out[rank] = (env, tot, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction_gloo():
    ws = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for rank in range(ws):
        env, tot, rate = out[rank]
        assert env == (ws, rank, rank)
        assert tot == 150.0                          # max over ranks
        assert abs(rate - 2 * 1000 * 10 / 0.150) < 1e-6
