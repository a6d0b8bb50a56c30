"""The multi-rank path of bench.py on the CPU: two gloo ranks, each timing its
own replica; the reported time is the maximum over ranks and every rank
agrees on it.  (The data path has no collective: replicas only.)"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, ws, port, results):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench

    assert bench.dist_env() == (ws, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    dist.barrier()
    per_rank_ms = 10.0 + 3.5 * rank
    results[rank] = bench.max_over_ranks(per_rank_ms, dist, "cpu")
    assert bench.max_over_ranks(per_rank_ms, None, "cpu") == per_rank_ms
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    ws = 2
    with mp.get_context("spawn").Manager() as m:
        results = m.dict()
        mp.start_processes(worker, args=(ws, free_port(), results), nprocs=ws, start_method="spawn", join=True)
        got = dict(results)
    assert got == {0: 13.5, 1: 13.5}
