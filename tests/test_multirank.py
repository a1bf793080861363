"""Replica path of bench.py on CPU with two gloo ranks: each rank solves its own copy,
and only the end-of-run aggregation (max time, summed updates) crosses ranks."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, upd = bench.aggregate_ranks(1.0 + rank, 100.0 * (rank + 1), device="cpu")
    out[rank] = (secs, upd, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        secs, upd, env = res[rank]
        assert secs == 2.0 and upd == 300.0
        assert env[0] == 2 and env[1] == rank


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_ranks(1.5, 42.0) == (1.5, 42.0)
