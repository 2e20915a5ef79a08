"""Multi-process path of the benchmark (independent replicas, one per rank):
rank environment parsing, slowest-rank timing and the whole-job throughput,
exercised with two gloo ranks on the CPU (127.0.0.1 rendezvous)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    ms = bench.max_over_ranks(1.0 + rank)
    out[rank] = (ws, r, local, ms, bench.replica_value(1000, ws, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ws, r, local, ms, val = res[rank]
        assert (ws, r, local) == (world, rank, rank)
        assert ms == 2.0
        assert val == pytest.approx(world * 1000 / 2e-3 / 1e6)


def test_single_process_environment_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
