"""The bench's multi-GPU mode runs one independent replica per rank (the
hot path has no exchange step): its whole-job reduction, units summed over
ranks and time maximised over ranks, checked with two gloo ranks on CPU."""
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import mdgen
    units = [1.0 + rank, 10.0 * (rank + 1), 100.0]
    tot, tmax = bench.whole_job(units, 1.0 + 0.5 * rank, world, torch.device("cpu"))
    # each rank owns its own seeded replica of the workload
    c = mdgen.config_lj_fluid(n=256, seed_k=rank)
    out[rank] = (tot, tmax, float(c["r"][0, 0]))
    dist.destroy_process_group()


def test_whole_job_reduction_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        tot, tmax, _ = res[rank]
        assert tot == [3.0, 30.0, 200.0]
        assert tmax == 1.5
    assert res[0][2] != res[1][2]  # distinct seeds per rank
