"""The N > 1 form of bench.py runs independent replicas (the path needs no
cross-GPU exchange): each rank times its own steps, the job time is the
slowest rank's, and the value counts every rank's evaluations.  Checked
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = [3.0, 5.5][rank]  # rank 1 is slower
    got = bench.max_over_ranks(mine, dist, torch.device("cpu"))
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_all_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == 5.5
    # two replicas of N = 1e6 points, K = 32, 10 steps in 5.5 ms
    assert bench.whole_job_value(1_000_000, 32, 10, 2, 5.5) == pytest.approx(2 * 1e6 * 32 * 10 / 5.5e-3)


def test_dist_env_defaults_to_one_rank(monkeypatch):
    for v in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)
    assert bench.dist_env() == (1, 0, 0)
