"""Sharded steps: the points split over processes, one small table exchanged
per step (the paper's OpenMP scheme of local sums merged before the master
divides, section "Parallel Lloyd's algorithm", with an all-gather).

* On the CPU (two gloo ranks): the host-side exchange -- the grid exponent
  reduced to the maximum on every rank, the totals gathered in rank order.
* On the GPU (two processes, each its own context on the one GPU, gloo on
  host tensors): a ragged split of the points, several steps; every shard's
  centroids, counts and E bit-identical to one context over all points, its
  labels equal to that context's labels of its points, and the whole equal to
  the FP64 oracle -- on the fused FP32 path (d = 3) and on the tensor-core
  GEMM path (d = 64, totals from the sorted mean calculation).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class _FakeShard:
    def __init__(self, ex):
        self.ex = ex

    def grid_exponent(self):
        return self.ex

    def set_grid_exponent(self, ex):
        self.ex = ex


def _cpu_rank(rank, ws, port, out):
    import torch.distributed as dist
    from paper_2405_12052_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    g = _FakeShard([7, -3][rank])
    ex = shard.common_grid_exponent(g, dist)
    # rank r's table: values that identify the rank and the column, with
    # high words set, so any reordering or truncation shows
    tab = np.arange(10, dtype=np.int64).reshape(5, 2) + 1000 * (rank + 1)
    tab[:, 1] = -rank - 1
    got = shard.gather_totals(tab, dist)
    out[rank] = (ex, g.ex, got.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_cpu_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ex, gex, got = out[r]
        assert ex == gex == 7
        got = np.array(got)
        assert got.shape == (2, 5, 2)
        for q in range(2):
            assert np.array_equal(got[q, :, 0], np.arange(0, 10, 2) + 1000 * (q + 1))
            assert np.all(got[q, :, 1] == -q - 1)


STEPS = 4


def _gpu_rank(rank, ws, port, x, mu0, split, out):
    import torch
    import torch.distributed as dist
    import paper_2405_12052_gb300 as km
    from paper_2405_12052_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    torch.cuda.set_device(0)
    lo, hi = split[rank], split[rank + 1]
    xs = np.ascontiguousarray(x[:, lo:hi])
    d, n = xs.shape
    k = mu0.shape[0]
    g = km.KMeans(n, d, k)
    g.set_points(xs)
    ex_local = g.grid_exponent()
    ex = shard.common_grid_exponent(g, dist)
    g.set_init(mu0)
    g.begin(STEPS, -1.0)
    recs = []
    for _ in range(STEPS):
        shard.sharded_step(g, dist)
        st = g.sync()
        recs.append((g.labels(), g.centroids(), g.counts(), st["E"], st["iters"]))
    g.close()
    out[rank] = (ex_local, ex, recs)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_steps_equal_one_context(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as km
    import synth
    km.build()
    x, _, _ = synth.aniso_mixture(150_011, 3, 20, seed=41)
    k = 32
    mu0, _ = synth.init_kmeanspp(x, k, seed=42)
    # the shards' ranges differ (sorted by the first coordinate, split at
    # 40 %): shard 1 needs a larger grid exponent than shard 0 or vice versa
    order = np.argsort(x[0], kind="stable")
    x = np.ascontiguousarray(x[:, order])
    n = x.shape[1]
    split = [0, int(0.4 * n), n]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, x, mu0, split, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    # one context over all points, the same steps
    g = km.KMeans(n, 3, k)
    g.set_points(x)
    g.set_init(mu0)
    ref_ex = g.grid_exponent()
    mu = mu0
    for t in range(STEPS):
        e, _ = g.step()
        z, c, cnt = g.labels(), g.centroids(), g.counts()
        zo, mo, co, _ = oracle.step(x, mu)
        assert np.array_equal(z, zo) and np.array_equal(cnt, co)
        mu = c
        for r in range(2):
            ex_local, ex, recs = out[r]
            assert ex == ref_ex and ex_local <= ex
            zr, cr, cntr, er, it = recs[t]
            assert it == t + 1
            assert np.array_equal(zr, z[split[r]:split[r + 1]]), (r, t)
            assert np.array_equal(cr, c), (r, t)      # bit-identical centroids
            assert np.array_equal(cntr, cnt), (r, t)  # global counts
            assert er == e, (r, t)                    # bit-identical E
    g.close()


@pytest.mark.gpu
def test_sharded_steps_tensor_core_path(oracle):
    """The same on the tensor-core GEMM path (d = 64): each shard's totals
    come from its sorted mean calculation; centroids, counts and E equal one
    context's bit for bit, labels that context's labels of its points."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as km
    import synth
    km.build()
    x, _, _ = synth.iso_mixture(60_013, 64, 24, sigma=1.0, box=8.0, seed=43)
    k = 64
    mu0, _ = synth.init_distinct(x, k, seed=44)
    order = np.argsort(x[0], kind="stable")
    x = np.ascontiguousarray(x[:, order])
    n = x.shape[1]
    split = [0, int(0.4 * n), n]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, x, mu0, split, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    g = km.KMeans(n, 64, k)
    g.set_points(x)
    g.set_init(mu0)
    assert g.stats()["path"] == 3
    ref_ex = g.grid_exponent()
    mu = mu0
    for t in range(STEPS):
        e, _ = g.step()
        z, c, cnt = g.labels(), g.centroids(), g.counts()
        zo, mo, co, _ = oracle.step(x, mu)
        assert np.array_equal(z, zo) and np.array_equal(cnt, co)
        mu = c
        for r in range(2):
            ex_local, ex, recs = out[r]
            assert ex == ref_ex and ex_local <= ex
            zr, cr, cntr, er, it = recs[t]
            assert it == t + 1
            assert np.array_equal(zr, z[split[r]:split[r + 1]]), (r, t)
            assert np.array_equal(cr, c), (r, t)
            assert np.array_equal(cntr, cnt), (r, t)
            assert er == e, (r, t)
    g.close()
