"""Failure detection on the GPU without a fault: every mbarrier wait of the
library's kernels is bounded; the self-test waits on a barrier that nothing
arrives on and must give up by its limit with the device still usable."""
import numpy as np
import pytest

import synth
from test_gpu_parity import lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


def test_bounded_wait_gives_up_and_the_device_stays_usable(km, oracle):
    r = km.selftest_bounded_wait()
    assert r["gave_up"], r
    assert 500.0 < r["elapsed_ms"] < 60_000.0, r
    # the same process keeps running the path: the fused kernel and the
    # tensor-core kernel (whose waits are the bounded ones)
    x, _, _ = synth.iso_mixture(20_000, 3, 8, seed=5)
    mu0, _ = synth.init_distinct(x, 8, seed=6)
    assert lockstep(km, oracle, x, mu0, steps=1)["path"] == 1
    x, _, _ = synth.iso_mixture(5_000, 64, 16, seed=7)
    mu0, _ = synth.init_distinct(x, 32, seed=8)
    assert lockstep(km, oracle, x, mu0, steps=1)["path"] == 3


def _attempt(km, fn):
    """'ok', or 'enomem' when the injected allocation failure surfaced as
    KM_ENOMEM (any other error fails the test)."""
    try:
        fn()
        return "ok"
    except km.KMError as e:
        assert e.status == -2, e
        return "enomem"


def test_allocation_failures_are_reported_and_freed(km):
    """Host-side fault injection: the n-th device allocation fails as out of
    memory, for n = 0, 1, ... until the workflow completes.  Every failure
    is KM_ENOMEM from the call that allocated, the context is destroyed
    cleanly, and the device memory returns to where it was."""
    import gc
    import torch
    x3, _, _ = synth.iso_mixture(30_000, 3, 8, seed=3)
    m3, _ = synth.init_distinct(x3, 8, seed=4)
    x64, _, _ = synth.iso_mixture(3_000, 64, 8, seed=5)
    m64, _ = synth.init_distinct(x64, 16, seed=6)

    def plain(x, mu0):
        def run():
            g = km.KMeans(x.shape[1], x.shape[0], mu0.shape[0])
            try:
                g.set_points(x)
                g.set_init(mu0)
                g.step()
                g.objective()
            finally:
                g.close()
        return run

    insts = synth.batch_instances(3, seed=7, n_lo=500, n_hi=3_000)

    def batch():
        # creation, points (with the range scans), starts, the tuner's trial
        # launches, the graph-driven run and the objective: every allocation
        # of a batch's life is walked
        b = km.KMeansBatch([w["n"] for w in insts], [w["d"] for w in insts], [w["k"] for w in insts])
        try:
            b.set_points([w["x"] for w in insts])
            b.set_init([w["mu0"] for w in insts])
            b.run(5, 1e-6)
            b.objective()
        finally:
            b.close()

    def setnet():
        km.SetNet(3, 16).close()

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for name, fn in (("fused", plain(x3, m3)), ("tensor", plain(x64, m64)), ("batch", batch),
                     ("setnet", setnet)):
        seen = []
        for n in range(0, 80):
            km.debug_fail_alloc_after(n)
            try:
                r = _attempt(km, fn)
            finally:
                km.debug_fail_alloc_after(-1)
            gc.collect()
            seen.append(r)
            if r == "ok":
                break
        assert seen[-1] == "ok" and seen[0] == "enomem" and seen.count("ok") == 1, (name, seen)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) < 64 << 20, (free0, free1)
