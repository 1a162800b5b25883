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
