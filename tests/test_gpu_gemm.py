"""GPU parity of the tensor-core (tcgen05, BF16 or FP16 operands) GEMM-form
path, d = 64.

Labels and counts must equal the FP64 oracle's exactly (the 16-bit screen
only proposes candidates; every decision is exact), centroids within 1e-6
relative, E within 1e-9 absolute.
"""
import math

import numpy as np
import pytest

import synth
from test_gpu_parity import assert_centroids_close, lockstep, E_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


TC = ["bf16", "f16"]


@pytest.mark.parametrize("tc", TC)
@pytest.mark.parametrize("n,k", [(20_000, 64), (20_000, 300), (5_003, 1024), (129, 7), (1_000, 1), (4_096, 257),
                                 (100, 10), (1, 1), (2, 2)])
def test_gemm_lockstep(km, oracle, n, k, tc):
    x, _, _ = synth.iso_mixture(n, 64, 40, sigma=1.0, box=10.0, seed=n + k)
    mu0, _ = synth.init_distinct(x, k, seed=k)
    st = lockstep(km, oracle, x, mu0, steps=2, tc_operands=tc)
    assert st["path"] == 3


@pytest.mark.parametrize("tc", TC)
def test_gemm_split_clusters_are_resolved_exactly(km, oracle, tc):
    # twice as many centroids as Gaussians: many points have two near-equal
    # nearest centres, far inside the 16-bit error window
    x, comp, means = synth.iso_mixture(30_000, 64, 16, sigma=1.0, box=10.0, seed=7)
    mu0 = np.concatenate([means, means + 0.05]).astype(np.float64)
    st = lockstep(km, oracle, x, mu0, steps=3, tc_operands=tc)
    assert st["path"] == 3 and st["flagged"] > 0


@pytest.mark.parametrize("scale,offset", [(1e-6, 0.0), (3e4, 0.0), (1.0, 1e4), (1e5, -3e6)])
def test_gemm_f16_operand_scaling(km, oracle, scale, offset):
    """FP16 holds magnitudes up to 65504 with 11 significand bits down to
    6.1e-5: coordinates far outside that range (tiny, huge, offset) are
    scaled by powers of two into it, so the labels stay exact and the
    candidate window stays narrow."""
    x, _, _ = synth.iso_mixture(12_000, 64, 24, sigma=1.0, box=10.0, seed=17)
    x = (x.astype(np.float64) * scale + offset).astype(np.float32)
    mu0, _ = synth.init_distinct(x, 48, seed=18)
    st = lockstep(km, oracle, x, mu0, steps=2, tc_operands="f16")
    assert st["path"] == 3


def test_gemm_f16_window_is_narrower(km, oracle):
    """The same split clusters with FP16 operands leave far fewer points
    with several candidates than with BF16 (11 against 8 significand bits)."""
    x, _, means = synth.iso_mixture(30_000, 64, 16, sigma=1.0, box=10.0, seed=7)
    mu0 = np.concatenate([means, means + 0.3]).astype(np.float64)
    flagged = {}
    for tc in TC:
        flagged[tc] = lockstep(km, oracle, x, mu0, steps=1, tc_operands=tc)["flagged"]
    assert flagged["f16"] < flagged["bf16"], flagged


@pytest.mark.parametrize("tc", TC)
def test_gemm_full_run(km, oracle, tc):
    x, _, _ = synth.iso_mixture(40_000, 64, 50, sigma=1.0, box=10.0, seed=3, weights="dirichlet")
    mu0, _ = synth.init_distinct(x, 50, seed=4)
    ref = oracle.run(x, mu0, 60, 1e-6)
    g = km.KMeans(x.shape[1], 64, 50, tc_operands=tc)
    g.set_points(x)
    g.set_init(mu0)
    r = g.run(60, 1e-6)
    assert r["iters"] == ref["iters"] and r["converged"] == ref["converged"]
    assert np.array_equal(r["labels"], ref["labels"])
    assert np.array_equal(g.counts(), ref["counts"])
    assert_centroids_close(r["centroids"], ref["centroids"], x)
    assert abs(r["E"] - ref["E"]) <= E_ABS
    g.close()


@pytest.mark.slow
def test_gemm_full_scale_lockstep(km, oracle):
    """N = 1e7, d = 64, K = 1024 (BF16 tensor-core distances) at full size: one
    step from the seeded start, every label and count equal to the oracle's,
    every centroid within 1e-6 of the oracle's centroid, E within its bound."""
    w = synth.workload("precision_highd_64d_n1e7_k1024")
    st = lockstep(km, oracle, w["x"], w["mu0"], steps=1)
    assert st["path"] == 3


@pytest.mark.parametrize("tc", TC)
def test_gemm_duplicate_centroids_near_tie_and_rescue_lists(km, oracle, tc):
    """Exact duplicates: 12 copies of one centre (a near tie with more
    candidates than one list entry of 8 would hold) and 30 copies of another
    (more than a near-tie entry holds: the all-K rescue).  The oracle takes
    the lowest index among equal distances; so must the GPU."""
    x, _, _ = synth.iso_mixture(20_000, 64, 30, sigma=1.0, box=10.0, seed=11)
    base, _ = synth.init_distinct(x, 40, seed=12)
    mu0 = np.concatenate([base, np.repeat(base[:1], 12, 0), np.repeat(base[1:2], 30, 0)])
    st = lockstep(km, oracle, x, mu0, steps=2, tc_operands=tc)
    assert st["path"] == 3 and st["flagged"] > 0
