"""The fused kernel's constant-bank screen table at d = 3, K = 32.

One context per device holds the table in the constant bank; any other
context of the same shape alive at the same time runs the kernel that reads
the table from shared memory.  Both must give the oracle's labels and counts
bit-exact and its centroids within 1e-6 relative, and each other's results bit
for bit; once the holder is destroyed, a new context claims the table again.
"""
import numpy as np
import pytest

import synth
from test_gpu_parity import assert_centroids_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


def _ctx(km, x, mu):
    d, n = x.shape
    g = km.KMeans(n, d, mu.shape[0])
    g.set_points(x)
    g.set_init(mu)
    return g


def test_two_live_contexts_and_handover(km, oracle):
    x, _, _ = synth.aniso_mixture(400_009, 3, 24, seed=61)
    mu0, _ = synth.init_kmeanspp(x, 32, seed=62)
    holder = _ctx(km, x, mu0)
    other = _ctx(km, x, mu0)
    mu = np.array(mu0, dtype=np.float64)
    for t in range(3):
        # interleaved steps: the holder's table write must not disturb the other
        eh, _ = holder.step()
        eo, _ = other.step()
        z_ref, mu_ref, cnt_ref, _ = oracle.step(x, mu)
        for g in (holder, other):
            assert g.stats()["path"] == 1
            assert np.array_equal(g.labels(), z_ref), t
            assert np.array_equal(g.counts(), cnt_ref), t
            assert_centroids_close(g.centroids(), mu_ref, x)
        assert np.array_equal(holder.centroids(), other.centroids()) and eh == eo
        mu = holder.centroids()
        holder.set_init(mu)
        other.set_init(mu)
    holder.close()
    # the table passes to the next context of the shape; the old one keeps its kernel
    nxt = _ctx(km, x, mu)
    en, _ = nxt.step()
    eo, _ = other.step()
    z_ref, mu_ref, cnt_ref, _ = oracle.step(x, mu)
    for g in (nxt, other):
        assert np.array_equal(g.labels(), z_ref)
        assert np.array_equal(g.counts(), cnt_ref)
        assert_centroids_close(g.centroids(), mu_ref, x)
    assert np.array_equal(nxt.centroids(), other.centroids()) and en == eo
    nxt.close()
    other.close()
