"""GPU k-means++ seeding against the oracle's, with the same uniforms: the
chosen point indices and centres are equal (the GPU's chunked FP64 sums
could differ from the sequential ones only for a target within rounding of
a running-sum boundary, which these seeds do not hit)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


@pytest.mark.parametrize("n,d,k,seed", [(1_000, 2, 8, 0), (50_003, 3, 32, 1), (8_191, 3, 64, 2),
                                        (120_000, 64, 16, 3), (4_097, 1, 5, 4)])
def test_kmeanspp_matches_oracle(km, oracle, n, d, k, seed):
    x, _, _ = synth.iso_mixture(n, d, max(k // 2, 1), sigma=1.0, box=10.0, seed=seed)
    u = np.random.default_rng(100 + seed).random(k)
    g = km.KMeans(n, d, k)
    g.set_points(x)
    mu, idx = g.init_kmeanspp(u)
    mu_ref, idx_ref = oracle.kmeanspp(x, k, u)
    assert np.array_equal(idx, idx_ref)
    assert np.array_equal(mu, mu_ref)
    # the seeding became the start of the run
    r = g.run(5, 0.0)
    ref = oracle.run(x, mu_ref, 5, 0.0)
    assert np.array_equal(r["labels"], ref["labels"])
    # the objective of the final labels and centres, in the oracle's order
    # (the centres agree to within their own rounding)
    assert abs(g.objective() - ref["objective"]) <= 1e-12 * ref["objective"]
    g.close()


def test_kmeanspp_degenerate_inputs(km, oracle):
    # all points equal: every D^2 is 0, no running sum exceeds 0, so every
    # later centre is the last point; u[0] near 1 picks the last point first
    x = np.full((2, 9_000), 3.0, dtype=np.float32)
    u = np.array([0.9999999, 0.0, 0.5, 0.25])
    g = km.KMeans(9_000, 2, 4)
    g.set_points(x)
    mu, idx = g.init_kmeanspp(u)
    mu_ref, idx_ref = oracle.kmeanspp(x, 4, u)
    assert np.array_equal(idx, idx_ref) and idx[0] == 8_999 and np.all(idx[1:] == 8_999)
    assert np.array_equal(mu, mu_ref)
    with pytest.raises(km.KMError):
        g.init_kmeanspp(np.array([0.1, 0.2, 1.0, 0.3]))
    g.close()
