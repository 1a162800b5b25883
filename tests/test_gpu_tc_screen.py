"""The fused step with its screen on the TF32 tensor cores (dist_path="tensor"
for d <= 3, K <= 32): the screen values come from tcgen05.mma on split TF32
operands, with the tensor core's error bound added to the flag threshold.

Bar (as for every path): labels and counts bit-exact against the FP64
oracle in lockstep, centroids within 1e-6 relative, E within 1e-9; and,
because everything after the screen is the FFMA2 kernel's (recompute, flag
rule, re-check, exact integer sums), the results equal the FFMA2 path's bit
for bit.  Cases: d = 1, 2, 3; K = 1, 5, 17, 31, 32; ragged N (a partial
256-point super-tile); coordinates offset by 1e4; 1-byte labels; the final
labels pass; and K = 33 refused.
"""
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


def _steps(km, x, mu0, path, steps, **kw):
    d, n = x.shape
    g = km.KMeans(n, d, mu0.shape[0], dist_path=path, **kw)
    g.set_points(x)
    g.set_init(mu0)
    out = []
    for _ in range(steps):
        e, e2 = g.step()
        out.append((g.labels().astype(np.int64), g.centroids(), g.counts(), e, e2))
    st = g.stats()
    g.close()
    return out, st


@pytest.mark.parametrize("d,k,n", [(3, 32, 200_003), (3, 17, 70_001), (2, 31, 100_000), (1, 5, 33_333),
                                   (3, 1, 1_000), (2, 32, 255)])
def test_tc_screen_oracle_lockstep(km, oracle, d, k, n):
    x, _, _ = synth.aniso_mixture(n, d, max(k // 2, 1), seed=300 + d * k)
    mu0, _ = synth.init_distinct(x, k, seed=301 + k)
    st = lockstep(km, oracle, x, mu0, steps=3, dist_path="tensor")
    assert st["path"] == 4


def test_tc_screen_equals_ffma2_path(km):
    x, _, _ = synth.aniso_mixture(1_000_037, 3, 24, seed=311)
    mu0, _ = synth.init_kmeanspp(x, 32, seed=312)
    a, sa = _steps(km, x, mu0, "tensor", 4)
    b, sb = _steps(km, x, mu0, "simt", 4)
    assert sa["path"] == 4 and sb["path"] == 1
    for (za, ma, ca, ea, e2a), (zb, mb, cb, eb, e2b) in zip(a, b):
        assert np.array_equal(za, zb) and np.array_equal(ca, cb)
        assert np.array_equal(ma, mb) and ea == eb and e2a == e2b


def test_tc_screen_offset_and_byte_labels(km, oracle):
    x, _, _ = synth.iso_mixture(150_001, 3, 32, sigma=1.0, box=50.0, seed=321, weights="dirichlet", offset=1e4)
    mu0, _ = synth.init_distinct(x, 32, seed=322)
    st = lockstep(km, oracle, x, mu0, steps=2, dist_path="tensor", label_bytes=1)
    assert st["path"] == 4


def test_tc_screen_final_labels_pass(km, oracle):
    x, _, _ = synth.aniso_mixture(120_011, 2, 12, seed=331)
    mu0, _ = synth.init_distinct(x, 16, seed=332)
    d, n = x.shape
    g = km.KMeans(n, d, 16, dist_path="tensor", label_policy="final")
    g.set_points(x)
    g.set_init(mu0)
    r = g.run(20, 1e-9)
    z_ref, _, _, _ = oracle.step(x, r["centroids"])
    assert np.array_equal(r["labels"], z_ref)
    g.close()


def test_tc_screen_refuses_k33(km):
    with pytest.raises(km.KMError):
        km.KMeans(1000, 3, 33, dist_path="tensor")
