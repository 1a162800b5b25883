"""GPU parity of the batched form: every instance's labels, counts and
iteration count equal the FP64 oracle's run on that instance alone,
centroids within 1e-6 relative and E within 1e-9 absolute."""
import numpy as np
import pytest

import synth
from test_gpu_parity import assert_centroids_close, E_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


def _batch(km, insts, **kw):
    b = km.KMeansBatch([w["n"] for w in insts], [w["d"] for w in insts], [w["k"] for w in insts], **kw)
    b.set_points([w["x"] for w in insts])
    b.set_init([w["mu0"] for w in insts])
    return b


def _check_against_oracle(b, insts, r, oracle, max_iter, tol):
    labs = b.split_labels(r["labels"])
    mus = b.split_centroids(r["centroids"])
    cnts = b.split_counts(b.counts())
    for i, w in enumerate(insts):
        ref = oracle.run(w["x"], w["mu0"], max_iter, tol)
        assert r["iters"][i] == ref["iters"], i
        assert bool(r["converged"][i]) == ref["converged"], i
        assert np.array_equal(labs[i], ref["labels"]), i
        assert np.array_equal(cnts[i], ref["counts"]), i
        assert_centroids_close(mus[i], ref["centroids"], w["x"])
        assert abs(r["E"][i] - ref["E"]) <= E_ABS, i


def test_batch_matches_oracle_per_instance(km, oracle):
    insts = synth.batch_instances(48, seed=5, n_lo=200, n_hi=20_000)
    b = _batch(km, insts)
    r = b.run(100, 1e-6)
    _check_against_oracle(b, insts, r, oracle, 100, 1e-6)
    info = b.info()
    assert info["tuned"] == 1 and info["tile_points"] in (512, 1024, 8192, 32768) and info["tune_candidates"] == 8
    b.close()


@pytest.mark.parametrize("shape", [(512, 128), (1024, 512), (8192, 256), (32768, 256)])
def test_batch_every_shape_matches_oracle(km, oracle, shape):
    """Every launch shape the tuner times gives the oracle's results: the
    batch kernel's tiles, and the fused kernel's tile machinery (tiles of
    8192 and 32768 points: instances of d = 1, 2 and 3 following one another
    in a block, partial tiles, rows not 16-byte aligned in the packed
    layout, labels at odd offsets)."""
    insts = synth.batch_instances(40, seed=15, n_lo=300, n_hi=30_000)
    x1 = np.linspace(-3, 3, 1001, dtype=np.float32)[None, :]
    insts.insert(3, dict(x=x1, mu0=np.array([[-1.0], [0.5], [2.0]]), n=1001, d=1, k=3))
    b = _batch(km, insts)
    b.set_shape(*shape)
    r = b.run(60, 1e-6)
    _check_against_oracle(b, insts, r, oracle, 60, 1e-6)
    info = b.info()
    assert (info["tile_points"], info["threads"]) == shape
    b.close()


def test_batch_one_step_and_edges(km, oracle):
    """One step (max_iter = 1), plus the degenerate shapes: K = 1, K = N
    (each point its own cluster), an instance of duplicated points (exact
    ties decided by the lowest index) and d = 1."""
    insts = synth.batch_instances(6, seed=9, n_lo=300, n_hi=3_000)
    x1 = np.linspace(-3, 3, 17, dtype=np.float32)[None, :]
    insts.append(dict(x=x1, mu0=np.array([[0.0]]), n=17, d=1, k=1))
    xs = np.random.default_rng(3).normal(size=(2, 40)).astype(np.float32)
    insts.append(dict(x=xs, mu0=xs.T.astype(np.float64), n=40, d=2, k=40))
    xd = np.repeat(np.array([[0, 4], [0, 0], [0, 0]], dtype=np.float32), 50, axis=1)
    insts.append(dict(x=xd, mu0=np.array([[2.0, 0, 0], [2.0, 0, 0], [-1.0, 0, 0]]), n=100, d=3, k=3))
    b = _batch(km, insts, use_graph=False)
    r = b.run(1, 0.0)
    _check_against_oracle(b, insts, r, oracle, 1, 0.0)
    b.close()


def test_batch_graph_and_plain_loops_agree_and_resume(km, oracle):
    insts = synth.batch_instances(12, seed=2, n_lo=500, n_hi=8_000)
    b1 = _batch(km, insts)
    r1 = b1.run(40, 1e-6)
    b2 = _batch(km, insts, use_graph=False)
    r2 = b2.run(40, 1e-6)
    assert np.array_equal(r1["labels"], r2["labels"]) and np.array_equal(r1["centroids"], r2["centroids"])
    assert np.array_equal(r1["iters"], r2["iters"])
    # 3 steps, then up to 37 more, continue the same iterations: centroids
    # equal the one-run result (a converged fixed point stays fixed), and an
    # instance still running after 3 steps takes the same total count
    b3 = _batch(km, insts)
    b3.run(3, 1e-6)
    r3 = b3.run(37, 1e-6)
    assert np.array_equal(r3["centroids"], r1["centroids"])
    assert np.array_equal(r3["labels"], r1["labels"])
    late = r1["iters"] > 3
    assert np.array_equal(r3["iters"][late], r1["iters"][late])
    for c in (b1, b2, b3):
        c.close()


def test_tuner_cache_reuses_the_shape(km, oracle, tmp_path):
    """The tuner's choice is kept in a cache file keyed by the device and the
    instance sizes; a second batch of the same sizes takes it without timing
    and gives the same results."""
    insts = [synth.batch_instance(i, n, d, k) for i, (n, d, k) in
             enumerate([(3000, 2, 5), (12000, 3, 17), (700, 3, 4)])]
    cache = str(tmp_path / "tune.json")
    b1 = _batch(km, insts)
    shape1 = b1.tune(cache=cache)
    assert len(b1.info()["tune_ms"]) == 8
    r1 = b1.run(100, 1e-6)
    b1.close()
    b2 = _batch(km, insts)
    shape2 = b2.tune(cache=cache)
    assert shape2 == shape1 and b2.info()["tune_ms"] == []
    r2 = b2.run(100, 1e-6)
    assert np.array_equal(r1["labels"], r2["labels"]) and np.array_equal(r1["centroids"], r2["centroids"])
    _check_against_oracle(b2, insts, r2, oracle, 100, 1e-6)
    b2.close()
    with pytest.raises(km.KMError):
        b3 = _batch(km, insts)
        try:
            b3._check(b3._L.km_batch_set_shape(b3._h, 768, 256))
        finally:
            b3.close()


def test_batch_objective_matches_the_oracle(km, oracle):
    """Per-instance objective of the final labels and centroids against the
    oracle's objective of its own final state (FP64, summation orders
    differ: 1e-12 relative)."""
    insts = synth.batch_instances(12, seed=21, n_lo=300, n_hi=8_000)
    b = _batch(km, insts)
    r = b.run(100, 1e-6)
    objs = b.objective()
    for i, w in enumerate(insts):
        ref = oracle.run(w["x"], w["mu0"], 100, 1e-6)
        assert abs(objs[i] - ref["objective"]) <= 1e-12 * max(ref["objective"], 1.0), i
    b.close()


@pytest.mark.parametrize("scale", [1e-30, 1e20])
def test_batch_extreme_magnitudes(km, oracle, scale):
    """Instances with coordinates near FP32's underflow or whose squared
    distances overflow FP32: every instance still equals the oracle's run."""
    insts = synth.batch_instances(5, seed=31, n_lo=300, n_hi=2_000)
    for w in insts:
        w["x"] = (w["x"].astype(np.float64) * scale).astype(np.float32)
        w["mu0"] = w["x"][:, :w["k"]].T.astype(np.float64).copy()
    b = _batch(km, insts)
    r = b.run(30, 0.0)
    _check_against_oracle(b, insts, r, oracle, 30, 0.0)
    b.close()
