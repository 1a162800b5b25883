"""The oracle against facts that do not come from it (CPU only)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle_pins as P


def test_hand_worked(oracle):
    P.pin_hand_worked(oracle)


def test_ties(oracle):
    P.pin_ties(oracle)


def test_brute_force(oracle):
    P.pin_brute_force(oracle)


def test_closed_forms(oracle):
    P.pin_closed_forms(oracle)


def test_invariants(oracle):
    P.pin_invariants(oracle)


def test_planted_means(oracle):
    P.pin_planted_means(oracle)


def test_sklearn_same_fixed_point(oracle):
    """scikit-learn's Lloyd (GEMM-form distances, its own sums) reaches the same
    fixed point from the same start on well-separated data."""
    sk = pytest.importorskip("sklearn.cluster")
    import synth
    x, comp, means = synth.iso_mixture(30_000, 3, 5, sigma=1.0, box=40.0, seed=3)
    mu0, _ = synth.init_distinct(x, 5, seed=4)
    r = oracle.run(x, mu0, max_iter=300, tol=1e-12)
    km = sk.KMeans(n_clusters=5, init=mu0, n_init=1, algorithm="lloyd", tol=0.0, max_iter=300)
    km.fit(x.T.astype(np.float64))
    assert np.array_equal(km.labels_, r["labels"])
    assert np.allclose(km.cluster_centers_, r["centroids"], rtol=0, atol=1e-9)


def test_thread_count_independent(oracle, tmp_path):
    """Fixed chunking makes every output bit-identical for 1 thread and for all
    threads."""
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r); import synth, oracle;"
        "x,_,_ = synth.iso_mixture(300_000, 3, 9, sigma=1.5, box=6.0, seed=2);"
        "mu0,_ = synth.init_distinct(x, 9, seed=3);"
        "r = oracle.default().run(x, mu0, 30, 1e-9);"
        "np.savez(%r, z=r['labels'], mu=r['centroids'], e=r['E'], it=r['iters'])"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", str(max(2, os.cpu_count() or 2))):
        f = str(tmp_path / f"o{nt}.npz")
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        subprocess.check_call([sys.executable, "-c", code % (root, f)], env=env)
        outs.append(np.load(f))
    a, b = outs
    for key in ("z", "mu", "e", "it"):
        assert np.array_equal(a[key], b[key]), key


def test_kmeanspp_closed_form(oracle):
    """k-means++ with given uniforms: first index floor(u0 N); later indices are
    the first whose running sum of D^2 exceeds u_c * total."""
    x = np.array([[0.0, 1.0, 3.0]], dtype=np.float32)
    # first = floor(0 * 3) = 0; D^2 = (0, 1, 9), total 10
    mu, idx = oracle.kmeanspp(x, 2, [0.0, 0.05])     # target 0.5 -> index 1
    assert list(idx) == [0, 1] and mu[1, 0] == 1.0
    mu, idx = oracle.kmeanspp(x, 2, [0.0, 0.5])      # target 5 -> index 2
    assert list(idx) == [0, 2]
    mu, idx = oracle.kmeanspp(x, 2, [0.99, 0.0])     # first = floor(2.97) = 2; D^2 = (9, 4, 0)
    assert idx[0] == 2 and idx[1] == 0               # target 0: first running sum > 0 is index 0
    mu, idx = oracle.kmeanspp(x, 3, [0.0, 0.5, 0.9])  # after {0, 3}: D^2 = (0, 1, 0)
    assert list(idx) == [0, 2, 1]
