"""km_lloyd_step_noalloc: the one entry point that allocates nothing.

Some callers cannot call cudaMalloc (an allocator that must not be entered
after start-up, a real-time loop, a host framework that owns all device
memory); this entry point keeps its scratch in a fixed file-scope device
array and works only on buffers the caller passes.  Here it is called through
the C ABI on caller-owned device buffers and compared with the FP64 oracle
step by step (each call starts from the oracle's previous centroids; two or
more calls in a row, so the shared scratch is reused): labels and counts
bit-exact, centroids within 1e-6 relative, E within 1e-9 absolute.  Its
distance screen is its own (the unshifted FP32 direct form with its own error
bound), so the cases include data offset by 1e4, exact ties and planted near
ties that only the FP64 re-decision settles, empty clusters, K = 1, the
256-column limit of the scratch and a padded row stride.  It must also agree
with km_step (the context-based entry point).  This file is collected last so
that a run stopping at the first failure has run every other test already.
"""
import ctypes
import math

import numpy as np
import pytest

import synth
from test_gpu_parity import assert_centroids_close, E_ABS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as km
    km.build()
    return km, km.lib(), torch


class Buffers:
    """Caller-owned device buffers for one problem (the row stride may exceed N)."""

    def __init__(self, torch, x, k, pad=0):
        d, n = x.shape
        dev = torch.device("cuda")
        self.torch, self.n, self.d, self.k = torch, n, d, k
        self.xt = torch.zeros((d, n + pad), dtype=torch.float32, device=dev)
        self.xt[:, :n] = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        self.ld = n + pad
        self.mu_in = torch.empty((k, d), dtype=torch.float64, device=dev)
        self.labels = torch.empty(n, dtype=torch.int32, device=dev)
        self.mu_out = torch.empty((k, d), dtype=torch.float64, device=dev)
        self.counts = torch.empty(k, dtype=torch.int64, device=dev)
        self.e2 = torch.empty(1, dtype=torch.float64, device=dev)

    def step(self, L, mu):
        torch = self.torch
        self.mu_in.copy_(torch.from_numpy(np.ascontiguousarray(mu, dtype=np.float64)))
        err = ctypes.create_string_buffer(256)
        st = L.km_lloyd_step_noalloc(self.xt.data_ptr(), self.ld, self.n, self.d, self.k, self.mu_in.data_ptr(),
                                     self.labels.data_ptr(), self.mu_out.data_ptr(), self.counts.data_ptr(),
                                     self.e2.data_ptr(), torch.cuda.current_stream().cuda_stream, err, 256)
        assert st == 0, err.value.decode()
        torch.cuda.synchronize()
        return (self.labels.cpu().numpy(), self.mu_out.cpu().numpy(), self.counts.cpu().numpy(),
                float(self.e2.item()))


def lockstep_noalloc(env, oracle, x, mu0, steps=2, pad=0):
    km, L, torch = env
    k = mu0.shape[0]
    b = Buffers(torch, x, k, pad)
    mu = np.array(mu0, dtype=np.float64)
    for t in range(steps):
        z, mo, cnt, e2 = b.step(L, mu)
        z_ref, mu_ref, cnt_ref, e2_ref = oracle.step(x, mu)
        assert np.array_equal(z, z_ref), (t, np.flatnonzero(z != z_ref)[:10])
        assert np.array_equal(cnt, cnt_ref), t
        assert_centroids_close(mo, mu_ref, x)
        assert abs(math.sqrt(e2) - math.sqrt(e2_ref)) <= max(E_ABS, 1e-12 * math.sqrt(e2_ref)), t
        mu = mu_ref
    return mu


@pytest.mark.parametrize("d,k,n,pad", [(3, 16, 300_007, 0), (1, 128, 50_001, 37), (2, 85, 70_003, 0),
                                       (3, 64, 40_000, 5), (3, 1, 10_001, 0)])
def test_noalloc_oracle_lockstep(env, oracle, d, k, n, pad):
    """Shapes up to the 256-column limit (d = 1, K = 128 and d = 3, K = 64),
    a padded row stride, K = 1; three calls in a row."""
    x, _, _ = synth.aniso_mixture(n, d, max(k // 2, 1), seed=100 + d * k)
    mu0, _ = synth.init_distinct(x, k, seed=200 + d * k)
    lockstep_noalloc(env, oracle, x, mu0, steps=3, pad=pad)


def test_noalloc_offset_data(env, oracle):
    """Every coordinate offset by 1e4 (cancellation in the unshifted direct
    form: the error bound sends more points to FP64, the labels stay exact)."""
    x, _, _ = synth.iso_mixture(100_003, 3, 64, sigma=1.0, box=50.0, seed=31, weights="dirichlet", offset=1e4)
    mu0, _ = synth.init_distinct(x, 64, seed=32)
    lockstep_noalloc(env, oracle, x, mu0, steps=2)


def test_noalloc_exact_and_near_ties_and_empty_cluster(env, oracle):
    """Points exactly half-way between two centres (a tie: the lowest k
    wins), points a relative 1e-7 off half-way (a near tie, decided in FP64),
    duplicate centres, and a centre far from every point (an empty cluster
    keeps its centre)."""
    rng = np.random.default_rng(5)
    base = rng.uniform(-5, 5, size=(2000, 2)).astype(np.float32)
    # centres 0 and 1 at (+-1, 0): points on the line x0 = 0 are exact ties
    tie = np.stack([np.zeros(500, np.float32), rng.uniform(-3, 3, 500).astype(np.float32)], axis=1)
    near = tie.copy()
    near[:, 0] = np.float32(1e-7) * rng.choice([-1, 1], 500).astype(np.float32)
    x = np.concatenate([base, tie, near]).T.copy()
    mu0 = np.array([[-1.0, 0.0], [1.0, 0.0], [1.0, 0.0], [0.0, 3.0], [1e3, 1e3]])
    z_ref, _, cnt_ref, _ = oracle.step(x, mu0)
    assert cnt_ref[2] == 0 and cnt_ref[4] == 0  # duplicate (higher index) and far centres stay empty
    mu = lockstep_noalloc(env, oracle, x, mu0, steps=2)
    assert np.array_equal(mu[4], mu0[4])


def test_noalloc_matches_km_step(env):
    """The allocation-free step and the context-based km_step give the same
    labels, counts and centroids (two steps)."""
    km, L, torch = env
    x, _, _ = synth.aniso_mixture(200_003, 3, 12, seed=21)
    k = 16
    mu0, _ = synth.init_kmeanspp(x, k, seed=22)
    d, n = x.shape
    g = km.KMeans(n, d, k)
    g.set_points(x)
    g.set_init(mu0)
    b = Buffers(torch, x, k)
    mu = mu0
    for _ in range(2):
        e, _ = g.step()
        z, mo, cnt, e2 = b.step(L, mu)
        assert np.array_equal(z, g.labels()) and np.array_equal(cnt, g.counts())
        assert_centroids_close(mo, g.centroids(), x)
        assert abs(math.sqrt(e2) - e) <= E_ABS
        mu = g.centroids()
    g.close()


def _call_raw(L, torch, xt, ld, n, d, k):
    dev = torch.device("cuda")
    mu = torch.zeros((k, d), dtype=torch.float64, device=dev)
    labels = torch.empty(max(min(n, 1 << 20), 1), dtype=torch.int32, device=dev)
    mu_out = torch.empty((k, d), dtype=torch.float64, device=dev)
    counts = torch.empty(k, dtype=torch.int64, device=dev)
    e2 = torch.empty(1, dtype=torch.float64, device=dev)
    err = ctypes.create_string_buffer(256)
    st = L.km_lloyd_step_noalloc(xt.data_ptr(), ld, n, d, k, mu.data_ptr(), labels.data_ptr(), mu_out.data_ptr(),
                                 counts.data_ptr(), e2.data_ptr(), torch.cuda.current_stream().cuda_stream, err, 256)
    return st, err.value.decode()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    """K (d + 1) > 256 and N > 304 * 2^19 are refused before any data is read
    (so a small buffer stands in for the oversized point set)."""
    km, L, torch = env
    xt = torch.zeros((3, 1000), dtype=torch.float32, device=torch.device("cuda"))
    st, msg = _call_raw(L, torch, xt, 1000, 1000, 3, 65)  # K*(d+1) = 260
    assert st == -1 and "256" in msg
    big = 304 * 2**19 + 1
    st, msg = _call_raw(L, torch, xt, big, big, 1, 4)
    assert st == -1 and "304 * 2^19" in msg


def test_noalloc_marks_invalid_data(env):
    """A NaN, an infinity or |x| >= 2^99 cannot be held by the fixed-point
    grid: the step marks every centroid and E^2 NaN and every count -1; a
    following call on finite data is exact again."""
    km, L, torch = env
    x = np.random.default_rng(3).normal(size=(2, 5000)).astype(np.float32)
    mu0 = np.array([[-1.0, 0.0], [1.0, 0.0]])
    for bad in (np.nan, np.inf, np.float32(2.0**100)):
        xb = x.copy()
        xb[1, 17] = bad
        b = Buffers(torch, xb, 2)
        _, mo, cnt, e2 = b.step(L, mu0)
        assert np.all(np.isnan(mo)) and math.isnan(e2) and np.all(cnt == -1), bad
    b = Buffers(torch, x, 2)
    _, mo, cnt, _ = b.step(L, mu0)
    assert cnt.sum() == 5000 and np.all(np.isfinite(mo))
