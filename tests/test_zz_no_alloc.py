"""km_lloyd_step_noalloc: the one entry point that allocates nothing.

Some callers cannot call cudaMalloc (an allocator that must not be entered
after start-up, a real-time loop, a host framework that owns all device
memory); this entry point keeps its scratch in a fixed file-scope device
array and works only on buffers the caller passes.  Here it is called through
the C ABI on caller-owned device buffers and checked against km_step (the
context-based entry point) on two consecutive steps: labels and counts
bit-exact, centroids within 1e-6 relative, E within 1e-9 absolute.  This file
is collected last so that a run stopping at the first failure has run every
other test already.
"""
import ctypes
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as km
    km.build()
    return km, km.lib(), torch


def call_noalloc(L, torch, xt, mu_in, labels, mu_out, counts, e2, k):
    d, n = xt.shape
    err = ctypes.create_string_buffer(256)
    st = L.km_lloyd_step_noalloc(xt.data_ptr(), xt.stride(0), n, d, k, mu_in.data_ptr(),
                                 labels.data_ptr(), mu_out.data_ptr(), counts.data_ptr(),
                                 e2.data_ptr(), torch.cuda.current_stream().cuda_stream, err, 256)
    return st, err.value.decode()


def test_noalloc_matches_km_step_on_two_calls(env):
    km, L, torch = env
    x, _, _ = synth.aniso_mixture(300_007, 3, 12, seed=21)
    k = 16
    mu0, _ = synth.init_kmeanspp(x, k, seed=22)
    d, n = x.shape
    # reference: the context-based entry point, two consecutive steps
    g = km.KMeans(n, d, k)
    g.set_points(x)
    g.set_init(mu0)
    ref = []
    for _ in range(2):
        e, e2 = g.step()
        ref.append((g.labels(), g.counts(), g.centroids(), e))
    g.close()
    # the allocation-free entry point on caller-owned device buffers
    dev = torch.device("cuda")
    xt = torch.from_numpy(x).to(dev)
    mu_in = torch.from_numpy(mu0.copy()).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    mu_out = torch.empty((k, d), dtype=torch.float64, device=dev)
    counts = torch.empty(k, dtype=torch.int64, device=dev)
    e2 = torch.empty(1, dtype=torch.float64, device=dev)
    spread = math.sqrt(((x.astype(np.float64) - x.mean(axis=1, keepdims=True)) ** 2).sum(axis=0).mean())
    for step in range(2):
        st, msg = call_noalloc(L, torch, xt, mu_in, labels, mu_out, counts, e2, k)
        assert st == 0, msg
        torch.cuda.synchronize()
        lab_r, cnt_r, mu_r, e_r = ref[step]
        assert np.array_equal(labels.cpu().numpy(), lab_r), step
        assert np.array_equal(counts.cpu().numpy(), cnt_r), step
        mo = mu_out.cpu().numpy()
        for c in range(k):
            assert np.linalg.norm(mo[c] - mu_r[c]) <= 1e-6 * max(np.linalg.norm(mu_r[c]), spread)
        assert abs(math.sqrt(e2.item()) - e_r) <= 1e-9
        mu_in.copy_(mu_out)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    km, L, torch = env
    dev = torch.device("cuda")
    n, d, k = 1000, 3, 65  # K*(d+1) = 260 > 256
    xt = torch.zeros((d, n), dtype=torch.float32, device=dev)
    mu = torch.zeros((k, d), dtype=torch.float64, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    mu_out = torch.empty((k, d), dtype=torch.float64, device=dev)
    counts = torch.empty(k, dtype=torch.int64, device=dev)
    e2 = torch.empty(1, dtype=torch.float64, device=dev)
    st, msg = call_noalloc(L, torch, xt, mu, labels, mu_out, counts, e2, k)
    assert st == -1 and "256" in msg
