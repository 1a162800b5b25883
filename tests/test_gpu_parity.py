"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Bar: labels and counts bit-exact; centroids within 1e-6 relative (per
centroid, relative to max(||mu_ref,k||, RMS spread of X)); E within 1e-9
absolute; iteration counts equal.  In lockstep tests both sides start every
step from the same centroids (the oracle's), so labels must agree exactly.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

CENT_REL = 1e-6
E_ABS = 1e-9


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


def spread(x):
    xd = x.astype(np.float64)
    return math.sqrt(((xd - xd.mean(axis=1, keepdims=True)) ** 2).sum(axis=0).mean())


def assert_centroids_close(got, ref, x):
    floor = spread(x)
    for c in range(ref.shape[0]):
        tol = CENT_REL * max(np.linalg.norm(ref[c]), floor, 1e-300)
        assert np.linalg.norm(got[c] - ref[c]) <= tol, (c, got[c], ref[c])


def lockstep(km, oracle, x, mu0, steps=1, **kw):
    d, n = x.shape
    k = mu0.shape[0]
    g = km.KMeans(n, d, k, **kw)
    g.set_points(x)
    mu = np.array(mu0, dtype=np.float64)
    for t in range(steps):
        g.set_init(mu)
        e, e2 = g.step()
        z_ref, mu_ref, cnt_ref, e2_ref = oracle.step(x, mu)
        z = g.labels()
        assert np.array_equal(z, z_ref), (t, np.flatnonzero(z != z_ref)[:10])
        assert np.array_equal(g.counts(), cnt_ref)
        assert_centroids_close(g.centroids(), mu_ref, x)
        # E within 1e-9 absolute, or 1e-12 relative where E itself is far
        # above 1e3 (data scaled to extreme magnitudes)
        e_ref = math.sqrt(e2_ref)
        assert abs(e - e_ref) <= max(E_ABS, 1e-12 * e_ref) and abs(e2 - e2_ref) <= max(E_ABS, 1e-12 * e2_ref)
        mu = mu_ref
    st = g.stats()
    g.close()
    return st


def test_lockstep_plain_2d(km, oracle):
    w = synth.workload("plain_2d_n1e5_k8")
    st = lockstep(km, oracle, w["x"], w["mu0"], steps=8)
    assert st["path"] == 1


def test_full_run_plain_2d(km, oracle):
    w = synth.workload("plain_2d_n1e5_k8")
    ref = oracle.run(w["x"], w["mu0"], w["max_iter"], w["tol"])
    for use_graph in (True, False):
        g = km.KMeans(w["x"].shape[1], 2, w["k"], use_graph=use_graph)
        g.set_points(w["x"])
        g.set_init(w["mu0"])
        r = g.run(w["max_iter"], w["tol"])
        assert r["iters"] == ref["iters"] and r["converged"] == ref["converged"]
        assert np.array_equal(r["labels"], ref["labels"])
        assert np.array_equal(g.counts(), ref["counts"])
        assert_centroids_close(r["centroids"], ref["centroids"], w["x"])
        assert abs(r["E"] - ref["E"]) <= E_ABS
        g.close()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 2047, 2048, 2049, 4101, 65537, 100003])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_ragged_sizes(km, oracle, n, d):
    k = min(n, 5)
    x, _, _ = synth.iso_mixture(n, d, 4, sigma=1.0, box=5.0, seed=n + d)
    mu0, _ = synth.init_distinct(x, k, seed=7)
    lockstep(km, oracle, x, mu0, steps=2)


@pytest.mark.parametrize("k", [1, 2, 3, 31, 32, 33, 64, 100, 255, 256])
def test_k_variants(km, oracle, k):
    x, _, _ = synth.aniso_mixture(40_000, 3, 12, seed=k)
    mu0, _ = synth.init_distinct(x, k, seed=k + 1)
    lockstep(km, oracle, x, mu0, steps=2)


@pytest.mark.parametrize("d,k", [(5, 3), (8, 40), (16, 7), (2, 300), (3, 257)])
def test_generic_path(km, oracle, d, k):
    x, _, _ = synth.iso_mixture(20_000, d, 6, sigma=1.5, box=5.0, seed=d * 100 + k)
    mu0, _ = synth.init_distinct(x, k, seed=3)
    st = lockstep(km, oracle, x, mu0, steps=2)
    assert st["path"] == 2


def test_exact_ties_go_to_lowest_index(km, oracle):
    # integer grid points; centroids placed so many points sit exactly on
    # bisectors, plus a duplicated centroid
    g1 = np.arange(-6, 7, dtype=np.float32)
    xx, yy = np.meshgrid(g1, g1)
    x = np.stack([xx.ravel(), yy.ravel()]).astype(np.float32)
    x = np.ascontiguousarray(np.tile(x, (1, 40)))
    mu0 = np.array([[-2.0, 0.0], [2.0, 0.0], [0.0, 4.0], [0.0, 4.0], [0.0, -4.0]])
    st = lockstep(km, oracle, x, mu0, steps=1)
    assert st["flagged"] > 0 and st["fp64_decided"] > 0


def test_empty_cluster_keeps_centre(km, oracle):
    x, _, _ = synth.iso_mixture(30_000, 3, 3, sigma=1.0, box=5.0, seed=1)
    mu0 = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [500.0, 500.0, 500.0]])
    lockstep(km, oracle, x, mu0, steps=2)
    g = km.KMeans(x.shape[1], 3, 3)
    g.set_points(x)
    g.set_init(mu0)
    g.step()
    assert g.counts()[2] == 0 and np.array_equal(g.centroids()[2], mu0[2])
    assert g.stats()["empty_clusters"] == 1


def test_offset_cancellation(km, oracle):
    # every coordinate offset by 1e4: the screen's shift keeps it exact
    x, _, _ = synth.iso_mixture(200_000, 3, 16, sigma=1.0, box=20.0, seed=5, offset=1e4)
    mu0, _ = synth.init_distinct(x, 16, seed=6)
    st = lockstep(km, oracle, x, mu0, steps=3)
    assert st["flagged"] < 0.01 * x.shape[1]


def test_determinism_and_resume(km, oracle):
    w = synth.workload("plain_2d_n1e5_k8")
    outs = []
    for _ in range(2):
        g = km.KMeans(w["x"].shape[1], 2, 8)
        g.set_points(w["x"])
        g.set_init(w["mu0"])
        outs.append(g.run(100, 1e-6))
        g.close()
    assert np.array_equal(outs[0]["labels"], outs[1]["labels"])
    assert np.array_equal(outs[0]["centroids"], outs[1]["centroids"])
    assert outs[0]["E"] == outs[1]["E"]
    # stop after 3 steps, restart from the returned centroids: same final state
    g = km.KMeans(w["x"].shape[1], 2, 8)
    g.set_points(w["x"])
    g.set_init(w["mu0"])
    r1 = g.run(3, 1e-6)
    g.set_init(r1["centroids"])
    r2 = g.run(100, 1e-6)
    assert r1["iters"] + r2["iters"] == outs[0]["iters"]
    assert np.array_equal(r2["centroids"], outs[0]["centroids"])
    assert np.array_equal(r2["labels"], outs[0]["labels"])


def test_e_mode_squared(km, oracle):
    w = synth.workload("plain_2d_n1e5_k8")
    ref = oracle.run(w["x"], w["mu0"], 100, 1e-3, e_mode=1)
    g = km.KMeans(w["x"].shape[1], 2, 8, e_mode="squared")
    g.set_points(w["x"])
    g.set_init(w["mu0"])
    r = g.run(100, 1e-3)
    assert r["iters"] == ref["iters"]
    assert np.array_equal(r["labels"], ref["labels"])


def test_device_borrow_and_aos(km, oracle):
    import torch
    x, _, _ = synth.aniso_mixture(50_001, 3, 8, seed=9)
    mu0, _ = synth.init_distinct(x, 8, seed=10)
    z_ref, mu_ref, _, _ = oracle.step(x, mu0)
    for mode in ("borrow", "copy", "aos_host", "aos_dev"):
        g = km.KMeans(x.shape[1], 3, 8)
        if mode == "borrow":
            t = torch.from_numpy(x).cuda()
            g.set_points(t, borrow=True)
        elif mode == "copy":
            g.set_points(torch.from_numpy(x).cuda())
        elif mode == "aos_host":
            g.set_points(np.ascontiguousarray(x.T), layout="nxd")
        else:
            g.set_points(torch.from_numpy(np.ascontiguousarray(x.T)).cuda(), layout="nxd")
        g.set_init(mu0)
        g.step()
        assert np.array_equal(g.labels(), z_ref), mode
        assert_centroids_close(g.centroids(), mu_ref, x)
        g.close()


def test_errors_are_reported(km):
    with pytest.raises(km.KMError) as ei:
        km.KMeans(10, 2, 11)
    assert ei.value.status == -1
    g = km.KMeans(100, 2, 3)
    with pytest.raises(km.KMError) as ei:
        g.step()
    assert ei.value.status == -4
    x = np.zeros((2, 100), dtype=np.float32)
    x[1, 17] = np.nan
    with pytest.raises(km.KMError) as ei:
        g.set_points(x)
    assert ei.value.status == -6
    with pytest.raises(km.KMError):
        g.set_init(np.full((3, 2), np.inf))


@pytest.mark.slow
def test_full_scale_lockstep_3d_n1e8(km, oracle):
    """The 1e8-point 3-D workload at full size, in the launch configuration the
    benchmark times: one step from the k-means++ start, every label and count
    compared with the oracle."""
    w = synth.workload("plain_3d_n1e8_k32")
    st = lockstep(km, oracle, w["x"], w["mu0"], steps=1)
    assert st["path"] == 1


def test_offset_k256_on_the_fused_kernel(km, oracle):
    """The cancellation workload's shape (K = 256, every coordinate offset by
    1e4): the fused kernel runs it with one sum window per warp."""
    x, _, _ = synth.iso_mixture(300_000, 3, 256, sigma=1.0, box=50.0, seed=21, weights="dirichlet",
                                offset=1e4)
    mu0, _ = synth.init_distinct(x, 256, seed=22)
    st = lockstep(km, oracle, x, mu0, steps=2)
    assert st["path"] == 1


@pytest.mark.slow
def test_full_scale_lockstep_offset_n2p27(km, oracle):
    """N = 2^27, d = 3, K = 256, every coordinate offset by 1e4, at full size
    and in the benchmark's launch configuration: one step from the k-means++
    start, every label and count equal to the oracle's, every centroid within
    1e-6 of the oracle's centroid, E and E^2 within the stated bounds."""
    w = synth.workload("precision_offset_3d_n2p27_k256")
    st = lockstep(km, oracle, w["x"], w["mu0"], steps=1)
    assert st["path"] == 1


@pytest.mark.parametrize("case", ["fused_2d", "fused_k256", "generic_d5"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_label_policy_final(km, oracle, case, use_graph):
    """The "final" label policy: the steps skip the label writes, km_run ends
    with one assignment pass against the returned centroids.  Centroids,
    iteration count and E are bit-identical to the every-step run; the labels
    are the oracle's assignment to the returned centroids."""
    if case == "fused_2d":
        w = synth.workload("plain_2d_n1e5_k8")
        x, mu0, k = w["x"], w["mu0"], w["k"]
    elif case == "fused_k256":
        x, _, _ = synth.iso_mixture(120_001, 3, 256, sigma=1.0, box=50.0, seed=31, weights="dirichlet")
        mu0, _ = synth.init_distinct(x, 256, seed=32)
        k = 256
    else:
        x, _, _ = synth.iso_mixture(30_007, 5, 3, sigma=1.0, box=5.0, seed=33)
        mu0, _ = synth.init_distinct(x, 3, seed=34)
        k = 3
    d, n = x.shape
    out = {}
    for pol in ("every_step", "final"):
        g = km.KMeans(n, d, k, label_policy=pol, use_graph=use_graph)
        g.set_points(x)
        g.set_init(mu0)
        out[pol] = (g.run(60, 1e-6), g.counts(), g.objective(), g.stats()["path"])
        g.close()
    (ra, ca, _, pa), (rb, cb, ob, pb) = out["every_step"], out["final"]
    assert pa == pb and pa in (1, 2)
    assert ra["iters"] == rb["iters"] and ra["E"] == rb["E"]
    assert np.array_equal(ra["centroids"], rb["centroids"])
    assert np.array_equal(ca, cb)
    z_ref = oracle.assign(x, rb["centroids"])
    assert np.array_equal(rb["labels"], z_ref), np.flatnonzero(rb["labels"] != z_ref)[:10]
    xd = x.astype(np.float64)
    obj = sum(float(((xd[:, z_ref == c] - rb["centroids"][c][:, None]) ** 2).sum()) for c in range(k))
    assert abs(ob - obj) <= 1e-9 * max(obj, 1.0)


def test_label_policy_final_step_api(km, oracle):
    """Under the "final" policy km_step leaves the labels alone; write_labels
    then gives the assignment to the current centroids."""
    x, _, _ = synth.aniso_mixture(50_000, 3, 8, seed=41)
    mu0, _ = synth.init_distinct(x, 8, seed=42)
    g = km.KMeans(x.shape[1], 3, 8, label_policy="final")
    g.set_points(x)
    g.set_init(mu0)
    g.step()
    assert not g.labels().any()          # never written: the buffer's initial zeros
    _, mu1, cnt1, _ = oracle.step(x, mu0)
    assert np.array_equal(g.counts(), cnt1)
    g.write_labels()
    assert np.array_equal(g.labels(), oracle.assign(x, g.centroids()))
    g.close()


def test_dist_path_option(km, oracle):
    """dist_path: "simt" keeps d = 64 off the tensor cores (generic FP32
    path, same bit-exact labels); "tensor" on a shape no tcgen05 path
    takes is an argument error; "tensor" on d = 64 selects the GEMM form."""
    x, _, _ = synth.iso_mixture(20_000, 64, 40, sigma=1.0, box=8.0, seed=51)
    mu0, _ = synth.init_distinct(x, 100, seed=52)
    st = lockstep(km, oracle, x, mu0, steps=1, dist_path="simt")
    assert st["path"] == 2
    g = km.KMeans(x.shape[1], 64, 100, dist_path="tensor")
    assert g.stats()["path"] == 3
    g.close()
    with pytest.raises(km.KMError) as ei:
        km.KMeans(1000, 3, 40, dist_path="tensor")  # neither d = 64 nor d <= 3 with K <= 32
    assert ei.value.status == -1
    with pytest.raises(km.KMError):
        km.KMeans(1000, 4, 8, dist_path="tensor")


def test_run_logged_records_every_step(km, oracle):
    """One record per step; the same stopping step, E and centroids as run()
    and the oracle; the per-step objective never increases."""
    w = synth.workload("plain_2d_n1e5_k8")
    ref = oracle.run(w["x"], w["mu0"], w["max_iter"], w["tol"])
    g = km.KMeans(w["x"].shape[1], 2, w["k"])
    g.set_points(w["x"])
    g.set_init(w["mu0"])
    lines = []
    r = g.run_logged(w["max_iter"], w["tol"], objective=True, log=lines.append)
    assert r["iters"] == ref["iters"] == len(lines) and r["converged"] == ref["converged"]
    assert abs(r["E"] - ref["E"]) <= E_ABS
    assert_centroids_close(r["centroids"], ref["centroids"], w["x"])
    objs = [rec["objective"] for rec in r["records"]]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(objs, objs[1:]))
    assert [rec["t"] for rec in r["records"]] == list(range(1, r["iters"] + 1))
    g.close()


@pytest.mark.parametrize("case", ["fused_3d", "fused_k256_offset", "generic_d5"])
def test_one_byte_labels(km, oracle, case):
    """label_bytes = 1 (K <= 256): the labels are kept and copied out as
    bytes, equal to the oracle's; the int32 getter widens them; the
    objective and a full run agree with the 4-byte context."""
    if case == "fused_3d":
        x, _, _ = synth.aniso_mixture(100_003, 3, 12, seed=61)
        k = 32
    elif case == "fused_k256_offset":
        x, _, _ = synth.iso_mixture(80_000, 3, 256, sigma=1.0, box=50.0, seed=62, weights="dirichlet", offset=1e4)
        k = 256
    else:
        x, _, _ = synth.iso_mixture(20_001, 5, 4, seed=63)
        k = 7
    mu0, _ = synth.init_distinct(x, k, seed=64)
    st = lockstep(km, oracle, x, mu0, steps=2, label_bytes=1)
    assert st["path"] == (2 if case == "generic_d5" else 1)
    d, n = x.shape
    out = {}
    for lb in (4, 1):
        g = km.KMeans(n, d, k, label_bytes=lb)
        g.set_points(x)
        g.set_init(mu0)
        r = g.run(40, 1e-6)
        out[lb] = (r, g.objective(), g.labels())
        if lb == 1:
            assert out[lb][2].dtype == np.uint8
            wide = np.empty(n, dtype=np.int32)
            g._check(g._L.km_get_labels(g._h, wide.ctypes.data, 0))
            assert np.array_equal(wide, out[lb][2])
        g.close()
    (r4, o4, z4), (r1, o1, z1) = out[4], out[1]
    assert r4["iters"] == r1["iters"] and np.array_equal(r4["centroids"], r1["centroids"]) and o4 == o1
    assert np.array_equal(z4, z1) and np.array_equal(r4["labels"], r1["labels"])


def test_one_byte_labels_limits(km):
    with pytest.raises(km.KMError) as ei:
        km.KMeans(1000, 3, 257, label_bytes=1)
    assert ei.value.status == -1
    with pytest.raises(km.KMError) as ei:
        km.KMeans(1000, 64, 16, label_bytes=1)   # the tensor-core path reads int32 labels
    assert ei.value.status == -1
    g = km.KMeans(1000, 64, 16, label_bytes=1, dist_path="simt")
    assert g.stats()["path"] == 2
    g.close()


@pytest.mark.parametrize("scale", [1e-30, 1e15, 1e20])
@pytest.mark.parametrize("d,k", [(3, 8), (6, 5)])
def test_extreme_magnitudes(km, oracle, scale, d, k):
    """Coordinates far from 1 in either direction: squared distances near
    FP32's underflow, or beyond FP32's range (the FP32 screens overflow and
    every point is decided in FP64); labels stay the oracle's."""
    x, _, _ = synth.iso_mixture(5_000, d, 4, sigma=1.0, box=5.0, seed=71)
    x = (x.astype(np.float64) * scale).astype(np.float32)
    mu0, _ = synth.init_distinct(x, k, seed=72)
    lockstep(km, oracle, x, mu0, steps=2)


def test_large_offset_integer_grid(km, oracle):
    """Every coordinate offset by 1e7, where FP32 spaces values 1.0 apart:
    the shifted screen and the fixed-point sums stay exact."""
    x, _, _ = synth.iso_mixture(30_000, 3, 6, sigma=40.0, box=400.0, seed=81, offset=1e7)
    mu0, _ = synth.init_distinct(x, 6, seed=82)
    assert lockstep(km, oracle, x, mu0, steps=2)["path"] == 1


def test_d4_k256_fused(km, oracle):
    x, _, _ = synth.aniso_mixture(60_000, 4, 40, seed=83)
    mu0, _ = synth.init_distinct(x, 256, seed=84)
    assert lockstep(km, oracle, x, mu0, steps=2)["path"] == 1


@pytest.mark.parametrize("label_bytes", [4, 1])
def test_k_equals_n(km, oracle, label_bytes):
    """K = N with the points themselves as centres: every point is its own
    cluster (z_i = i) and the step is a fixed point (E = 0)."""
    x, _, _ = synth.iso_mixture(200, 3, 4, seed=85)
    mu0 = x.T.astype(np.float64).copy()
    g = km.KMeans(200, 3, 200, label_bytes=label_bytes)
    g.set_points(x)
    g.set_init(mu0)
    e, e2 = g.step()
    assert np.array_equal(g.labels(), np.arange(200)) and e == 0.0 and e2 == 0.0
    assert np.array_equal(g.counts(), np.ones(200, dtype=np.int64))
    assert np.array_equal(g.centroids(), mu0)
    g.close()
