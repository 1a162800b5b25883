"""Host-side logic that needs no GPU: the bench's traffic lookup and
roofline helpers, the learned initialiser's parameter layout (against the
oracle's), and the paper-size sweep's shapes."""
import json
import os

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_profiled_traffic_scales_and_checks_the_source(monkeypatch, tmp_path):
    import bench
    rec = [{"kernel": "assign_fast_kernel<3>", "n": 1000, "d": 3, "k": 32, "dram_bytes_per_launch": 5000.0,
            "source_sha": "abc"}]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda files=None: "abc")
    assert bench.profiled_traffic("assign_fast_kernel<3>", 4000, 32, 3) == 20000.0   # scaled by N
    assert bench.profiled_traffic("assign_fast_kernel<3>", 4000, 64, 3) is None      # another K
    assert bench.profiled_traffic("other_kernel", 4000, 32, 3) is None
    monkeypatch.setattr(bench, "source_hash", lambda files=None: "changed")
    assert bench.profiled_traffic("assign_fast_kernel<3>", 4000, 32, 3) is None      # kernel changed since


def test_committed_traffic_records_name_their_commands():
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert {r["kernel"] for r in recs} >= {"assign_fast_kernel<3>", "gemm_assign_kernel"}
    for r in recs:
        assert r["command"].startswith("ncu ") and "--clock-control none" in r["command"]
        assert r["dram_bytes_per_launch"] == r["dram_read_bytes"] + r["dram_write_bytes"]


def test_whole_job_value_and_peaks():
    import bench
    assert bench.whole_job_value(100, 8, 10, 2, 1000.0) == 100 * 8 * 10 * 2
    pk, src = bench.peaks()
    assert src in ("measured", "fallback") and float(pk.get("hbm_gbs", 6800.0)) > 0


def test_learned_parameter_layout_matches_the_oracle():
    from paper_2405_12052_gb300 import learned
    from oracle import setnet
    flat = learned.init_params(3, 16, seed=4)
    shapes = setnet.shapes(3, 16)
    assert flat.size == sum(int(np.prod(s)) for s in shapes.values())
    p = setnet.unflatten(flat.astype(np.float64), 3, 16)
    for name in ("b1", "b2", "b3", "b4"):
        assert not p[name].any()                       # zero biases
    for name, (rows, cols) in (("W1", (128, 3)), ("W2", (128, 128)), ("W3", (128, 128)), ("W4", (48, 128))):
        w = p[name]
        assert w.shape == (rows, cols)
        assert np.abs(w).max() <= np.sqrt(6.0 / cols) + 1e-6   # He-uniform on the fan-in


def test_paper_sweep_shapes():
    cases = synth.paper_sweep()
    assert ("2d", 100_000, 8) in cases and ("3d", 1_000_000, 4) in cases and ("3d", 1_000_000, 11) in cases
    w = synth.sweep_case("3d", 2_000, 4)
    assert w["x"].shape == (3, 2_000) and w["mu0"].shape == (4, 3) and w["x"].dtype == np.float32
