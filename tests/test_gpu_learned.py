"""What the trained set network gains, and what the fallback guarantees.

* Training on the GPU kernels lowers the held-out Chamfer loss.
* The committed network (trained on 200,000 mixtures) has a lower held-out
  loss than the untrained one.
* Learned start + Lloyd with the k-means++ fallback never ends with an
  objective above the k-means++ result's (beyond 1e-6 relative); the
  iterations and objectives of both starts are printed."""
import json
import os

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


def test_training_lowers_the_held_out_loss(km):
    from paper_2405_12052_gb300 import learned
    x, means = learned.mixtures(2048 + 64, S=1024, seed=77)
    t, _ = learned.converged_targets(x, means)
    xv, tv = x[2048:].contiguous(), t[2048:].contiguous()
    net0 = km.SetNet(3, 16)
    net0.set_params(learned.init_params(3, 16, seed=0))
    l0 = net0.loss_grad(xv, tv)
    net, hist = learned.train(x[:2048], t[:2048], epochs=4, batch=32, lr=2e-3, log_every=10_000, log=lambda s: None)
    l1 = net.loss_grad(xv, tv)
    assert l1 < 0.8 * l0, (l0, l1)


def test_committed_network_and_fallback(km, oracle):
    from paper_2405_12052_gb300 import learned
    if not os.path.exists(learned.WEIGHTS):
        pytest.skip("no committed weights")
    net = learned.load()
    x, means = learned.mixtures(256, seed=31337)
    t, _ = learned.converged_targets(x, means)
    untrained = km.SetNet(3, 16)
    untrained.set_params(learned.init_params(3, 16, seed=0))
    assert net.loss_grad(x, t) < 0.7 * untrained.loss_grad(x, t)
    report = []
    for s in range(3):
        xs = synth.aniso_mixture(200_000, 3, 16, seed=950 + s)[0]
        g = km.KMeans(200_000, 3, 16)
        g.set_points(xs)
        u = np.random.default_rng(s).random(16)
        r = learned.run_with_fallback(g, net, u, seed=s)
        kept = min(r["objective_learned"], r["objective_kpp"]) if r["used"] == "learned" else r["objective_kpp"]
        assert kept <= r["objective_kpp"] * (1 + 1e-6)
        assert (r["used"] == "learned") == (r["objective_learned"] <= r["objective_kpp"] * (1 + 1e-6))
        report.append({k: v for k, v in r.items() if k != "centroids"})
        g.close()
    print(json.dumps(report))


def test_rotated_sample_start(km, oracle):
    """init_multi: the start is the converged sample centres of the
    hypothesis with the lowest sample objective (checked against the oracle
    on the sample), and the run checked against k-means++ never ends above its
    objective by more than 1e-6 relative."""
    import torch
    from paper_2405_12052_gb300 import learned
    if not os.path.exists(learned.WEIGHTS):
        pytest.skip("no committed weights")
    net = learned.load()
    x = synth.aniso_mixture(300_000, 3, 16, seed=977)[0]
    xt = torch.from_numpy(x).cuda()
    g = km.KMeans(x.shape[1], 3, 16)
    g.set_points(xt, borrow=True)
    r = learned.init_multi(g, net, xt, hypotheses=8, seed=3)
    objs = r["sample_objectives"]
    assert r["hypothesis"] == int(np.argmin(objs)) and len(objs) == 8
    # the chosen start is (nearly) a fixed point of Lloyd's iteration on the
    # sample, and reassigning the sample to it cannot raise its objective
    idx = np.sort(np.random.Generator(np.random.PCG64(3)).choice(x.shape[1], 4096, replace=False))
    xs = np.ascontiguousarray(x[:, idx])
    z = oracle.assign(xs, r["mu0"])
    assert oracle.objective(xs, r["mu0"], z) <= objs[r["hypothesis"]] * (1 + 1e-9)
    _, mu1, _, e2 = oracle.step(xs, r["mu0"])
    assert e2 < 1e-6 * max(1.0, float((r["mu0"] ** 2).sum()))
    u = np.random.default_rng(5).random(16)
    rr = learned.run_with_fallback(g, net, u, seed=3, hypotheses=8, x=xt)
    kept = rr["objective_learned"] if rr["used"] == "learned" else rr["objective_kpp"]
    assert kept <= rr["objective_kpp"] * (1 + 1e-6)
    print(json.dumps({k: v for k, v in rr.items() if k != "centroids"}))
    g.close()


def test_learned_start_against_kmeanspp_on_held_out_mixtures(km):
    """The measured gain and shortfall of the learned start (64 rotated
    samples) against k-means++ + Lloyd on six held-out N = 1e6 anisotropic
    mixtures (seeds 900..905, the bench's recipe at a tenth of its size),
    tol 1e-6, at most 300 steps.  Recorded on GB300 when this test was
    written: from the learned start Lloyd needs fewer full-data steps than
    from k-means++ in 5 of 6 mixtures, and ends within 1e-6 of (or below) the
    k-means++ objective in 3 of 6 (objective ratios 2.03, 1.08, 1.003, 0.65,
    0.90, 0.92); the whole learned path (64 predictions, the batched sample
    runs, the full run) takes longer than k-means++ + Lloyd.  Asserted: the
    judged result never ends above the k-means++ objective (beyond 1e-6
    relative), and the learned start needs fewer full-data steps in at least
    4 of the 6; the objective ratios are printed."""
    import torch
    from paper_2405_12052_gb300 import learned
    if not os.path.exists(learned.WEIGHTS):
        pytest.skip("no committed weights")
    net = learned.load()
    n = 1_000_000
    rows = []
    for s in range(6):
        x = synth.aniso_mixture(n, 3, 16, seed=900 + s)[0]
        xt = torch.from_numpy(x).cuda()
        g = km.KMeans(n, 3, 16)
        g.set_points(xt, borrow=True)
        u = np.random.default_rng(700 + s).random(16)
        r = learned.run_with_fallback(g, net, u, seed=s, hypotheses=64, x=xt)
        kept = r["objective_learned"] if r["used"] == "learned" else r["objective_kpp"]
        assert kept <= r["objective_kpp"] * (1 + 1e-6)
        rows.append({"seed": 900 + s, "iters_learned": r["iters_learned"], "iters_kpp": r["iters_kpp"],
                     "objective_ratio": r["objective_learned"] / r["objective_kpp"], "used": r["used"]})
        g.close()
    fewer = sum(q["iters_learned"] < q["iters_kpp"] for q in rows)
    within = sum(q["objective_ratio"] <= 1 + 1e-6 for q in rows)
    print(json.dumps({"fewer_steps": fewer, "objective_within_1e-6_or_lower": within, "rows": rows}))
    assert fewer >= 4, rows
