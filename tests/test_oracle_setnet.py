"""Pins of the FP64 set-network oracle (learned initialiser) against what
the mathematics fixes: central finite differences of the loss, closed forms
of the Chamfer loss and of Adam's first step, and the invariances of the
architecture (point order, target order, affine maps of the input)."""
import numpy as np
import pytest

from oracle import setnet as sn


def _tiny(seed=0, d=3, k=4, h=8, B=2, S=5):
    rng = np.random.default_rng(seed)
    params = sn.init_params(d, k, h, seed=seed)
    for n in params:  # non-zero biases so every branch is exercised
        if n.startswith("b"):
            params[n] = rng.normal(scale=0.3, size=params[n].shape)
    x = rng.normal(size=(B, S, d)) * [2.0, 0.5, 1.0][:d] + [1.0, -3.0, 0.2][:d]
    t = rng.normal(size=(B, k, d))
    return params, x, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_central_differences(seed):
    params, x, t = _tiny(seed)
    k = t.shape[1]
    _, grads = sn.loss_and_grads(params, x, t, k)
    flat = sn.flatten(params)
    g_flat = sn.flatten(grads)
    h = 1e-6
    num = np.empty_like(flat)
    for q in range(flat.size):
        fp, fm = flat.copy(), flat.copy()
        fp[q] += h
        fm[q] -= h
        lp, _ = sn.loss_and_grads(sn.unflatten(fp, 3, k, 8), x, t, k)
        lm, _ = sn.loss_and_grads(sn.unflatten(fm, 3, k, 8), x, t, k)
        num[q] = (lp - lm) / (2 * h)
    assert np.linalg.norm(num - g_flat) <= 1e-6 * np.linalg.norm(num)


def test_chamfer_closed_forms():
    rng = np.random.default_rng(3)
    t = rng.normal(size=(3, 5, 2))
    loss, dp = sn.chamfer(t.copy(), t)
    assert loss == 0.0 and np.all(dp == 0)
    # K = 1: loss = 2 |p - t|^2, gradient 4 (p - t) / B
    p1, t1 = np.array([[[1.0, 2.0]]]), np.array([[[4.0, -2.0]]])
    loss, dp = sn.chamfer(p1, t1)
    assert loss == 2 * 25.0 and np.array_equal(dp, 4 * (p1 - t1))
    # two predictions on one target: the far one still gets pulled by term 1
    p2, t2 = np.array([[[0.0], [3.0]]]), np.array([[[1.0], [10.0]]])
    loss, _ = sn.chamfer(p2, t2)
    assert loss == pytest.approx(((1 + 4) + (1 + 49)) / 2)


def test_invariances():
    params, x, t = _tiny(4, B=1, S=7)
    k = t.shape[1]
    c = sn.predict(params, x, k)
    perm = np.random.default_rng(0).permutation(x.shape[1])
    assert np.allclose(sn.predict(params, x[:, perm], k), c, rtol=0, atol=1e-12)
    a, b = np.array([3.0, 0.5, 2.0]), np.array([-7.0, 1.0, 100.0])
    assert np.allclose(sn.predict(params, x * a + b, k), c * a + b, rtol=1e-12, atol=1e-9)
    l1, _ = sn.loss_and_grads(params, x, t, k)
    l2, _ = sn.loss_and_grads(params, x, t[:, ::-1], k)
    assert l1 == pytest.approx(l2, rel=1e-14)


def test_adam_first_step_closed_form():
    params, x, t = _tiny(5)
    _, grads = sn.loss_and_grads(params, x, t, 4)
    # first step: m^ = g, v^ = g^2, so the update is lr * g / (|g| + eps)
    new = sn.adam(params, grads, {}, lr=1e-3, eps=1e-300)
    for n in sn.PARAM_NAMES:
        expect = params[n] - 1e-3 * np.sign(grads[n])
        assert np.allclose(new[n], expect, rtol=0, atol=1e-15)


def test_planted_mistake_fails_the_difference_check():
    """A backward pass that drops the relu mask of the head is caught."""
    params, x, t = _tiny(6)
    xs, m, s = sn.standardise(x)
    ts = (t - m[:, None, :]) / s[:, None, :]
    p, cache = sn.forward(params, xs, 4)
    _, dp = sn.chamfer(p, ts)
    cache_bad = dict(cache)
    cache_bad["z3"] = np.abs(cache["z3"]) + 1.0  # every head unit treated as active
    g_bad = sn.flatten(sn.backward(params, cache_bad, dp))
    g_ok = sn.flatten(sn.backward(params, cache, dp))
    if np.any(cache["z3"] <= 0):
        assert np.linalg.norm(g_bad - g_ok) > 1e-3 * np.linalg.norm(g_ok)
