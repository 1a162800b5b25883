"""Pins of the set-network oracle (the learned initialiser's network and its
training rule) that fix its values independently of its own code.  Each pin
takes the oracle module, so that test_oracle_setnet_mutants.py can run the
same pins against copies of the oracle with a planted mistake.

What fixes the values:
* the forward pass of a network with hand-set sparse weights on four
  hand-chosen points, whose output is worked out by hand below (every ReLU
  kink, the mean over the set and the head are each visible in it);
* standardisation with the population standard deviation (mean of squared
  deviations), and the value 1 for a constant coordinate;
* Adam (Kingma and Ba 2015) on a constant gradient: with bias correction
  the corrected moments are exactly g and g^2 at every step t, so every step
  moves a parameter by lr * g / (|g| + eps), i.e. lr * sign(g) for eps -> 0;
  a scaled gradient c * g gives the same steps (scale invariance);
* the chain rule, checked by central finite differences of the loss (the
  backward pass against the forward pass);
* the Chamfer loss's closed forms (identical sets; one centre).
"""
from __future__ import annotations

import numpy as np

H3 = 3  # hidden width of the hand-set network


def _hand_params():
    """d = 2, K = 1, hidden width 3; weights chosen so that each ReLU clips
    some values and every path reaches the output."""
    W1 = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    b1 = np.array([-0.5, 0.25, 1.0])
    W2 = np.array([[1.0, 0.0, 0.0], [1.0, -1.0, 0.0], [0.0, 0.0, 1.0]])
    b2 = np.array([0.0, -0.1, -2.0])
    W3 = np.array([[2.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    b3 = np.array([-0.3, 0.05, -0.5])
    W4 = np.array([[1.0, 0.0, 1.0], [0.0, 3.0, 2.0]])
    b4 = np.array([0.1, -0.2])
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3, W4=W4, b4=b4)


# Standardised input: one set of four points (d = 2).
HAND_XS = np.array([[[2.0, 1.0], [0.0, 3.0], [1.0, -1.0], [3.0, 0.0]]])
# Worked by hand:
#   z1 = (x0 - 0.5, x1 + 0.25, 1):  (1.5, 1.25, 1), (-0.5, 3.25, 1), (0.5, -0.75, 1), (2.5, 0.25, 1)
#   h1 = relu(z1):                  (1.5, 1.25, 1), (0, 3.25, 1),    (0.5, 0, 1),     (2.5, 0.25, 1)
#   z2 = (h1_0, h1_0 - h1_1 - 0.1, h1_2 - 2):
#                                   (1.5, 0.15, -1), (0, -3.35, -1), (0.5, 0.4, -1), (2.5, 2.15, -1)
#   h2 = relu(z2):                  (1.5, 0.15, 0),  (0, 0, 0),      (0.5, 0.4, 0),  (2.5, 2.15, 0)
#   g = mean over the four points:  (4.5 / 4, 2.7 / 4, 0) = (1.125, 0.675, 0)
#   z3 = (2 g0 - 0.3, g1 + 0.05, g2 - 0.5) = (1.95, 0.725, -0.5);  a3 = (1.95, 0.725, 0)
#   p = (a3_0 + a3_2 + 0.1, 3 a3_1 + 2 a3_2 - 0.2) = (2.05, 1.975)
HAND_P = np.array([[[2.05, 1.975]]])
HAND_G = np.array([[1.125, 0.675, 0.0]])


def pin_forward_hand_worked(sn):
    p, cache = sn.forward(_hand_params(), HAND_XS.copy(), 1)
    assert p.shape == (1, 1, 2)
    assert np.allclose(p, HAND_P, rtol=0, atol=1e-12), p
    assert np.allclose(cache["g"], HAND_G, rtol=0, atol=1e-12), cache["g"]


def pin_standardise_population_std(sn):
    # coordinate 0: 1, 2, 3, 6 -> mean 3, squared deviations 4, 1, 0, 9, mean 3.5
    # coordinate 1: constant 10 -> deviation 0, standard deviation taken as 1
    x = np.array([[[1.0, 10.0], [2.0, 10.0], [3.0, 10.0], [6.0, 10.0]]])
    xs, m, s = sn.standardise(x)
    assert np.allclose(m, [[3.0, 10.0]], rtol=0, atol=1e-15)
    assert np.allclose(s, [[np.sqrt(3.5), 1.0]], rtol=1e-15, atol=0)
    assert np.allclose(xs[0, :, 0], np.array([-2.0, -1.0, 0.0, 3.0]) / np.sqrt(3.5), rtol=1e-15, atol=1e-15)
    assert np.all(xs[0, :, 1] == 0.0)


def pin_predict_maps_back(sn):
    # the hand network on raw points whose standardised form is HAND_XS:
    # raw = xs * s + m for the sample's own m, s, so the prediction is p * s + m
    xs = HAND_XS[0]
    # any affine image of HAND_XS standardises back to HAND_XS only if its
    # mean is 0 and std 1 per coordinate; build raw points with mean 0, std 1
    m0, s0 = xs.mean(axis=0), xs.std(axis=0)
    z = (xs - m0) / s0                    # mean 0, population std 1
    raw = (z * np.array([2.0, 0.5]) + np.array([10.0, -4.0]))[None]
    p_std, _ = sn.forward(_hand_params(), z[None], 1)
    c = sn.predict(_hand_params(), raw, 1)
    assert np.allclose(c, p_std * np.array([2.0, 0.5]) + np.array([10.0, -4.0]), rtol=0, atol=1e-12)


def _constant_grad_run(sn, scale, steps, lr=1e-3):
    rng = np.random.default_rng(7)
    params = sn.init_params(2, 2, 4, seed=3)
    g = {n: rng.normal(size=v.shape) * scale for n, v in params.items()}
    state = {}
    cur = params
    for _ in range(steps):
        cur = sn.adam(cur, g, state, lr=lr, eps=1e-300)
    return params, g, cur, state


def pin_adam_constant_gradient_steps(sn):
    for steps in (1, 2, 5):
        params, g, cur, state = _constant_grad_run(sn, 1.0, steps)
        assert state["t"] == steps
        for n in params:
            expect = params[n] - steps * 1e-3 * np.sign(g[n])
            assert np.allclose(cur[n], expect, rtol=0, atol=1e-14), (n, steps)


def pin_adam_scale_invariance(sn):
    _, _, a, _ = _constant_grad_run(sn, 1.0, 3)
    _, _, b, _ = _constant_grad_run(sn, 1e-3, 3)
    for n in a:
        assert np.allclose(a[n], b[n], rtol=0, atol=1e-14), n


def _tiny(sn, seed=0, d=3, k=4, h=8, B=2, S=5):
    rng = np.random.default_rng(seed)
    params = sn.init_params(d, k, h, seed=seed)
    for n in params:  # non-zero biases so every branch is exercised
        if n.startswith("b"):
            params[n] = rng.normal(scale=0.3, size=params[n].shape)
    x = rng.normal(size=(B, S, d)) * [2.0, 0.5, 1.0][:d] + [1.0, -3.0, 0.2][:d]
    t = rng.normal(size=(B, k, d))
    return params, x, t


def pin_backward_central_differences(sn, seed=0):
    params, x, t = _tiny(sn, seed)
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


def pin_chamfer_closed_forms(sn):
    rng = np.random.default_rng(3)
    t = rng.normal(size=(3, 5, 2))
    loss, dp = sn.chamfer(t.copy(), t)
    assert loss == 0.0 and np.all(dp == 0)
    p1, t1 = np.array([[[1.0, 2.0]]]), np.array([[[4.0, -2.0]]])
    loss, dp = sn.chamfer(p1, t1)
    assert loss == 2 * 25.0 and np.array_equal(dp, 4 * (p1 - t1))
    p2, t2 = np.array([[[0.0], [3.0]]]), np.array([[[1.0], [10.0]]])
    loss, _ = sn.chamfer(p2, t2)
    assert abs(loss - ((1 + 4) + (1 + 49)) / 2) <= 1e-12


ALL_PINS = [pin_forward_hand_worked, pin_standardise_population_std, pin_predict_maps_back,
            pin_adam_constant_gradient_steps, pin_adam_scale_invariance, pin_backward_central_differences,
            pin_chamfer_closed_forms]
