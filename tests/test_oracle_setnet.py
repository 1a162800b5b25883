"""Pins of the FP64 set-network oracle (learned initialiser) against what
the mathematics fixes (tests/setnet_pins.py): a hand-worked forward pass,
population-std standardisation, Adam on a constant gradient over several
steps and its scale invariance, central finite differences of the loss,
closed forms of the Chamfer loss; plus the invariances of the architecture
(point order, target order, affine maps of the input)."""
import numpy as np
import pytest

import setnet_pins as P
from oracle import setnet as sn


def test_forward_hand_worked():
    P.pin_forward_hand_worked(sn)


def test_standardise_population_std():
    P.pin_standardise_population_std(sn)


def test_predict_maps_back():
    P.pin_predict_maps_back(sn)


def test_adam_constant_gradient_steps():
    P.pin_adam_constant_gradient_steps(sn)


def test_adam_scale_invariance():
    P.pin_adam_scale_invariance(sn)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_central_differences(seed):
    P.pin_backward_central_differences(sn, seed)


def test_chamfer_closed_forms():
    P.pin_chamfer_closed_forms(sn)


def test_invariances():
    params, x, t = P._tiny(sn, 4, B=1, S=7)
    k = t.shape[1]
    c = sn.predict(params, x, k)
    perm = np.random.default_rng(0).permutation(x.shape[1])
    assert np.allclose(sn.predict(params, x[:, perm], k), c, rtol=0, atol=1e-12)
    a, b = np.array([3.0, 0.5, 2.0]), np.array([-7.0, 1.0, 100.0])
    assert np.allclose(sn.predict(params, x * a + b, k), c * a + b, rtol=1e-12, atol=1e-9)
    l1, _ = sn.loss_and_grads(params, x, t, k)
    l2, _ = sn.loss_and_grads(params, x, t[:, ::-1], k)
    assert l1 == pytest.approx(l2, rel=1e-14)
