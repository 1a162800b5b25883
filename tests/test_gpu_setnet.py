"""The set network's FP32 GPU kernels against the FP64 CPU oracle: loss and
every parameter gradient (relative error <= 1e-4 per tensor), predictions,
one Adam step, determinism, and the initialiser on a context."""
import numpy as np
import pytest

import synth
from oracle import setnet as osn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def km():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2405_12052_gb300 as m
    m.build()
    return m


def _case(seed, B=3, S=256, d=3, k=16):
    rng = np.random.default_rng(seed)
    params = osn.init_params(d, k, 128, seed=seed)
    for n in params:
        if n.startswith("b"):
            params[n] = rng.normal(scale=0.05, size=params[n].shape)
    x = np.stack([synth.aniso_mixture(S, d, 4, seed=100 * seed + b)[0].T for b in range(B)]).astype(np.float32)
    t = (rng.normal(size=(B, k, d)) * 20).astype(np.float32)
    return params, x, t


def _params32(params):
    return osn.flatten(params).astype(np.float32)


@pytest.mark.parametrize("seed,B,S,d,k", [(0, 3, 256, 3, 16), (1, 2, 4096, 3, 16), (2, 4, 128, 2, 7)])
def test_loss_and_gradients_match_oracle(km, seed, B, S, d, k):
    params, x, t = _case(seed, B, S, d, k)
    p32 = _params32(params)
    # the oracle runs on the float32-rounded parameters and inputs
    pr = osn.unflatten(p32.astype(np.float64), d, k)
    ref_loss, ref_g = osn.loss_and_grads(pr, x.astype(np.float64), t.astype(np.float64), k)
    net = km.SetNet(d, k)
    net.set_params(p32)
    loss = net.loss_grad(x, t)
    g = osn.unflatten(net.grads().astype(np.float64), d, k)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    for n in osn.PARAM_NAMES:
        err = np.linalg.norm(g[n] - ref_g[n]) / max(np.linalg.norm(ref_g[n]), 1e-30)
        assert err <= 1e-4, (n, err)
    net.close()


def test_predict_and_adam_match_oracle(km):
    params, x, t = _case(3, B=2, S=512)
    p32 = _params32(params)
    pr = osn.unflatten(p32.astype(np.float64), 3, 16)
    net = km.SetNet(3, 16)
    net.set_params(p32)
    c = net.predict(x)
    cref = osn.predict(pr, x.astype(np.float64), 16)
    scale = np.abs(x).max()
    assert np.max(np.abs(c - cref)) <= 1e-4 * scale
    net.loss_grad(x, t)
    g = osn.unflatten(net.grads().astype(np.float64), 3, 16)
    net.adam(1e-3)
    new = osn.unflatten(net.params().astype(np.float64), 3, 16)
    ref = osn.adam(pr, g, {}, lr=1e-3)
    for n in osn.PARAM_NAMES:
        assert np.allclose(new[n], ref[n], rtol=1e-5, atol=1e-6), n
    net.close()


def test_adam_several_steps_match_oracle(km):
    """Five Adam steps on the kernel's own gradients of a fixed batch: the
    moments and the bias correction at t = 1..5 against the FP64 oracle's
    update rule applied to the same gradients."""
    params, x, t = _case(6, B=2, S=256)
    p32 = _params32(params)
    net = km.SetNet(3, 16)
    net.set_params(p32)
    ref = osn.unflatten(p32.astype(np.float64), 3, 16)
    state = {}
    for step in range(5):
        net.loss_grad(x, t)
        g = osn.unflatten(net.grads().astype(np.float64), 3, 16)
        net.adam(1e-3)
        ref = osn.adam(ref, g, state, lr=1e-3)
        got = osn.unflatten(net.params().astype(np.float64), 3, 16)
        for n in osn.PARAM_NAMES:
            assert np.allclose(got[n], ref[n], rtol=1e-5, atol=2e-6), (step, n)
        # continue from the kernel's parameters (float32), as training does
        ref = got
    net.close()


def test_training_is_deterministic(km):
    params, x, t = _case(4, B=4, S=256)
    p32 = _params32(params)
    outs = []
    for _ in range(2):
        net = km.SetNet(3, 16)
        net.set_params(p32)
        losses = [net.train_step(x, t, 1e-3) for _ in range(5)]
        outs.append((losses, net.params()))
        net.close()
    assert outs[0][0] == outs[1][0] and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][0][-1] < outs[0][0][0]  # the loss goes down on a fixed batch


def test_init_learned_on_a_context(km, oracle):
    params, _, _ = _case(5)
    net = km.SetNet(3, 16)
    net.set_params(_params32(params))
    x, _, _ = synth.aniso_mixture(30_000, 3, 16, seed=8)
    g = km.KMeans(30_000, 3, 16)
    g.set_points(x)
    mu = g.init_learned(net, 4096, seed=11)
    # the same sample through the oracle network: points floor(u_j N) for the
    # SplitMix64 stream of the seed
    def splitmix(seed, j):
        z = (seed + (j + 1) * 0x9E3779B97F4A7C15) & (2**64 - 1)
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
        return z ^ (z >> 31)
    idx = np.array([min(int((splitmix(11, j) >> 11) * 2.0**-53 * 30_000), 29_999) for j in range(4096)])
    sample = x[:, idx].T[None].astype(np.float64)
    ref = osn.predict(osn.unflatten(_params32(params).astype(np.float64), 3, 16), sample, 16)[0]
    assert np.max(np.abs(mu - ref)) <= 1e-4 * np.abs(x).max()
    r = g.run(20, 1e-6)
    rr = oracle.run(x, mu, 20, 1e-6)
    assert np.array_equal(r["labels"], rr["labels"]) and r["iters"] == rr["iters"]
    g.close()
    net.close()


def test_set_transforms_match_numpy(km):
    """km_sets_mean and km_sets_rotate_f32/_f64 against numpy in float64:
    per-set means, rotations about each set's centre and back (R^T)."""
    import torch
    rng = np.random.default_rng(9)
    B, S, d = 5, 777, 3
    x = (rng.normal(size=(B, S, d)) * [3.0, 0.5, 10.0] + [100.0, -2.0, 7.0]).astype(np.float32)
    R = np.stack([np.linalg.qr(rng.normal(size=(d, d)))[0] for _ in range(B)])
    xt = torch.from_numpy(x).cuda()
    m = km.sets_mean(xt).cpu().numpy()
    assert np.allclose(m, x.astype(np.float64).mean(axis=1), rtol=1e-14, atol=1e-12)
    out = km.sets_rotate(xt, torch.from_numpy(R), center=torch.from_numpy(m)).cpu().numpy()
    ref = np.einsum("bij,bsj->bsi", R, x.astype(np.float64) - m[:, None, :]) + m[:, None, :]
    assert np.max(np.abs(out - ref)) <= 2 ** -22 * np.abs(ref).max()
    back = km.sets_rotate(torch.from_numpy(ref).cuda(), torch.from_numpy(R), center=torch.from_numpy(m),
                          transpose=True).cpu().numpy()
    assert np.allclose(back, x.astype(np.float64), rtol=0, atol=1e-11 * np.abs(ref).max())
    # one set rotated B ways (set stride 0), about one centre
    one = km.sets_rotate(xt[0], torch.from_numpy(R), center=torch.from_numpy(m[0])).cpu().numpy()
    ref1 = np.einsum("bij,sj->bsi", R, x[0].astype(np.float64) - m[0]) + m[0]
    assert np.max(np.abs(one - ref1)) <= 2 ** -22 * np.abs(ref1).max()
