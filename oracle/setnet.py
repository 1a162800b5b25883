"""FP64 CPU oracle of the learned initialiser's set network (test
infrastructure: only tests/, the smoke check and bench.py's CPU legs use
it; the product path never does).

The network predicts K starting centres for Lloyd's algorithm from a sample
of S points (the paper's sensitivity of the result to the initial centres,
section "The Lloyd's algorithm"):

    standardise   x' = (x - m) / s, m and s the sample's per-coordinate mean
                  and population standard deviation (s = 1 where it is 0);
    per point     h1 = relu(W1 x' + b1),  h2 = relu(W2 h1 + b2)   (H = 128)
    pool          g = mean over the S points of h2
    head          a3 = relu(W3 g + b3),  p = W4 a3 + b4  -> K x d centres
                  in standardised coordinates; c = p * s + m.

Loss for a batch of B sets with targets T_b (K x d, standardised with the
set's own m and s): the mean over sets of the symmetric Chamfer distance
    (1/K) sum_k min_j |p_k - t_j|^2 + (1/K) sum_j min_k |p_k - t_j|^2
(ties: the lowest index).  Everything here is float64 numpy, written from
those definitions; the backward pass is the chain rule of the same
expressions (relu'(0) = 0).  The GPU kernels compute the same in float32.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def shapes(d: int, k: int, h: int = 128) -> dict:
    return {"W1": (h, d), "b1": (h,), "W2": (h, h), "b2": (h,), "W3": (h, h), "b3": (h,),
            "W4": (k * d, h), "b4": (k * d,)}


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], dtype=np.float64).reshape(-1) for n in PARAM_NAMES])


def unflatten(flat: np.ndarray, d: int, k: int, h: int = 128) -> dict:
    out, o = {}, 0
    for n in PARAM_NAMES:
        shp = shapes(d, k, h)[n]
        sz = int(np.prod(shp))
        out[n] = np.asarray(flat[o:o + sz], dtype=np.float64).reshape(shp)
        o += sz
    return out


def standardise(x: np.ndarray):
    """x: (B, S, d).  Returns (x', m (B, d), s (B, d))."""
    x = np.asarray(x, dtype=np.float64)
    m = x.mean(axis=1)
    s = np.sqrt(((x - m[:, None, :]) ** 2).mean(axis=1))
    s = np.where(s > 0, s, 1.0)
    return (x - m[:, None, :]) / s[:, None, :], m, s


def forward(params: dict, xs: np.ndarray, k: int):
    """xs: standardised (B, S, d).  Returns (p (B, K, d), cache)."""
    W1, b1, W2, b2 = params["W1"], params["b1"], params["W2"], params["b2"]
    W3, b3, W4, b4 = params["W3"], params["b3"], params["W4"], params["b4"]
    z1 = xs @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    g = h2.mean(axis=1)
    z3 = g @ W3.T + b3
    a3 = np.maximum(z3, 0.0)
    out = a3 @ W4.T + b4
    B, d = xs.shape[0], xs.shape[2]
    return out.reshape(B, k, d), dict(xs=xs, z1=z1, h1=h1, z2=z2, h2=h2, g=g, z3=z3, a3=a3)


def chamfer(p: np.ndarray, t: np.ndarray):
    """Mean over sets of the symmetric Chamfer distance, and d loss / d p."""
    B, K, d = p.shape
    diff = p[:, :, None, :] - t[:, None, :, :]            # (B, K, K, d): p_k - t_j
    dist = (diff ** 2).sum(axis=-1)                       # (B, K, K)
    jstar = dist.argmin(axis=2)                           # nearest target of each p_k
    kstar = dist.argmin(axis=1)                           # nearest prediction of each t_j
    bi = np.arange(B)[:, None]
    ki = np.arange(K)[None, :]
    term1 = dist[bi, ki, jstar].sum(axis=1) / K
    term2 = dist[bi, kstar, ki].sum(axis=1) / K
    loss = float((term1 + term2).mean())
    dp = np.zeros_like(p)
    dp += 2.0 * (p - t[bi, jstar]) / K
    for j in range(K):                                     # t_j pulls its nearest p
        kk = kstar[:, j]
        dp[np.arange(B), kk] += 2.0 * (p[np.arange(B), kk] - t[:, j]) / K
    return loss, dp / B


def backward(params: dict, cache: dict, dp: np.ndarray) -> dict:
    """Gradients of the loss given d loss / d p (B, K, d)."""
    W2, W3, W4 = params["W2"], params["W3"], params["W4"]
    B, S = cache["h2"].shape[:2]
    dout = dp.reshape(B, -1)
    g, a3, z3 = cache["g"], cache["a3"], cache["z3"]
    grads = {"W4": dout.T @ a3, "b4": dout.sum(axis=0)}
    dz3 = (dout @ W4) * (z3 > 0)
    grads["W3"] = dz3.T @ g
    grads["b3"] = dz3.sum(axis=0)
    dg = dz3 @ W3
    dz2 = (dg[:, None, :] / S) * (cache["z2"] > 0)
    grads["W2"] = np.einsum("bsi,bsj->ij", dz2, cache["h1"])
    grads["b2"] = dz2.sum(axis=(0, 1))
    dz1 = (dz2 @ W2) * (cache["z1"] > 0)
    grads["W1"] = np.einsum("bsi,bsj->ij", dz1, cache["xs"])
    grads["b1"] = dz1.sum(axis=(0, 1))
    return grads


def loss_and_grads(params: dict, x: np.ndarray, targets: np.ndarray, k: int):
    """Raw points x (B, S, d) and raw targets (B, K, d): loss and gradients."""
    xs, m, s = standardise(x)
    ts = (np.asarray(targets, dtype=np.float64) - m[:, None, :]) / s[:, None, :]
    p, cache = forward(params, xs, k)
    loss, dp = chamfer(p, ts)
    return loss, backward(params, cache, dp)


def predict(params: dict, x: np.ndarray, k: int) -> np.ndarray:
    """Centres (B, K, d) in the points' coordinates."""
    xs, m, s = standardise(x)
    p, _ = forward(params, xs, k)
    return p * s[:, None, :] + m[:, None, :]


def adam(params: dict, grads: dict, state: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8) -> dict:
    """One Adam step (Kingma and Ba 2015) with bias correction; state holds
    t, m and v per parameter (created on first use)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = {}
    for n in PARAM_NAMES:
        m = state.setdefault("m_" + n, np.zeros_like(params[n]))
        v = state.setdefault("v_" + n, np.zeros_like(params[n]))
        m[...] = beta1 * m + (1 - beta1) * grads[n]
        v[...] = beta2 * v + (1 - beta2) * grads[n] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        out[n] = params[n] - lr * mh / (np.sqrt(vh) + eps)
    return out


def init_params(d: int, k: int, h: int = 128, seed: int = 0) -> dict:
    """He-uniform weights (fan-in), zero biases; seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for n, shp in shapes(d, k, h).items():
        if n.startswith("W"):
            lim = np.sqrt(6.0 / shp[1])
            out[n] = rng.uniform(-lim, lim, size=shp)
        else:
            out[n] = np.zeros(shp)
    return out
