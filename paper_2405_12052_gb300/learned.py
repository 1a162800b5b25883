"""Learned initialiser: training data, training and use of the set network.

The network (CUDA forward, backward and Adam kernels behind the C ABI,
``SetNet``) predicts K starting centres from a 4096-point sample; Lloyd's
iteration then runs from them.  Training pairs are seeded anisotropic
Gaussian mixtures (d = 3, K = 16 components: Haar rotations, axis standard
deviations uniform in [0.5, 2], means uniform in [-50, 50]^3, Dirichlet(1)
weights) with, as targets, the centres the plain method converges to from
the generating means (``KMeansBatch``, tol 1e-6).  The k-means++ start plus
Lloyd remains the fallback and decides by the final objective
(``run_with_fallback``).

Only array plumbing (drawing the synthetic mixtures, gathering batches) uses
torch; every step of the network and of Lloyd's iteration runs in the
library's kernels.  Usage on a GPU:

    python -m paper_2405_12052_gb300.learned train --mixtures 200000 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import KMeans, KMeansBatch, SetNet

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "setnet_d3_k16.npz")


def mixtures(count: int, S: int = 4096, d: int = 3, k: int = 16, seed: int = 0, device="cuda",
             chunk: int = 4096):
    """``count`` seeded anisotropic mixtures of S points each, drawn on the
    GPU in chunks of ``chunk`` mixtures (chunk c from generator seed
    seed * 1000003 + c).  Returns (x [count, S, d] float32, means
    [count, k, d] float64)."""
    import torch
    xs, ms = [], []
    for c, c0 in enumerate(range(0, count, chunk)):
        m = min(chunk, count - c0)
        g = torch.Generator(device=device).manual_seed(int(seed) * 1000003 + c)
        means = torch.rand(m, k, d, generator=g, device=device, dtype=torch.float64) * 100.0 - 50.0
        a = torch.randn(m, k, d, d, generator=g, device=device, dtype=torch.float64)
        # Haar rotation: Gram-Schmidt on Gaussian columns (QR with a positive
        # diagonal), written out for small d
        cols = []
        for j in range(d):
            v = a[..., :, j]
            for u in cols:
                v = v - (v * u).sum(-1, keepdim=True) * u
            cols.append(v / torch.linalg.vector_norm(v, dim=-1, keepdim=True))
        q = torch.stack(cols, dim=-1)
        sig = torch.rand(m, k, d, generator=g, device=device, dtype=torch.float64) * 1.5 + 0.5
        w = -torch.log(torch.rand(m, k, generator=g, device=device, dtype=torch.float64))  # Dirichlet(1)
        cdf = torch.cumsum(w / w.sum(dim=1, keepdim=True), dim=1)
        u = torch.rand(m, S, generator=g, device=device, dtype=torch.float64)
        comp = torch.searchsorted(cdf, u).clamp_(max=k - 1)                     # [m, S]
        z = torch.randn(m, S, d, generator=g, device=device, dtype=torch.float64)
        bi = torch.arange(m, device=device)[:, None]
        x = means[bi, comp] + torch.einsum("csij,csj->csi", q[bi, comp], z * sig[bi, comp])
        xs.append(x.to(torch.float32))
        ms.append(means)
    return torch.cat(xs), torch.cat(ms)


def converged_targets(x, means, chunk: int = 16384, tol: float = 1e-6, max_iter: int = 300):
    """Centres the plain method converges to on each set, starting from the
    generating means (batched Lloyd).  x: [count, S, d] CUDA float32."""
    import torch
    count, S, d = x.shape
    k = means.shape[1]
    out = torch.empty(count, k, d, dtype=torch.float32, device=x.device)
    iters = []
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        m = c1 - c0
        b = KMeansBatch(np.full(m, S), np.full(m, d), np.full(m, k))
        b.set_points(x[c0:c1].permute(0, 2, 1).contiguous().reshape(-1))
        b.set_init(means[c0:c1].cpu().numpy().reshape(-1))
        r = b.run(max_iter, tol, want_labels=False)
        out[c0:c1] = torch.from_numpy(r["centroids"].reshape(m, k, d)).to(torch.float32).to(x.device)
        iters.append(r["iters"])
        b.close()
    return out, np.concatenate(iters)


def init_params(d: int, k: int, seed: int = 0, h: int = 128) -> np.ndarray:
    """He-uniform weights (fan-in), zero biases, flattened in the network's
    order W1, b1, W2, b2, W3, b3, W4, b4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for rows, cols in ((h, d), (h, h), (h, h), (k * d, h)):
        lim = math.sqrt(6.0 / cols)
        parts.append(rng.uniform(-lim, lim, size=rows * cols))
        parts.append(np.zeros(rows))
    return np.concatenate(parts).astype(np.float32)


def _rotations(m: int, d: int, g, device):
    """m seeded Haar-random orthogonal maps (QR of Gaussian matrices, signs
    fixed: rotations and reflections), as a (m, d, d) float64 tensor: the
    random input of the training augmentation."""
    import torch
    a = torch.randn(m, d, d, generator=g, device=device, dtype=torch.float64)
    q, r = torch.linalg.qr(a)
    return q * torch.sign(torch.diagonal(r, dim1=-2, dim2=-1)).unsqueeze(-2)


def train(x, t, *, epochs: int = 3, batch: int = 64, lr: float = 1e-3, lr_min: float = 1e-5, seed: int = 0,
          log_every: int = 200, val=None, log=print, rotate: bool = False):
    """Adam on the symmetric Chamfer loss, cosine learning-rate decay.  With
    ``rotate`` every batch's sets and targets are turned by seeded Haar
    rotations about the origin (data augmentation: the network then meets
    the rotated samples that init_multi gives it)."""
    import torch
    count, S, d = x.shape
    k = t.shape[1]
    net = SetNet(d, k)
    net.set_params(init_params(d, k, seed))
    g = torch.Generator(device=x.device).manual_seed(seed + 1)
    steps = epochs * (count // batch)
    hist = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(count, generator=g, device=x.device)
        for s0 in range(0, count - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            xb, tb = x[idx].contiguous(), t[idx].contiguous()
            if rotate:
                from . import sets_rotate
                rot = _rotations(batch, d, g, x.device)
                xb = sets_rotate(xb, rot)
                tb = sets_rotate(tb, rot)
            rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / max(1, steps)))
            want = (step % log_every) == 0 or step == steps - 1
            loss = net.train_step(xb, tb, rate, want_loss=want)
            if want:
                entry = {"step": step, "epoch": ep, "loss": loss, "lr": rate, "s": time.perf_counter() - t0}
                if val is not None:
                    entry["val_loss"] = net.loss_grad(*val)
                hist.append(entry)
                log(json.dumps(entry))
            step += 1
    return net, hist


def save(net: SetNet, path: str, meta: dict):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=net.params(), d=net.d, k=net.k, meta=json.dumps(meta))


def load(path: str | None = None) -> SetNet:
    """The network from a weights file (default: KM_SETNET_WEIGHTS if set,
    else the committed weights)."""
    z = np.load(path or os.environ.get("KM_SETNET_WEIGHTS", WEIGHTS))
    net = SetNet(int(z["d"]), int(z["k"]))
    net.set_params(z["params"])
    return net


def _haar(rng, d: int) -> np.ndarray:
    """A Haar-distributed rotation (QR of a Gaussian matrix, signs fixed)."""
    q, r = np.linalg.qr(rng.standard_normal((d, d)))
    return q * np.sign(np.diag(r))[None, :]


def init_multi(g: KMeans, net: SetNet, x, *, hypotheses: int = 64, sample_n: int = 4096, seed: int = 0,
               max_iter: int = 300, tol: float = 1e-6) -> dict:
    """Learned start with test-time rotations.  One seeded sample of
    ``sample_n`` of the points x (d x N, a CUDA tensor: the context's
    points) is rotated about its mean by the identity and hypotheses - 1
    seeded Haar rotations (km_sets_mean, km_sets_rotate_f32); the network
    predicts K centres for each rotated copy (one batched forward pass) and
    they are rotated back (km_sets_rotate_f64).  Each prediction starts
    Lloyd's iteration on the sample (all of them in one batched run), and the
    converged sample centres with the lowest sample objective become the
    context's start.  The sample indices and the rotations are the random
    inputs, drawn here; every arithmetic step runs in the library's kernels.
    Returns the start and the per-hypothesis sample objectives."""
    import torch
    from . import sets_mean, sets_rotate
    d, n = int(x.shape[0]), int(x.shape[1])
    k = g.k
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.sort(rng.choice(n, size=sample_n, replace=False))
    xs = x[:, torch.from_numpy(idx).to(x.device)].t().contiguous()             # (S, d) float32, gathered
    m = sets_mean(xs)                                                           # (1, d) float64
    rots = torch.from_numpy(np.stack([np.eye(d)] + [_haar(rng, d) for _ in range(hypotheses - 1)]))
    batch = sets_rotate(xs, rots, center=m[0])                                  # (H, S, d) float32
    pred = torch.from_numpy(net.predict(batch)).to(x.device)                    # (H, K, d) float64
    starts = sets_rotate(pred, rots, center=m[0], transpose=True).cpu().numpy()
    b = KMeansBatch(np.full(hypotheses, sample_n), np.full(hypotheses, d), np.full(hypotheses, k))
    try:
        b.set_points(xs.t().contiguous().repeat(hypotheses, 1).reshape(-1))
        b.set_init(starts.reshape(-1))
        b.set_shape(1024, 256)
        rb = b.run(max_iter, tol, want_labels=False)
        objs = b.objective()
        best = int(np.argmin(objs))
        mu0 = b.split_centroids(rb["centroids"])[best].reshape(k, d)
    finally:
        b.close()
    g.set_init(mu0)
    return dict(mu0=mu0, hypothesis=best, sample_objectives=objs, sample_iters=rb["iters"])


def run_with_fallback(g: KMeans, net: SetNet, uniforms, *, sample_n: int = 4096, seed: int = 0,
                      max_iter: int = 300, tol: float = 1e-6, fallback: bool = True, hypotheses: int = 1,
                      x=None) -> dict:
    """Learned start + Lloyd; with ``fallback``, also k-means++ (the given K
    uniforms) + Lloyd, keeping the learned result only if its objective is
    within 1e-6 relative of the k-means++ result's (else the fallback).
    hypotheses > 1 takes the rotated-sample start (init_multi; x = the
    context's points)."""
    t0 = time.perf_counter()
    if hypotheses > 1:
        init_multi(g, net, x, hypotheses=hypotheses, sample_n=sample_n, seed=seed, max_iter=max_iter, tol=tol)
    else:
        g.init_learned(net, sample_n, seed)
    r = g.run(max_iter, tol, want_labels=False)
    obj = g.objective()
    t_learned = time.perf_counter() - t0
    out = dict(iters_learned=r["iters"], objective_learned=obj, wall_learned=t_learned,
               centroids=r["centroids"], used="learned")
    if fallback:
        t1 = time.perf_counter()
        g.init_kmeanspp(uniforms)
        rp = g.run(max_iter, tol, want_labels=False)
        objp = g.objective()
        out.update(iters_kpp=rp["iters"], objective_kpp=objp, wall_kpp=time.perf_counter() - t1)
        if obj > objp * (1 + 1e-6):
            out.update(used="kmeans++", centroids=rp["centroids"])
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--mixtures", type=int, default=200_000)
    tr.add_argument("--val", type=int, default=2048)
    tr.add_argument("--epochs", type=int, default=3)
    tr.add_argument("--batch", type=int, default=64)
    tr.add_argument("--lr", type=float, default=1e-3)
    tr.add_argument("--seed", type=int, default=0)
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--rotate", action="store_true", help="augment with random rotations")
    a = ap.parse_args(argv)
    if a.cmd == "train":
        dev = torch.device("cuda")
        t0 = time.perf_counter()
        x, means = mixtures(a.mixtures + a.val, seed=a.seed, device=dev)
        gen_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        tgt, its = converged_targets(x, means)
        tgt_s = time.perf_counter() - t0
        print(json.dumps({"generate_s": gen_s, "targets_s": tgt_s, "target_iters_mean": float(its.mean())}))
        xv, tv = x[a.mixtures:].contiguous(), tgt[a.mixtures:].contiguous()
        net, hist = train(x[:a.mixtures], tgt[:a.mixtures], epochs=a.epochs, batch=a.batch, lr=a.lr,
                          seed=a.seed, val=(xv[:256], tv[:256]), rotate=a.rotate)
        meta = dict(mixtures=a.mixtures, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed, S=4096,
                    rotate=a.rotate,
                    generate_s=gen_s, targets_s=tgt_s, final=hist[-1], history=hist[::5])
        save(net, a.out, meta)
        print(json.dumps({"saved": a.out, "final": hist[-1]}))


if __name__ == "__main__":
    main()
