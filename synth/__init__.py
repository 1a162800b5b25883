"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds NO arithmetic of Lloyd's method (no reassignment, no mean
update, no convergence error).  It draws points from Gaussian mixtures shaped
like the paper's workloads (section "Serial Lloyd's algorithm": mixtures of
bivariate Gaussians with N = 1e5..5e5, and three-dimensional sets with
N = 1e5..1e6) and draws starting centroids, which both sides then receive as
the same input.

All draws use numpy's PCG64 generator, seeded explicitly.  Points are float32
in the paper's d x N layout (X in R^{d x N}): coordinate j of point i is
X[j, i].
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "iso_mixture", "aniso_mixture", "haar_rotation", "init_distinct",
    "init_kmeanspp", "WORKLOADS", "workload",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_rotation(rng: np.random.Generator, d: int) -> np.ndarray:
    """Random rotation from the Haar measure: QR of a Gaussian matrix with the
    signs of R's diagonal folded into Q (Mezzadri, 2007)."""
    g = rng.standard_normal((d, d))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q


def _component_sizes(rng, n: int, n_comp: int, weights: str) -> np.ndarray:
    if weights == "equal":
        sizes = np.full(n_comp, n // n_comp, dtype=np.int64)
        sizes[: n - sizes.sum()] += 1
        return sizes
    if weights == "dirichlet":
        w = rng.dirichlet(np.ones(n_comp))
        return rng.multinomial(n, w).astype(np.int64)
    raise ValueError(weights)


def _assemble(rng, blocks, comp_sizes, d, n, shuffle=True):
    """Stack per-component blocks (each (d, n_c) float32) and shuffle columns."""
    xs = np.empty((d, n), dtype=np.float32)
    comp = np.empty(n, dtype=np.int32)
    at = 0
    for c, b in enumerate(blocks):
        m = b.shape[1]
        xs[:, at:at + m] = b
        comp[at:at + m] = c
        at += m
    if not shuffle:
        return xs, comp
    perm = rng.permutation(n)
    x = np.empty_like(xs)
    for j in range(d):
        np.take(xs[j], perm, out=x[j])
    return x, comp[perm]


def iso_mixture(n: int, d: int, n_comp: int, sigma: float = 1.0, box: float = 10.0,
                seed: int = 0, weights: str = "equal", offset: float = 0.0,
                shuffle: bool = True):
    """Isotropic Gaussian mixture: means uniform in [-box, box]^d (+ offset on
    every axis), standard deviation ``sigma``.  Returns (X, component, means)."""
    rng = _rng(seed)
    means = rng.uniform(-box, box, size=(n_comp, d)) + offset
    sizes = _component_sizes(rng, n, n_comp, weights)
    blocks = []
    for c in range(n_comp):
        z = rng.standard_normal((d, int(sizes[c])), dtype=np.float32)
        blk = (z.astype(np.float64) * sigma + means[c][:, None]).astype(np.float32)
        blocks.append(blk)
    x, comp = _assemble(rng, blocks, sizes, d, n, shuffle)
    return x, comp, means


def aniso_mixture(n: int, d: int, n_comp: int, sig_lo: float = 0.5, sig_hi: float = 2.0,
                  box: float = 50.0, seed: int = 0, weights: str = "dirichlet",
                  offset: float = 0.0, shuffle: bool = True):
    """Anisotropic Gaussian mixture: per component a Haar rotation R, axis
    standard deviations uniform in [sig_lo, sig_hi], mean uniform in
    [-box, box]^d (+ offset), Dirichlet(1) weights.  x = mean + R diag(sig) z."""
    rng = _rng(seed)
    means = rng.uniform(-box, box, size=(n_comp, d)) + offset
    rots = [haar_rotation(rng, d) for _ in range(n_comp)]
    sigs = rng.uniform(sig_lo, sig_hi, size=(n_comp, d))
    sizes = _component_sizes(rng, n, n_comp, weights)
    blocks = []
    for c in range(n_comp):
        m = int(sizes[c])
        blk = np.empty((d, m), dtype=np.float32)
        step = 1 << 22
        a = rots[c] * sigs[c][None, :]
        for lo in range(0, m, step):
            hi = min(m, lo + step)
            z = rng.standard_normal((d, hi - lo), dtype=np.float32).astype(np.float64)
            blk[:, lo:hi] = (a @ z + means[c][:, None]).astype(np.float32)
        blocks.append(blk)
    x, comp = _assemble(rng, blocks, sizes, d, n, shuffle)
    return x, comp, means


def init_distinct(x: np.ndarray, k: int, seed: int = 1):
    """K distinct points of X chosen uniformly (the paper's initialisation:
    'randomly selecting K points from the dataset').  Returns (mu0 (K, d)
    float64, indices)."""
    n = x.shape[1]
    if k > n:
        raise ValueError("K > N")
    idx = _rng(seed).choice(n, size=k, replace=False)
    return x[:, idx].T.astype(np.float64), idx


def init_kmeanspp(x: np.ndarray, k: int, seed: int = 1, sample: int | None = 1 << 20):
    """k-means++ seeding (D^2 sampling, Arthur & Vassilvitskii 2007) run on a
    seeded uniform subsample of at most ``sample`` points (all points when
    ``sample`` is None or >= N).  Returns (mu0 (K, d) float64, indices into X)."""
    rng = _rng(seed)
    n = x.shape[1]
    if sample is None or sample >= n:
        cand = np.arange(n)
    else:
        cand = np.sort(rng.choice(n, size=sample, replace=False))
    xs = x[:, cand].astype(np.float64)
    m = xs.shape[1]
    chosen = [int(rng.integers(m))]
    d2 = ((xs - xs[:, chosen[0]][:, None]) ** 2).sum(axis=0)
    for _ in range(1, k):
        cum = np.cumsum(d2)
        total = cum[-1]
        if not total > 0:
            pick = int(rng.integers(m))
        else:
            pick = int(np.searchsorted(cum, rng.random() * total, side="right"))
            pick = min(pick, m - 1)
        chosen.append(pick)
        d2 = np.minimum(d2, ((xs - xs[:, pick][:, None]) ** 2).sum(axis=0))
    idx = cand[np.array(chosen)]
    return x[:, idx].T.astype(np.float64), idx


def batch_sizes(count: int, seed: int = 0, n_lo: int = 1_000, n_hi: int = 1_000_000,
                d_choices=(2, 3), k_lo: int = 4, k_hi: int = 64):
    """Sizes of the batched workload: N_i log-uniform in [n_lo, n_hi], d_i
    uniform over ``d_choices``, K_i uniform in [k_lo, k_hi] (at most N_i)."""
    rng = _rng(seed)
    ns = np.maximum(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64), 1)
    ds = rng.choice(np.asarray(d_choices), count).astype(np.int64)
    ks = np.minimum(rng.integers(k_lo, k_hi + 1, count), ns)
    return ns, ds, ks


def batch_instance(i: int, n: int, d: int, k: int, box: float = 10.0, sigma: float = 1.0) -> dict:
    """Instance i of the batched workload: an isotropic mixture of K
    Gaussians (sigma, means U[-box, box]^d, equal weights, data seed
    1000 + i) and K seeded distinct points as the start (seed 2000 + i)."""
    x, _, _ = iso_mixture(int(n), int(d), int(k), sigma=sigma, box=box, seed=1000 + i, weights="equal")
    mu0, _ = init_distinct(x, int(k), seed=2000 + i)
    return dict(x=x, mu0=mu0, n=int(n), d=int(d), k=int(k))


def batch_instances(count: int, seed: int = 0, **kw) -> list:
    """The batched workload (see batch_sizes and batch_instance)."""
    ns, ds, ks = batch_sizes(count, seed, **kw)
    return [batch_instance(i, ns[i], ds[i], ks[i]) for i in range(count)]


# Named workloads.  Each returns dict(x, mu0, k, tol, max_iter, name, desc).
def _c1(scale=1.0):
    n = int(100_000 * scale)
    x, comp, means = iso_mixture(n, 2, 8, sigma=1.0, box=10.0, seed=0, weights="equal")
    mu0, _ = init_distinct(x, 8, seed=1)
    return dict(x=x, mu0=mu0, k=8, tol=1e-6, max_iter=100, comp=comp, means=means,
                desc="N=100000 d=2, 8 isotropic Gaussians sigma=1, means U[-10,10]^2, "
                     "equal weights, seed 0; K=8, 8 seeded distinct points (seed 1)")


def _c2(n=100_000_000):
    x, comp, means = aniso_mixture(n, 3, 32, 0.5, 2.0, box=50.0, seed=0, weights="dirichlet")
    mu0, _ = init_kmeanspp(x, 32, seed=1)
    return dict(x=x, mu0=mu0, k=32, tol=1e-6, max_iter=300, comp=comp, means=means,
                desc=f"N={n} d=3, 32 anisotropic Gaussians (Haar rotations, axis sigma "
                     "U[0.5,2], means U[-50,50]^3, Dirichlet(1) weights), seed 0; K=32, "
                     "k-means++ (seed 1) on a 2^20-point subsample")


def _pa(n=1 << 27):
    x, comp, means = iso_mixture(n, 3, 256, sigma=1.0, box=50.0, seed=2, weights="dirichlet",
                                 offset=1e4)
    mu0, _ = init_kmeanspp(x, 256, seed=3)
    return dict(x=x, mu0=mu0, k=256, tol=1e-6, max_iter=300, comp=comp, means=means,
                desc=f"N={n} d=3, 256 isotropic Gaussians sigma=1, means U[-50,50]^3 + 1e4 "
                     "per axis, Dirichlet(1) weights, seed 2; K=256, k-means++ (seed 3)")


def _pb(n=10_000_000):
    x, comp, means = iso_mixture(n, 64, 1024, sigma=1.0, box=10.0, seed=4, weights="dirichlet")
    mu0, _ = init_distinct(x, 1024, seed=5)
    return dict(x=x, mu0=mu0, k=1024, tol=1e-6, max_iter=300, comp=comp, means=means,
                desc=f"N={n} d=64, 1024 isotropic Gaussians sigma=1, means U[-10,10]^64, "
                     "Dirichlet(1) weights, seed 4; K=1024, distinct points (seed 5)")


WORKLOADS = {
    "plain_2d_n1e5_k8": _c1,
    "plain_3d_n1e8_k32": _c2,
    "precision_offset_3d_n2p27_k256": _pa,
    "precision_highd_64d_n1e7_k1024": _pb,
}


def workload(name: str, **kw) -> dict:
    w = WORKLOADS[name](**kw)
    w["name"] = name
    return w


def paper_sweep():
    """The paper's size sweep (tables 2-5): 2D N in {1e5, 2e5, 5e5} at K=8 and
    3D N in {1e5, 2e5, 4e5, 8e5, 1e6} at K=4, plus table 1's cluster counts
    (2D N = 5e5 and 3D N = 1e6 at K = 4, 8, 11)."""
    out = []
    for n in (100_000, 200_000, 500_000):
        out.append(("2d", n, 8))
    for n in (100_000, 200_000, 400_000, 800_000, 1_000_000):
        out.append(("3d", n, 4))
    for k in (4, 11):
        out.append(("2d", 500_000, k))
    for k in (8, 11):
        out.append(("3d", 1_000_000, k))
    return out


def sweep_case(kind: str, n: int, k: int, seed: int = 0):
    if kind == "2d":
        x, comp, means = iso_mixture(n, 2, k, sigma=1.0, box=10.0, seed=seed)
    else:
        x, comp, means = aniso_mixture(n, 3, k, 0.5, 2.0, box=10.0, seed=seed)
    mu0, _ = init_distinct(x, k, seed=seed + 1)
    return dict(x=x, mu0=mu0, k=k, tol=1e-6, max_iter=300)
