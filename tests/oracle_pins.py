"""Pins for the FP64 oracle: checks against facts that do not come from the
oracle itself (exact rational arithmetic, brute force, closed forms,
invariants, planted means).  Each function takes an ``oracle.Oracle`` and
raises AssertionError on a mismatch, so the same pins can also be run
against deliberately broken copies of the oracle (test_oracle_mutants.py).
"""
from __future__ import annotations

import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _x(rows):
    return np.ascontiguousarray(np.asarray(rows, dtype=np.float32))


def pin_hand_worked(orc):
    """The four-point example worked by hand in tests/golden/hand_worked_1d.json,
    both as d=1 and embedded as (x, 0) in d=2 and as (0, x, 0) in d=3."""
    g = json.load(open(os.path.join(GOLDEN, "hand_worked_1d.json")))
    pts = g["points_1d"]
    for d, axis in ((1, 0), (2, 0), (3, 1)):
        x = np.zeros((d, len(pts)), dtype=np.float32)
        x[axis] = pts
        mu = np.zeros((g["k"], d))
        mu[:, axis] = g["mu0"]
        for st in g["steps"]:
            z, mu_new, counts, e2 = orc.step(x, mu)
            assert list(z) == st["labels"], (d, list(z), st["labels"])
            want = [float(Fraction(v)) for v in st["mu"]]
            assert np.array_equal(mu_new[:, axis], np.array(want)), (mu_new, want)
            other = np.delete(mu_new, axis, axis=1)
            assert np.all(other == 0.0)
            # E2 involves 22/3, which is not a binary fraction: a few ulps apart at most
            assert abs(e2 - float(Fraction(st["E2"]))) <= 4e-16 * max(1.0, e2), (e2, st["E2"])
            assert counts.sum() == len(pts)
            mu = mu_new
        mu0 = np.zeros((g["k"], d))
        mu0[:, axis] = g["mu0"]
        r = orc.run(x, mu0, max_iter=50, tol=1e-6)
        assert r["iters"] == g["T_at_tol_1e-6"] and r["converged"]
        assert r["E"] == 0.0 and r["E2"] == 0.0
        assert r["objective"] == float(Fraction(g["objective_final"]))
        assert list(r["counts"]) == g["counts_final"]
        # stopped early: the labels returned are the ones the returned means
        # were computed from (step 1: z = (0,1,1,1), mu = (0, 22/3))
        r1 = orc.run(x, mu0, max_iter=1, tol=1e-6)
        assert r1["iters"] == 1 and not r1["converged"]
        assert list(r1["labels"]) == g["steps"][0]["labels"] and list(r1["counts"]) == [1, 3]
        assert r1["centroids"][1, axis] == float(Fraction(22, 3))
        # tol = 0 can never be met by the strict test E < tol
        r0 = orc.run(x, mu0, max_iter=7, tol=0.0)
        assert r0["iters"] == 7 and not r0["converged"]
        # the paper's squared error, e_mode = 1: step 2 has E^2 = 185/18 < 11 <= E^2 of step 1
        r1 = orc.run(x, mu0, max_iter=50, tol=11.0, e_mode=1)
        assert r1["iters"] == 2 and r1["converged"]
        assert abs(r1["E2"] - 185 / 18) <= 4e-16 * 185 / 18
        # the same tolerance on the unsquared E stops at step 1 (E = 19/3 < 11)
        r2 = orc.run(x, mu0, max_iter=50, tol=11.0, e_mode=0)
        assert r2["iters"] == 1


def pin_ties(orc):
    """Exact ties go to the lowest centroid index (the reading of an argmin that
    the paper leaves open)."""
    x = _x([[1.0, 3.0, -1.0]])
    assert list(orc.assign(x, np.array([[0.0], [2.0]]))) == [0, 1, 0]
    assert list(orc.assign(x, np.array([[2.0], [0.0]]))) == [0, 0, 1]
    # duplicate centroids: every point goes to the first copy
    xn = _x([[-1.0, 0.5, 1.0]])
    assert list(orc.assign(xn, np.array([[5.0], [0.0], [0.0]]))) == [1, 1, 1]
    # 2-D: (1, 1) is equidistant from (0, 0), (2, 2), (0, 2), (2, 0)
    x2 = _x([[1.0], [1.0]])
    mu = np.array([[2.0, 2.0], [0.0, 2.0], [0.0, 0.0], [2.0, 0.0]])
    assert list(orc.assign(x2, mu)) == [0]


def _brute_labels(x, mu):
    """Minimise sum_i D_i,z_i over all K^N labelings by enumeration."""
    d, n = x.shape
    k = mu.shape[0]
    xd = x.astype(np.float64)
    best, best_l = None, None
    for lab in itertools.product(range(k), repeat=n):
        s = 0.0
        for i, c in enumerate(lab):
            s += math.fsum((float(xd[j, i]) - float(mu[c, j])) ** 2 for j in range(d))
        if best is None or s < best:
            best, best_l = s, lab
    return np.array(best_l), best


def _brute_partition_optimum(x, k):
    """Global minimum of the K-means objective over all labelings (means are
    the group means; empty groups are allowed and contribute nothing)."""
    d, n = x.shape
    xd = x.astype(np.float64)
    best = None
    for lab in itertools.product(range(k), repeat=n):
        lab = np.array(lab)
        s = 0.0
        for c in range(k):
            pts = xd[:, lab == c]
            if pts.shape[1]:
                m = pts.mean(axis=1, keepdims=True)
                s += float(((pts - m) ** 2).sum())
        if best is None or s < best:
            best = s
    return best


def pin_brute_force(orc, cases=24, seed=123):
    """Tiny random cases (N <= 7, K <= 3): the reassignment equals the labeling
    that minimises the objective over all K^N labelings; the update's centroids
    are stationary points of the objective for those labels; Lloyd's final
    objective is never below the global optimum found by enumeration."""
    rng = np.random.default_rng(seed)
    for c in range(cases):
        d = 1 + c % 3
        n = 3 + c % 5
        k = 1 + c % 3
        x = rng.normal(size=(d, n)).astype(np.float32)
        mu = rng.normal(size=(k, d))
        z = orc.assign(x, mu)
        zb, _ = _brute_labels(x, mu)
        assert np.array_equal(z, zb), (c, z, zb)
        mu1, counts = orc.update(x, z, mu)
        xd = x.astype(np.float64)
        for q in range(k):
            m = z == q
            assert counts[q] == int(m.sum())
            if m.any():
                grad = (xd[:, m] - mu1[q][:, None]).sum(axis=1)
                assert np.all(np.abs(grad) <= 1e-12 * (1 + np.abs(xd[:, m]).sum(axis=1)))
            else:
                assert np.array_equal(mu1[q], mu[q])
        if k <= 3 and n <= 6:
            opt = _brute_partition_optimum(x, k)
            r = orc.run(x, xd[:, :k].T.copy(), max_iter=100, tol=1e-12)
            assert r["objective"] >= opt - 1e-9 * (1 + opt)


def pin_closed_forms(orc):
    rng = np.random.default_rng(7)
    # K = 1: the only centroid moves to the global mean, then stays (T = 2)
    x = rng.normal(3.0, 2.0, size=(3, 1000)).astype(np.float32)
    r = orc.run(x, x[:, :1].T.astype(np.float64), max_iter=10, tol=1e-12)
    mean = np.array([math.fsum(map(float, row)) / x.shape[1] for row in x])
    assert np.allclose(r["centroids"][0], mean, rtol=0, atol=1e-13)
    assert r["iters"] == 2 and r["E"] == 0.0
    assert np.all(r["labels"] == 0) and r["counts"][0] == 1000
    # K = N with mu0 = X: every point is its own cluster, nothing moves (T = 1)
    x = rng.normal(size=(2, 9)).astype(np.float32)
    r = orc.run(x, x.T.astype(np.float64), max_iter=10, tol=1e-9)
    assert list(r["labels"]) == list(range(9)) and r["iters"] == 1 and r["E"] == 0.0
    assert r["objective"] == 0.0
    # 1-D, K = 2: the boundary is the midpoint of the two centroids
    xs = np.linspace(-5, 5, 101).astype(np.float32)[None, :]
    z = orc.assign(xs, np.array([[-1.0], [3.0]]))
    assert np.array_equal(z, (xs[0].astype(np.float64) > 1.0).astype(np.int32))
    # an empty cluster keeps its previous centre
    x = _x([[0.0, 1.0, 2.0]])
    mu0 = np.array([[1.0], [100.0]])
    z, mu1, counts, e2 = orc.step(x, mu0)
    assert list(counts) == [3, 0] and mu1[1, 0] == 100.0 and mu1[0, 0] == 1.0 and e2 == 0.0


def pin_invariants(orc, n=200_000, seed=11):
    """On a mixture larger than several of the oracle's 65,536-point chunks:
    labels are argmins (checked against an independently written distance
    table), centroids are the means of their points, counts add up to N,
    sum_k n_k mu_k = sum_i x_i, the objective never increases, and a converged
    fixed point stays fixed with E == 0 exactly."""
    import synth
    x, _, _ = synth.iso_mixture(n, 2, 6, sigma=2.0, box=8.0, seed=seed)
    mu, _ = synth.init_distinct(x, 6, seed=seed + 1)
    xd = x.astype(np.float64)
    prev_obj = math.inf
    for t in range(40):
        z, mu1, counts, e2 = orc.step(x, mu)
        # argmin check on a sample, with an independent squared-distance table
        sel = np.arange(0, n, 97)
        dt = np.stack([((xd[:, sel] - mu[c][:, None]) ** 2).sum(axis=0) for c in range(mu.shape[0])])
        srt = np.sort(dt, axis=0)
        clear = (srt[1] - srt[0]) > 1e-9 * srt[1]
        assert np.array_equal(z[sel][clear], np.argmin(dt, axis=0)[clear])
        assert counts.sum() == n
        assert np.array_equal(counts, np.bincount(z, minlength=mu.shape[0]))
        for c in range(mu.shape[0]):
            if counts[c]:
                m = xd[:, z == c].mean(axis=1)
                assert np.allclose(mu1[c], m, rtol=1e-12, atol=1e-12)
        tot = (counts[:, None] * mu1).sum(axis=0)
        assert np.allclose(tot, xd.sum(axis=1), rtol=1e-11, atol=1e-9)
        obj = orc.objective(x, mu1, z)
        assert obj <= prev_obj * (1 + 1e-12)
        prev_obj = obj
        err = orc.error2(mu1, mu)
        assert err == e2
        mu = mu1
        if e2 == 0.0:
            break
    assert e2 == 0.0, "did not reach a fixed point"
    z2, mu2, counts2, e22 = orc.step(x, mu)
    assert e22 == 0.0 and np.array_equal(z2, z) and np.array_equal(mu2, mu)


def pin_planted_means(orc, seed=5):
    """Well-separated blobs (centres >= 20 sigma apart) with one starting point
    per blob: Lloyd recovers the generating components exactly (labels equal
    component ids up to a permutation) and each centroid is within
    4 sigma / sqrt(n_k) of its component's generating mean."""
    import synth
    rng = np.random.default_rng(seed)
    kc, d, n, sigma = 7, 3, 70_000, 1.0
    grid = np.array(list(itertools.product([-30.0, 0.0, 30.0], repeat=3)))
    means = grid[rng.choice(len(grid), size=kc, replace=False)]
    xs, comp = [], []
    for c in range(kc):
        xs.append(rng.normal(size=(d, n // kc)) * sigma + means[c][:, None])
        comp.append(np.full(n // kc, c))
    x = np.concatenate(xs, axis=1).astype(np.float32)
    comp = np.concatenate(comp)
    perm = rng.permutation(x.shape[1])
    x, comp = np.ascontiguousarray(x[:, perm]), comp[perm]
    first = np.array([np.flatnonzero(comp == c)[0] for c in range(kc)])
    mu0 = x[:, first].T.astype(np.float64)
    r = orc.run(x, mu0, max_iter=50, tol=1e-9)
    assert r["converged"]
    assert np.array_equal(r["labels"], comp.astype(np.int32))
    for c in range(kc):
        nk = r["counts"][c]
        assert np.linalg.norm(r["centroids"][c] - means[c]) <= 4 * sigma * math.sqrt(d) / math.sqrt(nk)


ALL_PINS = [pin_hand_worked, pin_ties, pin_brute_force, pin_closed_forms, pin_invariants,
            pin_planted_means]
