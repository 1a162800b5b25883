"""The TF32 split of the tensor-core screen (dist_path="tensor", d <= 3,
K <= 32), checked on the CPU: with xh = x~ with its 13 low significand bits
cleared, xl = x~ - xh, ah likewise for a coefficient, al = the TF32 head of
a - ah, and n = nh + nm + nl (three TF32 heads of the successive
remainders), the products the kernel forms

    xh.ah + tf32(xl).ah + xh.al + nh + nm + nl

differ from n + x~.a (computed here in FP64, where every product of two FP32
numbers is exact; the sums' own rounding, a few 2^-53 of the terms, is
allowed for) by at most 3 * 2^-20 * sum_j |x~_j a_j| -- the split part of the
kernel's error bound (the accumulation part depends on the tensor core's
unknown summation order and is bounded separately).  Also: the n split is
exact, and xh, al, nh, nm, nl are exact TF32 numbers.
"""
import numpy as np


def tf32_head(v):
    b = np.asarray(v, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def is_tf32(v):
    return np.all((np.asarray(v, dtype=np.float32).view(np.uint32) & np.uint32(0x1FFF)) == 0)


def test_split_error_within_bound():
    rng = np.random.default_rng(7)
    for trial in range(200):
        d = 3
        x = (rng.standard_normal(d) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
        a = (rng.standard_normal(d) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
        n = np.float32(rng.uniform(1.0, 2.0))
        xh = tf32_head(x)
        xl = (x - xh).astype(np.float32)                # exact in FP32
        assert np.array_equal(xh.astype(np.float64) + xl.astype(np.float64), x.astype(np.float64))
        xl_hw = tf32_head(xl)                           # the hardware may cut xl to TF32 (worst case)
        ah = tf32_head(a)
        al = tf32_head((a - ah).astype(np.float32))
        nh = tf32_head(n)
        nr = np.float32(n - nh)
        nm = tf32_head(nr)
        nl = np.float32(nr - nm)
        assert is_tf32(xh) and is_tf32(ah) and is_tf32(al) and is_tf32(nh) and is_tf32(nm) and is_tf32(nl)
        assert np.float64(nh) + np.float64(nm) + np.float64(nl) == np.float64(n)   # exact
        X, A = x.astype(np.float64), a.astype(np.float64)
        got = (np.sum(xh.astype(np.float64) * ah.astype(np.float64)) +
               np.sum(xl_hw.astype(np.float64) * ah.astype(np.float64)) +
               np.sum(xh.astype(np.float64) * al.astype(np.float64)) + np.float64(nh) + np.float64(nm) +
               np.float64(nl))
        want = np.float64(n) + np.sum(X * A)
        bound = 3 * 2.0 ** -20 * np.sum(np.abs(X * A))
        # FP64 here is exact up to its own rounding of at most a few 2^-53
        # relative steps of the terms, far below the bound
        assert abs(got - want) <= bound + 1e-15 * (abs(want) + np.sum(np.abs(X * A))), (trial, got - want, bound)


def test_bound_is_not_loose_by_orders():
    """The split error does reach a visible fraction of the bound for some
    inputs (a planted mistake such as dropping the xh.al term would exceed
    it)."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(2000):
        x = rng.uniform(1, 2, 3).astype(np.float32)
        a = rng.uniform(1, 2, 3).astype(np.float32)
        xh = tf32_head(x); xl = tf32_head((x - xh).astype(np.float32))
        ah = tf32_head(a); al = tf32_head((a - ah).astype(np.float32))
        X, A = x.astype(np.float64), a.astype(np.float64)
        got = np.sum(xh * ah.astype(np.float64)) + np.sum(xl * ah.astype(np.float64)) + np.sum(xh * al.astype(np.float64))
        err = abs(got - np.sum(X * A)) / (3 * 2.0 ** -20 * np.sum(np.abs(X * A)))
        worst = max(worst, err)
        # without the xh.al term the error is of order 2^-10, far above the bound
        got_bad = np.sum(xh * ah.astype(np.float64)) + np.sum(xl * ah.astype(np.float64))
        assert abs(got_bad - np.sum(X * A)) > 3 * 2.0 ** -20 * np.sum(np.abs(X * A)) or np.all(al == 0)
    assert 0.05 < worst <= 1.0
