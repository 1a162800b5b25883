"""FP64 CPU oracle of Lloyd's K-means -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_2405_12052_gb300``) never loads it and shares no code with it.

The arithmetic lives in ``lloyd.c`` (plain C, double precision, OpenMP over
fixed chunks so results do not depend on the thread count); this module only
builds it with gcc and marshals numpy arrays.  Each wrapper names the step of
the paper it restates:

* ``assign``     -- reassignment, z_i = argmin_k ||x_i - mu_k||^2
                    (section "The Lloyd's algorithm", step 2);
* ``update``     -- mean calculation, mu_k = sum 1(z_i=k) x_i / sum 1(z_i=k)
                    (same section, step 3);
* ``error2``     -- E^2 = sum_k ||mu_k^{t+1} - mu_k^t||^2
                    (section "Serial Lloyd's algorithm");
* ``run``        -- the loop of that section until E < tol or max_iter;
* ``objective``  -- sum_i ||x_i - mu_{z_i}||^2 (the abstract's objective);
* ``kmeanspp``   -- k-means++ seeding with caller-supplied uniforms (not in
                    the paper, which seeds with K random points).

Pins: every function is checked in ``tests/test_oracle_*.py`` against brute
force, closed forms, a hand-worked example, invariants and planted means.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lloyd.c")
_LIB = os.path.join(_HERE, "liblloyd_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile lloyd.c with gcc (no FMA contraction) into liblloyd_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path: str | None = None):
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_assign.argtypes = [P, i64, i64, i32, i32, P, P, P]
    lib.orc_assign.restype = ctypes.c_int
    lib.orc_update.argtypes = [P, i64, i64, i32, i32, P, P, P, P]
    lib.orc_update.restype = ctypes.c_int
    lib.orc_error2.argtypes = [i32, i32, P, P]
    lib.orc_error2.restype = f64
    lib.orc_objective.argtypes = [P, i64, i64, i32, P, P]
    lib.orc_objective.restype = f64
    lib.orc_step.argtypes = [P, i64, i64, i32, i32, P, P, P, P]
    lib.orc_step.restype = f64
    lib.orc_run.argtypes = [P, i64, i64, i32, i32, P, i32, f64, i32, P, P, P, P, P, P, P]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_kmeanspp.argtypes = [P, i64, i64, i32, i32, P, P, P]
    lib.orc_kmeanspp.restype = ctypes.c_int
    return lib


class Oracle:
    """Handle on one compiled copy of the oracle (default: the committed source)."""

    def __init__(self, lib_path: str | None = None):
        self.lib = _load(lib_path)

    # -- helpers ---------------------------------------------------------
    @staticmethod
    def _x(x):
        x = np.asarray(x)
        if x.dtype != np.float32 or x.ndim != 2:
            raise TypeError("X must be a float32 array of shape (d, N)")
        if not x.flags.c_contiguous:
            x = np.ascontiguousarray(x)
        return x, x.shape[0], x.shape[1], x.strides[0] // 4

    @staticmethod
    def _mu(mu, k, d):
        mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(k, d))
        return mu

    def threads(self) -> int:
        return int(self.lib.orc_threads())

    # -- paper steps -----------------------------------------------------
    def assign(self, x, mu, with_dmin: bool = False):
        x, d, n, ld = self._x(x)
        k = int(np.asarray(mu).size // d)
        mu = self._mu(mu, k, d)
        z = np.empty(n, dtype=np.int32)
        dmin = np.empty(n, dtype=np.float64) if with_dmin else None
        self.lib.orc_assign(x.ctypes.data, ld, n, d, k, mu.ctypes.data, z.ctypes.data,
                            dmin.ctypes.data if with_dmin else None)
        return (z, dmin) if with_dmin else z

    def update(self, x, z, mu_prev):
        x, d, n, ld = self._x(x)
        k = int(np.asarray(mu_prev).size // d)
        mu_prev = self._mu(mu_prev, k, d)
        z = np.ascontiguousarray(z, dtype=np.int32)
        if z.shape != (n,) or (n and (z.min() < 0 or z.max() >= k)):
            raise ValueError("labels must be N values in 0..K-1")
        mu_next = np.empty_like(mu_prev)
        counts = np.empty(k, dtype=np.int64)
        empty = self.lib.orc_update(x.ctypes.data, ld, n, d, k, z.ctypes.data,
                                    mu_prev.ctypes.data, mu_next.ctypes.data, counts.ctypes.data)
        if empty < 0:
            raise MemoryError("oracle update: allocation failed")
        return mu_next, counts

    def error2(self, a, b) -> float:
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        if a.shape != b.shape or a.ndim != 2:
            raise ValueError("centroid arrays must have the same (K, d) shape")
        return float(self.lib.orc_error2(a.shape[0], a.shape[1], a.ctypes.data, b.ctypes.data))

    def objective(self, x, mu, z) -> float:
        x, d, n, ld = self._x(x)
        k = int(np.asarray(mu).size // d)
        mu = self._mu(mu, k, d)
        z = np.ascontiguousarray(z, dtype=np.int32)
        return float(self.lib.orc_objective(x.ctypes.data, ld, n, d, mu.ctypes.data, z.ctypes.data))

    def step(self, x, mu_in):
        """One Lloyd step: returns (z, mu_out, counts, E2)."""
        x, d, n, ld = self._x(x)
        k = int(np.asarray(mu_in).size // d)
        mu_in = self._mu(mu_in, k, d)
        z = np.empty(n, dtype=np.int32)
        mu_out = np.empty_like(mu_in)
        counts = np.empty(k, dtype=np.int64)
        e2 = self.lib.orc_step(x.ctypes.data, ld, n, d, k, mu_in.ctypes.data, z.ctypes.data,
                               mu_out.ctypes.data, counts.ctypes.data)
        if e2 < 0:
            raise MemoryError("oracle step: allocation failed")
        return z, mu_out, counts, float(e2)

    def run(self, x, mu0, max_iter: int, tol: float, e_mode: int = 0) -> dict:
        x, d, n, ld = self._x(x)
        k = int(np.asarray(mu0).size // d)
        mu0 = self._mu(mu0, k, d)
        z = np.empty(n, dtype=np.int32)
        mu = np.empty_like(mu0)
        counts = np.empty(k, dtype=np.int64)
        iters = ctypes.c_int32(0)
        e, e2, obj = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        st = self.lib.orc_run(x.ctypes.data, ld, n, d, k, mu0.ctypes.data, int(max_iter),
                              float(tol), int(e_mode), z.ctypes.data, mu.ctypes.data,
                              counts.ctypes.data, ctypes.byref(iters), ctypes.byref(e),
                              ctypes.byref(e2), ctypes.byref(obj))
        if st < 0:
            raise MemoryError("oracle run: allocation failed")
        return dict(labels=z, centroids=mu, counts=counts, iters=int(iters.value),
                    E=float(e.value), E2=float(e2.value), objective=float(obj.value),
                    converged=(st == 0))

    def kmeanspp(self, x, k: int, u):
        """k-means++ seeding with the K uniforms ``u`` in [0, 1) supplied."""
        x, d, n, ld = self._x(x)
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape != (k,):
            raise ValueError("need K uniforms")
        mu = np.empty((k, d), dtype=np.float64)
        idx = np.empty(k, dtype=np.int64)
        if self.lib.orc_kmeanspp(x.ctypes.data, ld, n, d, k, u.ctypes.data, mu.ctypes.data,
                                 idx.ctypes.data) < 0:
            raise MemoryError("oracle k-means++: allocation failed")
        return mu, idx


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
