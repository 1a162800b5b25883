"""Python binding of libkm.so, the GB300 (sm_103a) Lloyd's K-means library.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels behind the C ABI declared in ``include/km.h``.  There is no CPU
fallback; if ``libkm.so`` is missing, ``lib()`` raises.  Points may be numpy
arrays (host memory) or CUDA torch tensors (device memory); torch is used
only for device buffers and the current stream.

Layout follows the paper (X in R^{d x N}): coordinate j of point i at
``x[j, i]``.  Labels are 0..K-1.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

__all__ = ["KMeans", "KMError", "lib", "header_symbols", "build", "LIB_PATH", "HEADER"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "km.h")

KM_OK, KM_NOT_CONVERGED = 0, 1
STATUS = {0: "KM_OK", 1: "KM_NOT_CONVERGED", -1: "KM_EINVAL", -2: "KM_ENOMEM", -3: "KM_ECUDA",
          -4: "KM_ESTATE", -5: "KM_ETIMEOUT", -6: "KM_ENUMERIC"}
KM_SOA_DxN, KM_AOS_NxD = 0, 1
KM_HOST, KM_DEVICE_COPY, KM_DEVICE_BORROW = 0, 1, 2
E_MODES = {"norm": 0, "squared": 1}


class KMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("e_mode", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("tie_rel", ctypes.c_double), ("stream", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("e", ctypes.c_double),
                ("e2", ctypes.c_double), ("flagged", ctypes.c_int64),
                ("fp64_decided", ctypes.c_int64), ("empty_clusters", ctypes.c_int32),
                ("overflowed", ctypes.c_int64), ("path", ctypes.c_int32)]


_lib = None


def build(force: bool = False) -> str:
    from . import native_build
    return native_build.build(force=force)


def lib(path: str | None = None):
    """Load libkm.so (raises if it has not been built)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2405_12052_gb300.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(p)
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    st = ctypes.c_int
    L.km_default_options.argtypes = [ctypes.POINTER(_Options)]
    L.km_default_options.restype = None
    L.km_version.restype = ctypes.c_char_p
    L.km_create.argtypes = [ctypes.POINTER(P), i64, i32, i32, ctypes.POINTER(_Options)]
    L.km_create.restype = st
    L.km_set_points.argtypes = [P, P, i64, i32, i32]
    L.km_set_points.restype = st
    L.km_set_init.argtypes = [P, P]
    L.km_set_init.restype = st
    L.km_step.argtypes = [P, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    L.km_step.restype = st
    L.km_run.argtypes = [P, i32, f64, P, P, ctypes.POINTER(i32), ctypes.POINTER(f64)]
    L.km_run.restype = st
    L.km_get_labels.argtypes = [P, P, i32]
    L.km_get_labels.restype = st
    L.km_get_centroids.argtypes = [P, P, i32]
    L.km_get_centroids.restype = st
    L.km_get_counts.argtypes = [P, P]
    L.km_get_counts.restype = st
    L.km_get_stats.argtypes = [P, ctypes.POINTER(_Stats)]
    L.km_get_stats.restype = st
    L.km_device_buffers.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(i64), ctypes.POINTER(P),
                                    ctypes.POINTER(P)]
    L.km_device_buffers.restype = st
    L.km_begin.argtypes = [P, i32, f64]
    L.km_begin.restype = st
    L.km_assign_async.argtypes = [P]
    L.km_assign_async.restype = st
    L.km_update_async.argtypes = [P]
    L.km_update_async.restype = st
    L.km_sync.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(f64), ctypes.POINTER(i32)]
    L.km_sync.restype = st
    L.km_stream.argtypes = [P]
    L.km_stream.restype = P
    L.km_lloyd_step_noalloc.argtypes = [P, i64, i64, i32, i32, P, P, P, P, P, P, ctypes.c_char_p, i32]
    L.km_lloyd_step_noalloc.restype = st
    L.km_last_error.argtypes = [P]
    L.km_last_error.restype = ctypes.c_char_p
    L.km_destroy.argtypes = [P]
    L.km_destroy.restype = None
    if path is None:
        _lib = L
    return L


def header_symbols(header: str = HEADER) -> list[str]:
    """Names of the functions km.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(km_[a-z0-9_]+)\s*\(", text)))


def _is_torch(t) -> bool:
    return type(t).__module__.startswith("torch")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return ctypes.c_void_p(None)


class KMeans:
    """One clustering problem: N points of dimension d, K clusters."""

    def __init__(self, n: int, d: int, k: int, *, e_mode: str = "norm", tie_rel: float = 1e-5,
                 use_graph: bool = True, stream=None):
        self._L = lib()
        self.n, self.d, self.k = int(n), int(d), int(k)
        opt = _Options()
        self._L.km_default_options(ctypes.byref(opt))
        opt.e_mode = E_MODES[e_mode]
        opt.use_graph = 1 if use_graph else 0
        opt.tie_rel = float(tie_rel)
        if stream is None:
            opt.stream = _current_stream()
        elif isinstance(stream, int):
            opt.stream = ctypes.c_void_p(stream)
        else:
            opt.stream = ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
        h = ctypes.c_void_p()
        s = self._L.km_create(ctypes.byref(h), self.n, self.d, self.k, ctypes.byref(opt))
        self._h = h
        self._check(s)
        self._keep = None

    # -- helpers --------------------------------------------------------
    def _check(self, s: int) -> int:
        if s < 0:
            msg = self._L.km_last_error(self._h).decode() if self._h else ""
            raise KMError(s, msg)
        return s

    def close(self):
        if getattr(self, "_h", None):
            self._L.km_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API -------------------------------------------------------------
    def set_points(self, x, layout: str = "dxn", borrow: bool = False):
        """x: (d, N) float32 (layout 'dxn', the paper's X) or (N, d) ('nxd');
        numpy (host) or a CUDA torch tensor (device; ``borrow`` keeps the
        pointer instead of copying)."""
        lay = KM_SOA_DxN if layout == "dxn" else KM_AOS_NxD
        if _is_torch(x):
            import torch
            if x.dtype != torch.float32 or x.dim() != 2:
                raise TypeError("points must be a 2-D float32 tensor")
            if x.stride(1) != 1:
                x = x.contiguous()
            ld = x.stride(0)
            mem = KM_DEVICE_BORROW if (borrow and x.is_cuda) else (KM_DEVICE_COPY if x.is_cuda else KM_HOST)
            if not x.is_cuda:
                x = x.numpy()
                ptr = x.ctypes.data
            else:
                ptr = x.data_ptr()
        else:
            x = np.asarray(x)
            if x.dtype != np.float32 or x.ndim != 2:
                raise TypeError("points must be a 2-D float32 array")
            if x.strides[1] != 4:
                x = np.ascontiguousarray(x)
            ld = x.strides[0] // 4
            ptr = x.ctypes.data
            mem = KM_HOST
        shape_ok = (x.shape == (self.d, self.n)) if lay == KM_SOA_DxN else (x.shape == (self.n, self.d))
        if not shape_ok:
            raise ValueError(f"points shape {tuple(x.shape)} does not match N={self.n}, d={self.d}")
        self._check(self._L.km_set_points(self._h, ptr, int(ld), lay, mem))
        self._keep = x if mem == KM_DEVICE_BORROW else None

    def set_init(self, mu0):
        mu0 = np.ascontiguousarray(np.asarray(mu0, dtype=np.float64).reshape(self.k, self.d))
        self._check(self._L.km_set_init(self._h, mu0.ctypes.data))

    def step(self):
        e, e2 = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.km_step(self._h, ctypes.byref(e), ctypes.byref(e2)))
        return e.value, e2.value

    def run(self, max_iter: int, tol: float, want_labels: bool = True) -> dict:
        labels = np.empty(self.n, dtype=np.int32) if want_labels else None
        mu = np.empty((self.k, self.d), dtype=np.float64)
        it, e = ctypes.c_int32(), ctypes.c_double()
        s = self._check(self._L.km_run(self._h, int(max_iter), float(tol),
                                       labels.ctypes.data if want_labels else None,
                                       mu.ctypes.data, ctypes.byref(it), ctypes.byref(e)))
        return dict(labels=labels, centroids=mu, iters=it.value, E=e.value,
                    converged=(s == KM_OK))

    # -- asynchronous pieces of a step (no synchronization) ---------------
    def begin(self, max_iter: int, tol: float):
        self._check(self._L.km_begin(self._h, int(max_iter), float(tol)))

    def assign_async(self):
        self._check(self._L.km_assign_async(self._h))

    def update_async(self):
        self._check(self._L.km_update_async(self._h))

    def sync(self) -> dict:
        it, e, done = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
        self._check(self._L.km_sync(self._h, ctypes.byref(it), ctypes.byref(e), ctypes.byref(done)))
        return dict(iters=it.value, E=e.value, done=bool(done.value))

    @property
    def stream_handle(self) -> int:
        return int(self._L.km_stream(self._h) or 0)

    def labels(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        self._check(self._L.km_get_labels(self._h, out.ctypes.data, KM_HOST))
        return out

    def labels_host_into(self, tensor):
        """Copy labels into a host (e.g. pinned) int32 torch tensor of N elements."""
        self._check(self._L.km_get_labels(self._h, tensor.data_ptr(), KM_HOST))

    def labels_into(self, tensor):
        """Copy labels into a CUDA int32 torch tensor of N elements."""
        self._check(self._L.km_get_labels(self._h, tensor.data_ptr(), KM_DEVICE_COPY))

    def centroids(self) -> np.ndarray:
        out = np.empty((self.k, self.d), dtype=np.float64)
        self._check(self._L.km_get_centroids(self._h, out.ctypes.data, KM_HOST))
        return out

    def counts(self) -> np.ndarray:
        out = np.empty(self.k, dtype=np.int64)
        self._check(self._L.km_get_counts(self._h, out.ctypes.data))
        return out

    def stats(self) -> dict:
        s = _Stats()
        self._check(self._L.km_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def device_buffers(self) -> dict:
        P = ctypes.c_void_p
        pts, lab, mu = P(), P(), P()
        ld = ctypes.c_int64()
        self._check(self._L.km_device_buffers(self._h, ctypes.byref(pts), ctypes.byref(ld),
                                              ctypes.byref(lab), ctypes.byref(mu)))
        return dict(points=pts.value, ld=ld.value, labels=lab.value, centroids=mu.value)
