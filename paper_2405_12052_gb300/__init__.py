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

__all__ = ["KMeans", "KMeansBatch", "SetNet", "KMError", "lib", "header_symbols", "build", "LIB_PATH", "HEADER",
           "sets_mean", "sets_rotate"]

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
                ("tie_rel", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("label_policy", ctypes.c_int32), ("dist_path", ctypes.c_int32),
                ("tc_operands", ctypes.c_int32), ("label_bytes", ctypes.c_int32)]


LABEL_POLICIES = {"every_step": 0, "final": 1}
DIST_PATHS = {"auto": 0, "simt": 1, "tensor": 2}
TC_OPERANDS = {"bf16": 0, "f16": 1}


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("e", ctypes.c_double),
                ("e2", ctypes.c_double), ("flagged", ctypes.c_int64),
                ("fp64_decided", ctypes.c_int64), ("empty_clusters", ctypes.c_int32),
                ("overflowed", ctypes.c_int64), ("path", ctypes.c_int32)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("flagged", ctypes.c_int64), ("fp64_decided", ctypes.c_int64), ("tile_points", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("grid", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("tune_candidates", ctypes.c_int32),
                ("tune_ms", ctypes.c_float * 8)]


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
    L.km_sets_mean.argtypes = [P, i64, i32, i32, i32, P, P]
    L.km_sets_mean.restype = st
    L.km_sets_rotate_f32.argtypes = [P, i64, i32, i32, i32, P, P, i64, i32, P, P]
    L.km_sets_rotate_f32.restype = st
    L.km_sets_rotate_f64.argtypes = [P, i64, i32, i32, i32, P, P, i64, i32, P, P]
    L.km_sets_rotate_f64.restype = st
    L.km_grid_exponent.argtypes = [P, ctypes.POINTER(i32)]
    L.km_grid_exponent.restype = st
    L.km_set_grid_exponent.argtypes = [P, i32]
    L.km_set_grid_exponent.restype = st
    L.km_shard_totals.argtypes = [P, P, i32]
    L.km_shard_totals.restype = st
    L.km_shard_update.argtypes = [P, P, i32, i32]
    L.km_shard_update.restype = st
    L.km_stream.argtypes = [P]
    L.km_stream.restype = P
    L.km_lloyd_step_noalloc.argtypes = [P, i64, i64, i32, i32, P, P, P, P, P, P, ctypes.c_char_p, i32]
    L.km_lloyd_step_noalloc.restype = st
    L.km_last_error.argtypes = [P]
    L.km_last_error.restype = ctypes.c_char_p
    L.km_destroy.argtypes = [P]
    L.km_destroy.restype = None
    L.km_init_kmeanspp.argtypes = [P, P, P, P]
    L.km_init_kmeanspp.restype = st
    L.km_setnet_create.argtypes = [ctypes.POINTER(P), i32, i32, P]
    L.km_setnet_create.restype = st
    L.km_setnet_param_count.argtypes = [P]
    L.km_setnet_param_count.restype = i64
    L.km_setnet_dims.argtypes = [P, ctypes.POINTER(i32)]
    L.km_setnet_dims.restype = i32
    L.km_setnet_stream.argtypes = [P]
    L.km_setnet_stream.restype = P
    L.km_setnet_set_params.argtypes = [P, P]
    L.km_setnet_set_params.restype = st
    L.km_setnet_get_params.argtypes = [P, P]
    L.km_setnet_get_params.restype = st
    L.km_setnet_get_grads.argtypes = [P, P]
    L.km_setnet_get_grads.restype = st
    L.km_setnet_loss_grad.argtypes = [P, P, P, i32, i32, i32, ctypes.POINTER(ctypes.c_float)]
    L.km_setnet_loss_grad.restype = st
    L.km_setnet_adam.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.km_setnet_adam.restype = st
    L.km_setnet_train_step.argtypes = [P, P, P, i32, i32, i32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
    L.km_setnet_train_step.restype = st
    L.km_setnet_predict.argtypes = [P, P, i32, i32, i32, P]
    L.km_setnet_predict.restype = st
    L.km_setnet_last_error.argtypes = [P]
    L.km_setnet_last_error.restype = ctypes.c_char_p
    L.km_setnet_destroy.argtypes = [P]
    L.km_setnet_destroy.restype = None
    L.km_debug_fail_alloc_after.argtypes = [i64]
    L.km_debug_fail_alloc_after.restype = None
    L.km_selftest_bounded_wait.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(f64)]
    L.km_selftest_bounded_wait.restype = st
    L.km_get_labels_u8.argtypes = [P, P, i32]
    L.km_get_labels_u8.restype = st
    L.km_write_labels.argtypes = [P]
    L.km_write_labels.restype = st
    L.km_objective.argtypes = [P, ctypes.POINTER(f64)]
    L.km_objective.restype = st
    L.km_init_learned.argtypes = [P, P, i32, ctypes.c_uint64, P]
    L.km_init_learned.restype = st
    L.km_batch_create.argtypes = [ctypes.POINTER(P), i32, P, P, P, ctypes.POINTER(_Options)]
    L.km_batch_create.restype = st
    L.km_batch_set_points.argtypes = [P, P, i32]
    L.km_batch_set_points.restype = st
    L.km_batch_set_init.argtypes = [P, P]
    L.km_batch_set_init.restype = st
    L.km_batch_objective.argtypes = [P, P]
    L.km_batch_objective.restype = st
    L.km_batch_set_shape.argtypes = [P, i32, i32]
    L.km_batch_set_shape.restype = st
    L.km_batch_tune.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.km_batch_tune.restype = st
    L.km_batch_run.argtypes = [P, i32, f64, P, P, P, P, P]
    L.km_batch_run.restype = st
    L.km_batch_get_counts.argtypes = [P, P]
    L.km_batch_get_counts.restype = st
    L.km_batch_get_info.argtypes = [P, ctypes.POINTER(_BatchInfo)]
    L.km_batch_get_info.restype = st
    L.km_batch_last_error.argtypes = [P]
    L.km_batch_last_error.restype = ctypes.c_char_p
    L.km_batch_destroy.argtypes = [P]
    L.km_batch_destroy.restype = None
    if path is None:
        _lib = L
    return L


def selftest_bounded_wait() -> dict:
    """Run the device-side bounded-wait self-test (a wait on an mbarrier that
    nothing arrives on must give up by its limit)."""
    g, ms = ctypes.c_int32(), ctypes.c_double()
    s = lib().km_selftest_bounded_wait(ctypes.byref(g), ctypes.byref(ms))
    if s != 0:
        raise KMError(s, "bounded-wait self-test failed")
    return {"gave_up": bool(g.value), "elapsed_ms": ms.value}


def debug_fail_alloc_after(n: int):
    """Testing hook: after n more device allocations by the library, the next
    one fails as out of memory (n < 0: off)."""
    lib().km_debug_fail_alloc_after(int(n))


def header_symbols(header: str = HEADER) -> list[str]:
    """Names of the functions km.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(km_[a-z0-9_]+)\s*\(", text)))


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return "unknown"


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
                 use_graph: bool = True, stream=None, label_policy: str = "every_step",
                 dist_path: str = "auto", tc_operands: str = "bf16", label_bytes: int = 4):
        self._L = lib()
        self.n, self.d, self.k = int(n), int(d), int(k)
        opt = _Options()
        self._L.km_default_options(ctypes.byref(opt))
        opt.e_mode = E_MODES[e_mode]
        self._e_mode = opt.e_mode
        opt.label_policy = LABEL_POLICIES[label_policy]
        opt.dist_path = DIST_PATHS[dist_path]
        opt.tc_operands = TC_OPERANDS[tc_operands]
        opt.label_bytes = int(label_bytes)
        self.label_bytes = int(label_bytes)
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

    def init_kmeanspp(self, u):
        """k-means++ seeding on the GPU with the K uniforms ``u`` in [0, 1);
        sets the starting centroids and returns (mu0 (K, d), indices)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape != (self.k,):
            raise ValueError("need K uniforms")
        mu = np.empty((self.k, self.d), dtype=np.float64)
        idx = np.empty(self.k, dtype=np.int64)
        self._check(self._L.km_init_kmeanspp(self._h, u.ctypes.data, mu.ctypes.data, idx.ctypes.data))
        return mu, idx

    def write_labels(self):
        """Labels of the current centroids (one assignment pass; for the
        "final" label policy)."""
        self._check(self._L.km_write_labels(self._h))

    def objective(self) -> float:
        """sum_i ||x_i - mu_{z_i}||^2 of the last step's labels and the
        current centroids (FP64, the oracle's summation order)."""
        o = ctypes.c_double()
        self._check(self._L.km_objective(self._h, ctypes.byref(o)))
        return o.value

    def init_learned(self, net: "SetNet", sample_n: int = 4096, seed: int = 0):
        """Starting centroids from the set network on a seeded sample of
        ``sample_n`` points; sets them and returns them (K, d)."""
        mu = np.empty((self.k, self.d), dtype=np.float64)
        self._check(self._L.km_init_learned(self._h, net._h, int(sample_n), int(seed) & (2**64 - 1),
                                            mu.ctypes.data))
        return mu

    def step(self):
        e, e2 = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.km_step(self._h, ctypes.byref(e), ctypes.byref(e2)))
        return e.value, e2.value

    def run(self, max_iter: int, tol: float, want_labels: bool = True) -> dict:
        """km_run; labels are int32 (uint8 for a context with 1-byte labels)."""
        wide = want_labels and self.label_bytes == 4
        labels = np.empty(self.n, dtype=np.int32) if wide else None
        mu = np.empty((self.k, self.d), dtype=np.float64)
        it, e = ctypes.c_int32(), ctypes.c_double()
        s = self._check(self._L.km_run(self._h, int(max_iter), float(tol),
                                       labels.ctypes.data if wide else None,
                                       mu.ctypes.data, ctypes.byref(it), ctypes.byref(e)))
        if want_labels and not wide:
            labels = self.labels()
        return dict(labels=labels, centroids=mu, iters=it.value, E=e.value,
                    converged=(s == KM_OK))

    def run_logged(self, max_iter: int, tol: float, objective: bool = False, log=None) -> dict:
        """Lloyd's loop one step per host round trip, with one record per
        step (t, E, E^2, empty clusters, points re-checked and decided in
        FP64, wall ms, evaluations/s, and the objective of the step's labels
        when asked: one more pass).  Same stopping rule and results as run();
        ``log`` receives each record as a JSON line."""
        import json
        import time
        squared = self._e_mode == E_MODES["squared"]
        recs = []
        converged = False
        for t in range(1, int(max_iter) + 1):
            t0 = time.perf_counter()
            e, e2 = self.step()
            ms = 1e3 * (time.perf_counter() - t0)
            st = self.stats()
            rec = {"t": t, "E": e, "E2": e2, "empty": st["empty_clusters"], "flagged": st["flagged"],
                   "fp64_decided": st["fp64_decided"], "ms": ms,
                   "evals_per_s": self.n * self.k / (ms / 1e3) if ms > 0 else None}
            if objective:
                rec["objective"] = self.objective()
            recs.append(rec)
            if log is not None:
                log(json.dumps(rec))
            if (e2 if squared else e) < tol:
                converged = True
                break
        return dict(iters=len(recs), E=recs[-1]["E"] if recs else None, converged=converged,
                    centroids=self.centroids(), records=recs)

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

    # -- sharded steps (the points split over several contexts) --
    def grid_exponent(self) -> int:
        """The fixed-point grid exponent this context uses (km_grid_exponent)."""
        ex = ctypes.c_int32()
        self._check(self._L.km_grid_exponent(self._h, ctypes.byref(ex)))
        return ex.value

    def set_grid_exponent(self, ex: int):
        """Use the shards' common (maximum) grid exponent."""
        self._check(self._L.km_set_grid_exponent(self._h, int(ex)))

    def shard_totals(self) -> np.ndarray:
        """This shard's column totals after assign_async: (K*(d+1), 2) int64,
        the int128 (low word, high word) of every column."""
        out = np.empty((self.k * (self.d + 1), 2), dtype=np.int64)
        self._check(self._L.km_shard_totals(self._h, out.ctypes.data, KM_HOST))
        return out

    def shard_update(self, tables):
        """The update from the R shards' totals gathered in rank order:
        an (R, K*(d+1), 2) int64 array (host)."""
        t = np.ascontiguousarray(tables, dtype=np.int64)
        if t.ndim != 3 or t.shape[1:] != (self.k * (self.d + 1), 2):
            raise ValueError("tables must be (ranks, K*(d+1), 2) int64")
        self._check(self._L.km_shard_update(self._h, t.ctypes.data, int(t.shape[0]), KM_HOST))

    @property
    def stream_handle(self) -> int:
        return int(self._L.km_stream(self._h) or 0)

    def labels(self) -> np.ndarray:
        """The N labels (int32; uint8 for a context with 1-byte labels)."""
        if self.label_bytes == 1:
            out8 = np.empty(self.n, dtype=np.uint8)
            self._check(self._L.km_get_labels_u8(self._h, out8.ctypes.data, KM_HOST))
            return out8
        out = np.empty(self.n, dtype=np.int32)
        self._check(self._L.km_get_labels(self._h, out.ctypes.data, KM_HOST))
        return out

    def labels_host_into(self, tensor):
        """Copy labels into a host (e.g. pinned) torch tensor of N elements:
        int32, or uint8 for a context with 1-byte labels (no widening)."""
        import torch
        f = self._L.km_get_labels_u8 if tensor.dtype == torch.uint8 else self._L.km_get_labels
        self._check(f(self._h, tensor.data_ptr(), KM_HOST))

    def labels_into(self, tensor):
        """Copy labels into a CUDA torch tensor of N elements (int32, or uint8
        for a context with 1-byte labels)."""
        import torch
        f = self._L.km_get_labels_u8 if tensor.dtype == torch.uint8 else self._L.km_get_labels
        self._check(f(self._h, tensor.data_ptr(), KM_DEVICE_COPY))

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


class KMeansBatch:
    """Many independent clustering problems (instance i: N_i points of
    dimension d_i in 1..3, K_i clusters in 1..64) run by shared launches."""

    def __init__(self, n, d, k, *, e_mode: str = "norm", tie_rel: float = 1e-5, use_graph: bool = True,
                 stream=None):
        self._L = lib()
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.d = np.ascontiguousarray(d, dtype=np.int32)
        self.k = np.ascontiguousarray(k, dtype=np.int32)
        self.count = len(self.n)
        if not (len(self.d) == len(self.k) == self.count):
            raise ValueError("n, d and k must have one entry per instance")
        self.x_off = np.concatenate([[0], np.cumsum(self.n * self.d)]).astype(np.int64)
        self.lab_off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.mu_off = np.concatenate([[0], np.cumsum(self.k.astype(np.int64) * self.d)]).astype(np.int64)
        self.k_off = np.concatenate([[0], np.cumsum(self.k.astype(np.int64))]).astype(np.int64)
        opt = _Options()
        self._L.km_default_options(ctypes.byref(opt))
        opt.e_mode = E_MODES[e_mode]
        opt.use_graph = 1 if use_graph else 0
        opt.tie_rel = float(tie_rel)
        opt.stream = _current_stream() if stream is None else ctypes.c_void_p(
            stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream))
        h = ctypes.c_void_p()
        s = self._L.km_batch_create(ctypes.byref(h), self.count, self.n.ctypes.data, self.d.ctypes.data,
                                    self.k.ctypes.data, ctypes.byref(opt))
        self._h = h
        self._check(s)

    def _check(self, s: int) -> int:
        if s < 0:
            msg = self._L.km_batch_last_error(self._h).decode() if self._h else ""
            raise KMError(s, msg)
        return s

    def close(self):
        if getattr(self, "_h", None):
            self._L.km_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_points(self, xs):
        """xs: a list of (d_i, N_i) float32 arrays, or one flat float32 array
        (numpy, or a CUDA torch tensor) in the concatenated layout."""
        if isinstance(xs, (list, tuple)):
            flat = np.concatenate([np.ascontiguousarray(x, dtype=np.float32).reshape(-1) for x in xs])
        else:
            flat = xs
        if _is_torch(flat):
            if flat.numel() != int(self.x_off[-1]):
                raise ValueError("flat points of the wrong size")
            mem = KM_DEVICE_COPY if flat.is_cuda else KM_HOST
            ptr = flat.data_ptr()
        else:
            flat = np.ascontiguousarray(flat, dtype=np.float32)
            if flat.size != int(self.x_off[-1]):
                raise ValueError("flat points of the wrong size")
            mem, ptr = KM_HOST, flat.ctypes.data
        self._check(self._L.km_batch_set_points(self._h, ptr, mem))

    def set_init(self, mus):
        """mus: a list of (K_i, d_i) arrays or the flat concatenation."""
        if isinstance(mus, (list, tuple)):
            flat = np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1) for m in mus])
        else:
            flat = np.asarray(mus, dtype=np.float64).reshape(-1)
        flat = np.ascontiguousarray(flat)
        if flat.size != int(self.mu_off[-1]):
            raise ValueError("flat centroids of the wrong size")
        self._check(self._L.km_batch_set_init(self._h, flat.ctypes.data))

    def objective(self) -> np.ndarray:
        """Per instance sum_i ||x_i - mu_{z_i}||^2 of the current labels and
        centroids (FP64)."""
        out = np.empty(self.count, dtype=np.float64)
        self._check(self._L.km_batch_objective(self._h, out.ctypes.data))
        return out

    def set_shape(self, tile_points: int, threads: int):
        """Use a launch shape the tuner times, without timing."""
        self._check(self._L.km_batch_set_shape(self._h, int(tile_points), int(threads)))

    def tune(self, cache: str | None = None) -> tuple[int, int]:
        """Time the launch shapes and keep the fastest.  With a cache file
        (``cache`` or the KM_TUNE_CACHE environment variable), a shape chosen
        before for the same device and the same instance sizes is reused
        without timing, and a new choice is added to the file."""
        path = cache if cache is not None else os.environ.get("KM_TUNE_CACHE")
        key = None
        if path:
            import hashlib
            import json
            h = hashlib.sha256()
            h.update(_device_name().encode())
            for a in (self.n, self.d, self.k):
                h.update(np.ascontiguousarray(a).tobytes())
            key = h.hexdigest()[:32]
            try:
                with open(path) as f:
                    hit = json.load(f).get(key)
            except (OSError, ValueError):
                hit = None
            if hit:
                self.set_shape(int(hit[0]), int(hit[1]))
                return int(hit[0]), int(hit[1])
        t, th = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._L.km_batch_tune(self._h, ctypes.byref(t), ctypes.byref(th)))
        if key:
            import json
            try:
                with open(path) as f:
                    db = json.load(f)
            except (OSError, ValueError):
                db = {}
            db[key] = [t.value, th.value]
            tmp = f"{path}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(db, f)
            os.replace(tmp, path)
        return t.value, th.value

    def run(self, max_iter: int, tol: float, want_labels: bool = True) -> dict:
        labels = np.empty(int(self.lab_off[-1]), dtype=np.int32) if want_labels else None
        mu = np.empty(int(self.mu_off[-1]), dtype=np.float64)
        its = np.empty(self.count, dtype=np.int32)
        es = np.empty(self.count, dtype=np.float64)
        conv = np.empty(self.count, dtype=np.int32)
        s = self._check(self._L.km_batch_run(self._h, int(max_iter), float(tol),
                                             labels.ctypes.data if want_labels else None, mu.ctypes.data,
                                             its.ctypes.data, es.ctypes.data, conv.ctypes.data))
        return dict(labels=labels, centroids=mu, iters=its, E=es, converged=conv.astype(bool),
                    all_converged=(s == KM_OK))

    def counts(self) -> np.ndarray:
        out = np.empty(int(self.k_off[-1]), dtype=np.int64)
        self._check(self._L.km_batch_get_counts(self._h, out.ctypes.data))
        return out

    def info(self) -> dict:
        s = _BatchInfo()
        self._check(self._L.km_batch_get_info(self._h, ctypes.byref(s)))
        out = {f: getattr(s, f) for f, _ in _BatchInfo._fields_ if f != "tune_ms"}
        out["tune_ms"] = [float(s.tune_ms[q]) for q in range(s.tune_candidates)]
        return out

    # per-instance views of flat results
    def split_labels(self, flat):
        return [flat[self.lab_off[i]:self.lab_off[i + 1]] for i in range(self.count)]

    def split_centroids(self, flat):
        return [flat[self.mu_off[i]:self.mu_off[i + 1]].reshape(int(self.k[i]), int(self.d[i]))
                for i in range(self.count)]

    def split_counts(self, flat):
        return [flat[self.k_off[i]:self.k_off[i + 1]] for i in range(self.count)]


class SetNet:
    """The learned initialiser's set network (d in 1..3, K in 1..64)."""

    def __init__(self, d: int, k: int, stream=None):
        self._L = lib()
        self.d, self.k = int(d), int(k)
        h = ctypes.c_void_p()
        st = _current_stream() if stream is None else ctypes.c_void_p(
            stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream))
        s = self._L.km_setnet_create(ctypes.byref(h), self.d, self.k, st)
        self._h = h
        self._check(s)
        self.nparam = int(self._L.km_setnet_param_count(self._h))

    def _check(self, s: int) -> int:
        if s < 0:
            msg = self._L.km_setnet_last_error(self._h).decode() if self._h else ""
            raise KMError(s, msg)
        return s

    def close(self):
        if getattr(self, "_h", None):
            self._L.km_setnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, a, shape_tail):
        """(pointer, mem kind, keep-alive) of points [B][S][d] or targets."""
        if _is_torch(a):
            import torch
            if a.dtype != torch.float32:
                raise TypeError("float32 tensors only")
            a = a.contiguous()
            return a.data_ptr(), (KM_DEVICE_BORROW if a.is_cuda else KM_HOST), a
        a = np.ascontiguousarray(a, dtype=np.float32)
        return a.ctypes.data, KM_HOST, a

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32).reshape(-1)
        if flat.size != self.nparam:
            raise ValueError(f"need {self.nparam} parameters")
        self._check(self._L.km_setnet_set_params(self._h, flat.ctypes.data))

    def params(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        self._check(self._L.km_setnet_get_params(self._h, out.ctypes.data))
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        self._check(self._L.km_setnet_get_grads(self._h, out.ctypes.data))
        return out

    def loss_grad(self, x, t) -> float:
        B, S = int(x.shape[0]), int(x.shape[1])
        px, mx, kx = self._arr(x, None)
        pt, mt, kt = self._arr(t, None)
        if mx != mt:
            raise ValueError("points and targets must live in the same memory")
        loss = ctypes.c_float()
        self._check(self._L.km_setnet_loss_grad(self._h, px, pt, B, S, mx, ctypes.byref(loss)))
        return float(loss.value)

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._check(self._L.km_setnet_adam(self._h, lr, beta1, beta2, eps))

    def train_step(self, x, t, lr: float, want_loss: bool = True):
        B, S = int(x.shape[0]), int(x.shape[1])
        px, mx, kx = self._arr(x, None)
        pt, mt, kt = self._arr(t, None)
        loss = ctypes.c_float()
        self._check(self._L.km_setnet_train_step(self._h, px, pt, B, S, mx, float(lr),
                                                 ctypes.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def predict(self, x) -> np.ndarray:
        B, S = int(x.shape[0]), int(x.shape[1])
        px, mx, kx = self._arr(x, None)
        out = np.empty((B, self.k, self.d), dtype=np.float64)
        self._check(self._L.km_setnet_predict(self._h, px, B, S, mx, out.ctypes.data))
        return out


def _cuda_stream(t):
    import torch
    return torch.cuda.current_stream(t.device).cuda_stream


def sets_mean(x, set_stride: int | None = None, sets: int | None = None):
    """km_sets_mean on a CUDA float32 tensor x of B sets (B, S, d) -- or one
    set (S, d) repeated `sets` times with set_stride 0.  Returns (B, d)
    float64 means on the device."""
    import torch
    if x.dim() == 2:
        x = x.unsqueeze(0)
    x = x.contiguous()
    B, S, d = x.shape
    stride = S * d if set_stride is None else set_stride
    B = sets or B
    out = torch.empty((B, d), dtype=torch.float64, device=x.device)
    st = lib().km_sets_mean(x.data_ptr(), stride, B, S, d, out.data_ptr(), _cuda_stream(x))
    if st != KM_OK:
        raise KMError(st, "km_sets_mean")
    return out


def sets_rotate(x, R, center=None, transpose: bool = False, set_stride: int | None = None):
    """km_sets_rotate_f32/_f64 on CUDA tensors: out[b] = R_b (x[b] - c_b) + c_b
    (R_b^T with transpose).  x: (B, S, d) float32 or float64, or (S, d) with
    set_stride 0 for one set rotated B ways; R: (B, d, d) float64; center:
    (B, d) float64, (d,) for one centre for every set, or None (the origin)."""
    import torch
    if x.dim() == 2:
        x = x.unsqueeze(0)
        stride = 0
    else:
        stride = x.shape[1] * x.shape[2]
    x = x.contiguous()
    if set_stride is not None:
        stride = set_stride
    R = R.to(device=x.device, dtype=torch.float64).contiguous()
    B, d = R.shape[0], R.shape[1]
    S = x.shape[1]
    c_ptr, c_stride = None, 0
    if center is not None:
        center = center.to(device=x.device, dtype=torch.float64).contiguous()
        c_ptr = center.data_ptr()
        c_stride = d if center.dim() == 2 else 0
    out = torch.empty((B, S, d), dtype=x.dtype, device=x.device)
    fn = lib().km_sets_rotate_f64 if x.dtype == torch.float64 else lib().km_sets_rotate_f32
    st = fn(x.data_ptr(), stride, B, S, d, R.data_ptr(), c_ptr, c_stride, 1 if transpose else 0, out.data_ptr(),
            _cuda_stream(x))
    if st != KM_OK:
        raise KMError(st, "km_sets_rotate")
    return out
