"""Thin ctypes binding of libdkm (include/dkm.h), same function names.

Argument marshalling only: every step of the k-means path runs in the CUDA
kernels of libdkm.so.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; their data pointers are passed straight through (the library
detects host vs device memory itself).  There is no fallback: if
libdkm.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdkm.so")

DKM_OK, DKM_EINVAL, DKM_ENOMEM, DKM_ECUDA, DKM_ETIMEOUT, DKM_EINTERNAL = range(6)
DKM_ALGO_INDEXED, DKM_ALGO_BRUTE = 0, 1


class DkmError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        super().__init__(f"{func} -> {_STATUS.get(status, status)}: {msg}")


_STATUS = {0: "DKM_OK", 1: "DKM_EINVAL", 2: "DKM_ENOMEM", 3: "DKM_ECUDA", 4: "DKM_ETIMEOUT",
           5: "DKM_EINTERNAL"}


class dkm_options(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("cells_per_centroid", ctypes.c_float),
                ("algo", ctypes.c_int), ("early_stop", ctypes.c_int), ("profile", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class dkm_plan_info(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 3), ("cell", ctypes.c_float),
                ("origin", ctypes.c_float * 3), ("bucket_cap", ctypes.c_int),
                ("cells", ctypes.c_int64), ("index_bytes", ctypes.c_size_t),
                ("scratch_bytes", ctypes.c_size_t)]


class dkm_timings(ctypes.Structure):
    _fields_ = [("setup_ms", ctypes.c_float), ("iterations_ms", ctypes.c_float),
                ("search_ms", ctypes.c_float), ("assign_ms", ctypes.c_float),
                ("update_ms", ctypes.c_float), ("finalize_ms", ctypes.c_float),
                ("passes", ctypes.c_int)]


class dkm_stats(ctypes.Structure):
    _fields_ = [("evals_per_point", ctypes.c_double), ("candidates_per_tile", ctypes.c_double),
                ("fallback_tiles", ctypes.c_int64), ("stayed_tiles", ctypes.c_int64),
                ("grid_overflow", ctypes.c_int64),
                ("tiles", ctypes.c_int64), ("tile_level", ctypes.c_int), ("passes", ctypes.c_int),
                ("stayed_points", ctypes.c_int64)]


class dkm_tuning(ctypes.Structure):
    _fields_ = [("cells_per_centroid", ctypes.c_float), ("tile_cut_div", ctypes.c_int),
                ("row_filter_min", ctypes.c_int), ("sort_max", ctypes.c_int),
                ("tile_group", ctypes.c_int), ("stay_test", ctypes.c_int),
                ("ms_per_pass", ctypes.c_float),
                ("ms_per_pass_before", ctypes.c_float), ("trials", ctypes.c_int),
                ("from_cache", ctypes.c_int)]


class dkm_peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int), ("sm_clock_mhz", ctypes.c_int),
                ("fp32_fma_tflops", ctypes.c_double), ("fp32x2_fma_tflops", ctypes.c_double),
                ("scalar_ms", ctypes.c_float), ("packed_ms", ctypes.c_float)]


_lib: Optional[ctypes.CDLL] = None

# (name, restype, argtypes); "status" functions return dkm_status
_SIGS = [
    ("dkm_default_options", None, [ctypes.POINTER(dkm_options)]),
    ("dkm_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("dkm_last_error", ctypes.c_char_p, []),
    ("dkm_plan", ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.POINTER(dkm_options),
                                ctypes.POINTER(dkm_plan_info)]),
    ("dkm_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(dkm_options)]),
    ("dkm_setup", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("dkm_assign", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64)]),
    ("dkm_update", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    ("dkm_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_double)]),
    ("dkm_fit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(dkm_options)]),
    ("dkm_create_batched", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.POINTER(dkm_options)]),
    ("dkm_run_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    ("dkm_fit_batched", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(dkm_options)]),
    ("dkm_get_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dkm_tuning)]),
    ("dkm_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dkm_tuning)]),
    ("dkm_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(dkm_tuning)]),
    ("dkm_query_memory", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(ctypes.c_size_t)]),
    ("dkm_get_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dkm_plan_info)]),
    ("dkm_last_timings", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dkm_timings)]),
    ("dkm_last_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dkm_stats)]),
    ("dkm_destroy", None, [ctypes.c_void_p]),
    ("dkm_lloyd_step_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_void_p]),
    ("dkm_soft_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("dkm_soft_backward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    ("dkm_selftest_wait", ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    ("dkm_hard_sse", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    ("dkm_hard_sse_backward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    ("dkm_device_peaks", ctypes.c_int, [ctypes.POINTER(dkm_peaks), ctypes.c_void_p]),
    ("dkm_soft_temperature", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_void_p]),
]

DKM_NOALLOC_MAX_K = 65536


def lib() -> ctypes.CDLL:
    """The loaded libdkm.so; raises if it was never built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdkm.so not found at {LIB_PATH}: run "
                              "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, func: str) -> None:
    if status != DKM_OK:
        raise DkmError(status, func, lib().dkm_last_error().decode())


def _arr(x: Any, dtype: str, numel: Optional[int] = None, name: str = "array"):
    """(pointer, keep-alive) of a contiguous torch tensor or numpy array."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):   # torch.Tensor
        want = {"float32": "torch.float32", "int32": "torch.int32", "int64": "torch.int64",
                "float64": "torch.float64"}[dtype]
        if str(x.dtype) != want:
            raise TypeError(f"{name} must be {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if numel is not None and x.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements, got {x.numel()}")
        return ctypes.c_void_p(x.data_ptr()), x
    a = x
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous {dtype} numpy array or torch tensor")
    if numel is not None and a.size != numel:
        raise ValueError(f"{name} must have {numel} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data), a


def dkm_default_options(**kw) -> dkm_options:
    o = dkm_options()
    lib().dkm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def dkm_status_string(s: int) -> str:
    return lib().dkm_status_string(int(s)).decode()


def dkm_last_error() -> str:
    return lib().dkm_last_error().decode()


def dkm_plan(n: int, d: int, k: int, bbox_lo, bbox_hi,
             opts: Optional[dkm_options] = None) -> dkm_plan_info:
    lo = np.ascontiguousarray(bbox_lo, dtype=np.float32)
    hi = np.ascontiguousarray(bbox_hi, dtype=np.float32)
    if lo.size != d or hi.size != d:
        raise ValueError("bbox_lo / bbox_hi must have d entries")
    out = dkm_plan_info()
    _check(lib().dkm_plan(n, d, k, lo.ctypes.data, hi.ctypes.data,
                          ctypes.byref(opts) if opts is not None else None, ctypes.byref(out)),
           "dkm_plan")
    return out


class Context:
    """Owns one dkm_ctx handle (dkm_destroy on close / garbage collection)."""

    def __init__(self, handle: int, n: int, d: int, k: int, B: int = 1):
        self.handle = ctypes.c_void_p(handle)
        self.n, self.d, self.k, self.B = n, d, k, B

    def close(self) -> None:
        if self.handle and self.handle.value:
            lib().dkm_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dkm_create(points, n: int, d: int, k: int, opts: Optional[dkm_options] = None) -> Context:
    p, _keep = _arr(points, "float32", n * d, "points")
    h = ctypes.c_void_p()
    _check(lib().dkm_create(ctypes.byref(h), p, n, d, k,
                            ctypes.byref(opts) if opts is not None else None), "dkm_create")
    return Context(h.value, n, d, k)


def dkm_setup(ctx: Context, points) -> None:
    p, _keep = _arr(points, "float32", ctx.n * ctx.d, "points")
    _check(lib().dkm_setup(ctx.handle, p), "dkm_setup")


def dkm_assign(ctx: Context, centroids, labels=None) -> Tuple[float, int]:
    c, _k1 = _arr(centroids, "float32", ctx.k * ctx.d, "centroids")
    lab, _k2 = _arr(labels, "int32", ctx.n, "labels")
    sse = ctypes.c_double()
    chg = ctypes.c_int64()
    _check(lib().dkm_assign(ctx.handle, c, lab, ctypes.byref(sse), ctypes.byref(chg)),
           "dkm_assign")
    return sse.value, chg.value


def dkm_update(ctx: Context, labels, centroids_inout, counts=None) -> None:
    lab, _k1 = _arr(labels, "int32", ctx.n, "labels")
    c, _k2 = _arr(centroids_inout, "float32", ctx.k * ctx.d, "centroids_inout")
    cnt, _k3 = _arr(counts, "int32", ctx.k, "counts")
    _check(lib().dkm_update(ctx.handle, lab, c, cnt), "dkm_update")


def dkm_run(ctx: Context, init_centroids, max_iter: int, centroids_out=None,
            labels_out=None) -> Tuple[int, float]:
    i, _k1 = _arr(init_centroids, "float32", ctx.k * ctx.d, "init_centroids")
    c, _k2 = _arr(centroids_out, "float32", ctx.k * ctx.d, "centroids_out")
    lab, _k3 = _arr(labels_out, "int32", ctx.n, "labels_out")
    it = ctypes.c_int()
    sse = ctypes.c_double()
    _check(lib().dkm_run(ctx.handle, i, int(max_iter), c, lab, ctypes.byref(it),
                         ctypes.byref(sse)), "dkm_run")
    return it.value, sse.value


def dkm_fit(points, n: int, d: int, k: int, init_centroids, max_iter: int, centroids_out=None,
            labels_out=None, opts: Optional[dkm_options] = None) -> Tuple[int, float]:
    p, _k0 = _arr(points, "float32", n * d, "points")
    i, _k1 = _arr(init_centroids, "float32", k * d, "init_centroids")
    c, _k2 = _arr(centroids_out, "float32", k * d, "centroids_out")
    lab, _k3 = _arr(labels_out, "int32", n, "labels_out")
    it = ctypes.c_int()
    sse = ctypes.c_double()
    _check(lib().dkm_fit(p, n, d, k, i, int(max_iter), c, lab, ctypes.byref(it),
                         ctypes.byref(sse), ctypes.byref(opts) if opts is not None else None),
           "dkm_fit")
    return it.value, sse.value


def _batch_sizes(offsets, ks):
    off = np.ascontiguousarray(np.asarray(offsets), dtype=np.int64)
    kv = np.ascontiguousarray(np.asarray(ks), dtype=np.int32)
    if off.ndim != 1 or kv.ndim != 1 or off.size != kv.size + 1:
        raise ValueError("offsets must have len(ks) + 1 entries")
    return off, kv


def dkm_create_batched(points, offsets, d: int, ks,
                       opts: Optional[dkm_options] = None) -> Context:
    """Context over B clouds: points[offsets[b]:offsets[b+1]] with ks[b] clusters."""
    off, kv = _batch_sizes(offsets, ks)
    n, B, K = int(off[-1]), int(kv.size), int(kv.sum())
    p, _keep = _arr(points, "float32", n * d, "points")
    h = ctypes.c_void_p()
    _check(lib().dkm_create_batched(ctypes.byref(h), p, off.ctypes.data, B, d, kv.ctypes.data,
                                    ctypes.byref(opts) if opts is not None else None),
           "dkm_create_batched")
    return Context(h.value, n, d, K, B)


def dkm_run_batched(ctx: Context, init_centroids, max_iter: int, centroids_out=None,
                    labels_out=None) -> Tuple[np.ndarray, np.ndarray]:
    """Lloyd on every cloud; returns (passes per cloud, final SSE per cloud)."""
    i, _k1 = _arr(init_centroids, "float32", ctx.k * ctx.d, "init_centroids")
    c, _k2 = _arr(centroids_out, "float32", ctx.k * ctx.d, "centroids_out")
    lab, _k3 = _arr(labels_out, "int32", ctx.n, "labels_out")
    it = np.zeros(ctx.B, np.int32)
    sse = np.zeros(ctx.B, np.float64)
    _check(lib().dkm_run_batched(ctx.handle, i, int(max_iter), c, lab, it.ctypes.data,
                                 sse.ctypes.data), "dkm_run_batched")
    return it, sse


def dkm_fit_batched(points, offsets, d: int, ks, init_centroids, max_iter: int,
                    centroids_out=None, labels_out=None,
                    opts: Optional[dkm_options] = None) -> Tuple[np.ndarray, np.ndarray]:
    off, kv = _batch_sizes(offsets, ks)
    n, B, K = int(off[-1]), int(kv.size), int(kv.sum())
    p, _k0 = _arr(points, "float32", n * d, "points")
    i, _k1 = _arr(init_centroids, "float32", K * d, "init_centroids")
    c, _k2 = _arr(centroids_out, "float32", K * d, "centroids_out")
    lab, _k3 = _arr(labels_out, "int32", n, "labels_out")
    it = np.zeros(B, np.int32)
    sse = np.zeros(B, np.float64)
    _check(lib().dkm_fit_batched(p, off.ctypes.data, B, d, kv.ctypes.data, i, int(max_iter), c,
                                 lab, it.ctypes.data, sse.ctypes.data,
                                 ctypes.byref(opts) if opts is not None else None),
           "dkm_fit_batched")
    return it, sse


def dkm_get_tuning(ctx: Context) -> dkm_tuning:
    out = dkm_tuning()
    _check(lib().dkm_get_tuning(ctx.handle, ctypes.byref(out)), "dkm_get_tuning")
    return out


def dkm_set_tuning(ctx: Context, tuning: Optional[dkm_tuning] = None, **kw) -> None:
    t = tuning if tuning is not None else dkm_get_tuning(ctx)
    for k, v in kw.items():
        if not hasattr(t, k):
            raise AttributeError(k)
        setattr(t, k, v)
    _check(lib().dkm_set_tuning(ctx.handle, ctypes.byref(t)), "dkm_set_tuning")


def dkm_autotune(ctx: Context, init_centroids, passes: int = 3,
                 use_cache: bool = True) -> dkm_tuning:
    """Time index settings on this context and keep the fastest."""
    i, _k1 = _arr(init_centroids, "float32", ctx.k * ctx.d, "init_centroids")
    out = dkm_tuning()
    _check(lib().dkm_autotune(ctx.handle, i, int(passes), 1 if use_cache else 0,
                              ctypes.byref(out)), "dkm_autotune")
    return out


def dkm_query_memory(ctx: Context) -> Tuple[int, int]:
    a = ctypes.c_size_t()
    b = ctypes.c_size_t()
    _check(lib().dkm_query_memory(ctx.handle, ctypes.byref(a), ctypes.byref(b)),
           "dkm_query_memory")
    return a.value, b.value


def dkm_get_plan(ctx: Context) -> dkm_plan_info:
    out = dkm_plan_info()
    _check(lib().dkm_get_plan(ctx.handle, ctypes.byref(out)), "dkm_get_plan")
    return out


def dkm_last_timings(ctx: Context) -> dkm_timings:
    out = dkm_timings()
    _check(lib().dkm_last_timings(ctx.handle, ctypes.byref(out)), "dkm_last_timings")
    return out


def dkm_last_stats(ctx: Context) -> dkm_stats:
    out = dkm_stats()
    _check(lib().dkm_last_stats(ctx.handle, ctypes.byref(out)), "dkm_last_stats")
    return out


def dkm_destroy(ctx: Context) -> None:
    ctx.close()


def dkm_soft_forward(points, offsets, B: int, d: int, k: int, init_centroids, T: int, tau, ckpt,
                     loss, stream: int = 0, stats=None, norms=None) -> None:
    """Soft k-means loss of B clouds; fills ckpt ((T+1) x B x k x d) and loss (B), and
    optionally the per-step statistics stats (T x 2 x n_total) and norms (T x B x k)."""
    off, _k0 = _arr(offsets, "int64", B + 1, "offsets")
    n_total = int(offsets[-1])
    p, _k1 = _arr(points, "float32", n_total * d, "points")
    c0, _k2 = _arr(init_centroids, "float32", B * k * d, "init_centroids")
    tv, _k3 = _arr(tau, "float32", B, "tau")
    ck, _k4 = _arr(ckpt, "float32", (T + 1) * B * k * d, "ckpt")
    ls, _k5 = _arr(loss, "float64", B, "loss")
    sv, _k6 = _arr(stats, "float32", T * 2 * n_total, "stats")
    nv, _k7 = _arr(norms, "float32", T * B * k, "norms")
    _check(lib().dkm_soft_forward(p, off, B, d, k, c0, int(T), tv, ck, ls, sv, nv,
                                  ctypes.c_void_p(stream or 0)), "dkm_soft_forward")


def dkm_soft_backward(points, offsets, B: int, d: int, k: int, ckpt, T: int, tau, dloss,
                      grad_points, grad_init, stream: int = 0, stats=None, norms=None) -> None:
    off, _k0 = _arr(offsets, "int64", B + 1, "offsets")
    n_total = int(offsets[-1])
    p, _k1 = _arr(points, "float32", n_total * d, "points")
    ck, _k2 = _arr(ckpt, "float32", (T + 1) * B * k * d, "ckpt")
    tv, _k3 = _arr(tau, "float32", B, "tau")
    dl, _k4 = _arr(dloss, "float64", B, "dloss")
    gp, _k5 = _arr(grad_points, "float32", n_total * d, "grad_points")
    gi, _k6 = _arr(grad_init, "float32", B * k * d, "grad_init")
    sv, _k7 = _arr(stats, "float32", T * 2 * n_total, "stats")
    nv, _k8 = _arr(norms, "float32", T * B * k, "norms")
    _check(lib().dkm_soft_backward(p, off, B, d, k, ck, int(T), tv, dl, sv, nv, gp, gi,
                                   ctypes.c_void_p(stream or 0)), "dkm_soft_backward")


def dkm_hard_sse(points, offsets, B: int, d: int, k: int, centroids, labels=None, loss=None,
                 grad_points=None, grad_centroids=None, stream: int = 0) -> None:
    off, _k0 = _arr(offsets, "int64", B + 1, "offsets")
    n_total = int(offsets[-1])
    p, _k1 = _arr(points, "float32", n_total * d, "points")
    c, _k2 = _arr(centroids, "float32", B * k * d, "centroids")
    lab, _k3 = _arr(labels, "int32", n_total, "labels")
    ls, _k4 = _arr(loss, "float64", B, "loss")
    gp, _k5 = _arr(grad_points, "float32", n_total * d, "grad_points")
    gc, _k6 = _arr(grad_centroids, "float32", B * k * d, "grad_centroids")
    _check(lib().dkm_hard_sse(p, off, B, d, k, c, lab, ls, gp, gc, ctypes.c_void_p(stream or 0)),
           "dkm_hard_sse")


def dkm_hard_sse_backward(points, offsets, B: int, d: int, k: int, centroids, labels, dloss,
                          grad_points=None, grad_centroids=None, stream: int = 0) -> None:
    off, _k0 = _arr(offsets, "int64", B + 1, "offsets")
    n_total = int(offsets[-1])
    p, _k1 = _arr(points, "float32", n_total * d, "points")
    c, _k2 = _arr(centroids, "float32", B * k * d, "centroids")
    lab, _k3 = _arr(labels, "int32", n_total, "labels")
    dl, _k4 = _arr(dloss, "float64", B, "dloss")
    gp, _k5 = _arr(grad_points, "float32", n_total * d, "grad_points")
    gc, _k6 = _arr(grad_centroids, "float32", B * k * d, "grad_centroids")
    _check(lib().dkm_hard_sse_backward(p, off, B, d, k, c, lab, dl, gp, gc,
                                       ctypes.c_void_p(stream or 0)), "dkm_hard_sse_backward")


def dkm_soft_temperature(points, offsets, B: int, d: int, tau, frac: float = 0.01,
                         stream: int = 0) -> None:
    """tau[b] = frac x squared bounding-box diagonal of cloud b (into tau, B floats)."""
    off, _k0 = _arr(offsets, "int64", B + 1, "offsets")
    n_total = int(offsets[-1])
    p, _k1 = _arr(points, "float32", n_total * d, "points")
    tv, _k2 = _arr(tau, "float32", B, "tau")
    _check(lib().dkm_soft_temperature(p, off, B, d, float(frac), tv,
                                      ctypes.c_void_p(stream or 0)), "dkm_soft_temperature")


def dkm_device_peaks(stream: int = 0) -> dkm_peaks:
    """Measured FP32 FMA throughput (scalar and packed f32x2) and SM count."""
    p = dkm_peaks()
    _check(lib().dkm_device_peaks(ctypes.byref(p), ctypes.c_void_p(stream or 0)),
           "dkm_device_peaks")
    return p


def dkm_selftest_wait() -> float:
    """Run the self-test of the radix sort's bounded wait (one pass whose
    awaited count is never published); raises unless the wait gave up by
    itself and reported it.  Returns the pass's wall time in seconds."""
    sec = ctypes.c_double()
    _check(lib().dkm_selftest_wait(ctypes.byref(sec)), "dkm_selftest_wait")
    return sec.value


def dkm_lloyd_step_noalloc(points, n: int, d: int, k: int, centroids, centroids_out, labels,
                           stream: int = 0) -> float:
    """One brute-force Lloyd step that allocates no device memory (for
    callers that cannot call cudaMalloc).  All arrays are device tensors;
    returns the SSE of the labels against the input centroids."""
    p, _k0 = _arr(points, "float32", n * d, "points")
    c, _k1 = _arr(centroids, "float32", k * d, "centroids")
    co, _k2 = _arr(centroids_out, "float32", k * d, "centroids_out")
    lab, _k3 = _arr(labels, "int32", n, "labels")
    sse = ctypes.c_double()
    _check(lib().dkm_lloyd_step_noalloc(p, n, d, k, c, co, lab, ctypes.byref(sse),
                                        ctypes.c_void_p(stream or 0)), "dkm_lloyd_step_noalloc")
    return sse.value
